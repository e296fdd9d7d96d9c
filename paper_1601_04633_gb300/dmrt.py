"""Python binding of libdmrt.so (the C ABI of include/dmrt.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. PyTorch provides the device workspace (its caching allocator) and
the CUDA stream. There is no CPU fallback: if the library is missing or no GPU
is present, the calls raise.

Low-level functions carry the C names (``dmrt_create``, ``dmrt_step``, ...);
``Cavity2D`` bundles them with a torch-owned workspace.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# DMRT_LIBRARY=bounds_check selects the bounds-checked build (every computed
# index checked in the kernels; a violation is reported as DMRT_E_BOUNDS).
LIB_PATH = os.path.join(_PKG, "_lib", "libdmrt_bc.so" if os.environ.get("DMRT_LIBRARY") == "bounds_check"
                        else "libdmrt.so")

DMRT_OK = 0
DMRT_E_ARG = -1
DMRT_E_UNSTABLE = -2
DMRT_E_CUDA = -3
DMRT_E_DIVERGED = -4
DMRT_E_TIMEOUT = -5
DMRT_E_SPACE = -6
DMRT_E_STATE = -7
DMRT_E_BOUNDS = -8
DMRT_FP32, DMRT_FP16, DMRT_BF16, DMRT_MIXED, DMRT_THETA32 = 0, 1, 2, 3, 4
DMRT_WALL_FIXED, DMRT_WALL_ADIABATIC = 0, 1
DMRT_KERNEL_AUTO, DMRT_KERNEL_DIRECT, DMRT_KERNEL_TMA, DMRT_KERNEL_CLUSTER = 0, 1, 2, 3
DMRT_ROUND_NEAREST, DMRT_ROUND_STOCHASTIC, DMRT_ROUND_AUTO = 0, 1, 2
DMRT_NOALLOC_MAX_NY = 8192
# Device plane order of the population buffers: entry d is the index, in the host
# order f1..f9, g1..g5 (paper numbering), of device plane d.
DEVICE_PLANE_ORDER = (0, 1, 3, 9, 10, 12, 2, 5, 6, 11, 4, 7, 8, 13)


def device_pitch(nx: int) -> int:
    """Elements per row of a device population plane."""
    return (int(nx) + 127) // 128 * 128

_ERRNAMES = {-1: "DMRT_E_ARG", -2: "DMRT_E_UNSTABLE", -3: "DMRT_E_CUDA", -4: "DMRT_E_DIVERGED",
             -5: "DMRT_E_TIMEOUT", -6: "DMRT_E_SPACE", -7: "DMRT_E_STATE", -8: "DMRT_E_BOUNDS"}


class DmrtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
        ("alpha", ctypes.c_double), ("Ma", ctypes.c_double),
        ("theta_hot", ctypes.c_double), ("theta_cold", ctypes.c_double),
        ("theta_ref", ctypes.c_double), ("theta_init", ctypes.c_double),
        ("left_wall", ctypes.c_int32), ("right_wall", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("kernel", ctypes.c_int32),
        ("nu_capacity", ctypes.c_int64),
        ("tma_rows", ctypes.c_int32), ("tma_stages", ctypes.c_int32),
        ("tma_npt", ctypes.c_int32), ("rounding", ctypes.c_int32),
    ]


class Consts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "nu", "alpha", "s_e", "s_nu", "s_q", "s_eps", "sig_k", "sig_e", "sig_nu",
        "a", "gbeta", "abb", "Ma", "fo_per_step")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Launch(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("tma_npt", ctypes.c_int32), ("tma_rows", ctypes.c_int32),
                ("tma_stages", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32), ("smem_bytes", ctypes.c_int64),
                ("graph_steps", ctypes.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class BatchOpts(ctypes.Structure):
    _fields_ = [("tma_npt", ctypes.c_int32), ("tma_rows", ctypes.c_int32),
                ("tma_stages", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("group_bytes", ctypes.c_int64), ("steps_per_launch", ctypes.c_int32),
                ("tensor_store", ctypes.c_int32), ("strip_fill", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()

# Exported symbols and their signatures: (restype, argtypes).
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)
SIGNATURES = {
    "dmrt_default_params": (None, [ctypes.POINTER(Params)]),
    "dmrt_derive": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(Consts)]),
    "dmrt_workspace_size": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_create": (ctypes.c_int, [ctypes.POINTER(Params), _DP, _VP, ctypes.c_size_t, _VP,
                                   ctypes.POINTER(_VP)]),
    "dmrt_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "dmrt_check": (ctypes.c_int, [_VP]),
    "dmrt_steps_done": (ctypes.c_int64, [_VP]),
    "dmrt_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int]),
    "dmrt_nusselt": (ctypes.c_int, [_VP, _DP, _DP, _DP, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int64)]),
    "dmrt_set_wall_profiles": (ctypes.c_int, [_VP, _DP, _DP]),
    "dmrt_nusselt_flux": (ctypes.c_int, [_VP, _DP, _DP]),
    "dmrt_energy": (ctypes.c_int, [_VP, _DP, _DP]),
    "dmrt_get_consts": (ctypes.c_int, [_VP, ctypes.POINTER(Consts)]),
    "dmrt_get_launch": (ctypes.c_int, [_VP, ctypes.POINTER(Launch)]),
    "dmrt_choose_launch": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 4),
    "dmrt_get_state": (ctypes.c_int, [_VP, _FP]),
    "dmrt_set_state": (ctypes.c_int, [_VP, _FP]),
    "dmrt_save": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_probe_bounded_wait": (ctypes.c_int, [ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_int64)]),
    "dmrt_load": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "dmrt_step_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), _VP, _VP, _VP, _VP, _VP, _VP]),
    "dmrt_adjoint_workspace_size": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_adjoint_workspace_min": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_adjoint_workspace_all": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_adjoint": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_size_t, _DP, _DP, _DP]),
    "dmrt_last_error": (ctypes.c_char_p, [_VP]),
    "dmrt_slab_workspace_size": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_create_slab": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_int32, _DP, _VP,
                                        ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "dmrt_slab_halo_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_slab_pack": (ctypes.c_int, [_VP, _VP, _VP]),
    "dmrt_slab_unpack": (ctypes.c_int, [_VP, _VP, _VP]),
    "dmrt_slab_step": (ctypes.c_int, [_VP, _VP, _VP]),
    "dmrt_batch_workspace_size": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "dmrt_batch_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32, ctypes.POINTER(_DP),
                                         ctypes.POINTER(BatchOpts), _VP, ctypes.c_size_t, _VP,
                                         ctypes.POINTER(_VP)]),
    "dmrt_batch_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "dmrt_batch_check": (ctypes.c_int, [_VP]),
    "dmrt_batch_size": (ctypes.c_int32, [_VP]),
    "dmrt_batch_group_count": (ctypes.c_int32, [_VP]),
    "dmrt_batch_context": (_VP, [_VP, ctypes.c_int32]),
    "dmrt_batch_get_launch": (ctypes.c_int, [_VP, ctypes.POINTER(Launch)]),
    "dmrt_batch_last_error": (ctypes.c_char_p, [_VP]),
    "dmrt_batch_destroy": (None, [_VP]),
    "dmrt_destroy": (None, [_VP]),
}


def load():
    """Load libdmrt.so (built by ``paper_1601_04633_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_1601_04633_gb300.build` "
                    "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc, handle=None):
    if rc != DMRT_OK:
        msg = load().dmrt_last_error(handle)
        raise DmrtError(rc, msg.decode() if msg else "")
    return rc


def _check_batch(rc, b=None):
    if rc != DMRT_OK:
        msg = load().dmrt_batch_last_error(b)
        raise DmrtError(rc, msg.decode() if msg else "")
    return rc


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


# ---- same-name wrappers ------------------------------------------------------

def dmrt_default_params() -> Params:
    p = Params()
    load().dmrt_default_params(ctypes.byref(p))
    return p


def dmrt_derive(p: Params) -> Consts:
    k = Consts()
    _check(load().dmrt_derive(ctypes.byref(p), ctypes.byref(k)))
    return k


def dmrt_workspace_size(p: Params) -> int:
    n = ctypes.c_size_t()
    _check(load().dmrt_workspace_size(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def dmrt_create(p: Params, theta0, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    """theta0: None or a float64 host array [ny][nx] (C order)."""
    h = _VP()
    th = None
    if theta0 is not None:
        th = np.ascontiguousarray(theta0, dtype=np.float64)
        if th.size != p.nx * p.ny:
            raise ValueError("theta0 must hold nx * ny values")
    _check(load().dmrt_create(ctypes.byref(p), _dptr(th), _VP(workspace_ptr), workspace_bytes,
                              _VP(stream_ptr), ctypes.byref(h)))
    return h


def dmrt_step(h, n: int):
    _check(load().dmrt_step(h, int(n)), h)


def dmrt_check(h):
    _check(load().dmrt_check(h), h)


def dmrt_steps_done(h) -> int:
    return load().dmrt_steps_done(h)


def dmrt_fields(h, u_ptr, v_ptr, theta_ptr, on_device: bool):
    _check(load().dmrt_fields(h, _VP(u_ptr), _VP(v_ptr), _VP(theta_ptr), int(bool(on_device))), h)


def dmrt_nusselt(h, ny: int, cap: int = 0):
    """Returns (nu_mean, nu_local[ny], series[count]) as numpy float64."""
    mean = ctypes.c_double()
    local = np.zeros(ny)
    series = np.zeros(max(cap, 0))
    count = ctypes.c_int64()
    _check(load().dmrt_nusselt(h, ctypes.byref(mean), _dptr(local),
                               _dptr(series) if cap > 0 else None, int(cap), ctypes.byref(count)), h)
    return mean.value, local, series[: count.value]


def dmrt_set_wall_profiles(h, hot=None, cold=None):
    hp = None if hot is None else np.ascontiguousarray(hot, dtype=np.float64)
    cp = None if cold is None else np.ascontiguousarray(cold, dtype=np.float64)
    _check(load().dmrt_set_wall_profiles(h, _dptr(hp), _dptr(cp)), h)


def dmrt_energy(h) -> tuple:
    """(sum of theta over the cavity, heat the next streaming brings in across
    the fixed-temperature walls), float64 sums taken on the GPU."""
    th = ctypes.c_double()
    win = ctypes.c_double()
    _check(load().dmrt_energy(h, ctypes.byref(th), ctypes.byref(win)), h)
    return th.value, win.value


def dmrt_get_consts(h) -> Consts:
    k = Consts()
    _check(load().dmrt_get_consts(h, ctypes.byref(k)), h)
    return k


def dmrt_get_launch(h) -> Launch:
    k = Launch()
    _check(load().dmrt_get_launch(h, ctypes.byref(k)), h)
    return k


def dmrt_choose_launch(p: Params, sms: int) -> tuple:
    """(kernel, nodes per thread, rows, stages) that parameters p run with on a
    GPU with `sms` SMs (host logic; the tile is 0, 0, 0 for the direct kernel)."""
    out = [ctypes.c_int32() for _ in range(4)]
    _check(load().dmrt_choose_launch(ctypes.byref(p), sms, *[ctypes.byref(x) for x in out]), None)
    return tuple(x.value for x in out)


def dmrt_get_state(h, nx: int, ny: int) -> np.ndarray:
    out = np.empty((14, ny, nx), dtype=np.float32)
    _check(load().dmrt_get_state(h, out.ctypes.data_as(_FP)), h)
    return out


def dmrt_set_state(h, state):
    a = np.ascontiguousarray(state, dtype=np.float32)
    _check(load().dmrt_set_state(h, a.ctypes.data_as(_FP)), h)


def dmrt_save(h) -> bytes:
    """Checkpoint of the context (state in its stored representation, step
    counters, wall profiles, Nusselt ring) as bytes."""
    need = ctypes.c_size_t(0)
    _check(load().dmrt_save(h, None, 0, ctypes.byref(need)), h)
    buf = ctypes.create_string_buffer(need.value)
    _check(load().dmrt_save(h, ctypes.cast(buf, _VP), need.value, ctypes.byref(need)), h)
    return buf.raw[: need.value]


def dmrt_load(h, blob: bytes):
    b = bytes(blob)
    _check(load().dmrt_load(h, ctypes.cast(ctypes.c_char_p(b), _VP), len(b)), h)


def dmrt_step_noalloc(p: Params, src_ptr: int, dst_ptr: int, nu_mean_ptr: int, stream_ptr: int,
                      hot_ptr: int = 0, cold_ptr: int = 0):
    """One step between caller-owned device buffers, with no device allocation."""
    _check(load().dmrt_step_noalloc(ctypes.byref(p), _VP(src_ptr), _VP(dst_ptr), _VP(hot_ptr or None),
                                    _VP(cold_ptr or None), _VP(nu_mean_ptr or None), _VP(stream_ptr)))


def dmrt_destroy(h):
    load().dmrt_destroy(h)


def dmrt_slab_workspace_size(p: Params, rows: int) -> int:
    n = ctypes.c_size_t()
    _check(load().dmrt_slab_workspace_size(ctypes.byref(p), int(rows), ctypes.byref(n)))
    return n.value


def dmrt_create_slab(p: Params, y0: int, rows: int, theta0, workspace_ptr: int, workspace_bytes: int,
                     stream_ptr: int):
    """Context of rows y0 .. y0 + rows - 1 of cavity p; theta0: None or [rows][nx] float64."""
    h = _VP()
    th = None
    if theta0 is not None:
        th = np.ascontiguousarray(theta0, dtype=np.float64)
        if th.size != p.nx * rows:
            raise ValueError("theta0 must hold nx * rows values")
    _check(load().dmrt_create_slab(ctypes.byref(p), int(y0), int(rows), _dptr(th), _VP(workspace_ptr),
                                   workspace_bytes, _VP(stream_ptr), ctypes.byref(h)))
    return h


def dmrt_slab_halo_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(load().dmrt_slab_halo_bytes(h, ctypes.byref(n)), h)
    return n.value


def dmrt_slab_pack(h, to_below_ptr: int, to_above_ptr: int):
    _check(load().dmrt_slab_pack(h, _VP(to_below_ptr or None), _VP(to_above_ptr or None)), h)


def dmrt_slab_unpack(h, from_below_ptr: int, from_above_ptr: int):
    _check(load().dmrt_slab_unpack(h, _VP(from_below_ptr or None), _VP(from_above_ptr or None)), h)


def dmrt_slab_step(h, to_below_ptr: int, to_above_ptr: int):
    _check(load().dmrt_slab_step(h, _VP(to_below_ptr or None), _VP(to_above_ptr or None)), h)


# ---- convenience object --------------------------------------------------------

def make_params(nx, ny, Ra, Pr, alpha=0.1, Ma=0.0, theta_hot=0.5, theta_cold=-0.5,
                theta_ref=None, theta_init=0.0, left_wall=DMRT_WALL_FIXED,
                right_wall=DMRT_WALL_FIXED, storage=DMRT_FP32, nu_capacity=1 << 20,
                kernel=DMRT_KERNEL_AUTO, tma_rows=0, tma_stages=0, tma_npt=0,
                rounding=DMRT_ROUND_AUTO) -> Params:
    p = dmrt_default_params()
    p.nx, p.ny, p.Ra, p.Pr, p.alpha, p.Ma = int(nx), int(ny), float(Ra), float(Pr), float(alpha), float(Ma)
    p.theta_hot, p.theta_cold = float(theta_hot), float(theta_cold)
    p.theta_ref = 0.5 * (theta_hot + theta_cold) if theta_ref is None else float(theta_ref)
    p.theta_init = float(theta_init)
    p.left_wall, p.right_wall, p.storage = int(left_wall), int(right_wall), int(storage)
    p.nu_capacity = int(nu_capacity)
    p.kernel, p.tma_rows, p.tma_stages = int(kernel), int(tma_rows), int(tma_stages)
    p.tma_npt = int(tma_npt)
    p.rounding = int(rounding)
    return p


class Cavity2D:
    """One side-heated cavity on the GPU, backed by a torch-allocated workspace."""

    def __init__(self, params: Params, theta0=None, device="cuda", stream=None,
                 theta_hot_profile=None):
        import torch

        self.p = params
        self.nx, self.ny = params.nx, params.ny
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = dmrt_workspace_size(params)
        # 256-byte aligned: torch's caching allocator returns 512-byte aligned blocks.
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        assert self.workspace.data_ptr() % 256 == 0
        self.h = dmrt_create(params, theta0, self.workspace.data_ptr(), nbytes,
                             self.stream.cuda_stream)
        self.consts = dmrt_get_consts(self.h)
        self.launch = dmrt_get_launch(self.h).as_dict()
        if theta_hot_profile is not None:
            dmrt_set_wall_profiles(self.h, hot=theta_hot_profile)

    @classmethod
    def from_inputs(cls, cav, **kw):
        """From a ``paper_1601_04633_gb300.inputs.Cavity`` description."""
        p = make_params(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha, theta_hot=cav.theta_hot,
                        theta_cold=cav.theta_cold, theta_init=cav.theta_init,
                        **{k: v for k, v in kw.items() if k in ("storage", "nu_capacity",
                                                                   "left_wall", "right_wall",
                                                                   "theta_ref", "kernel",
                                                                   "tma_rows", "tma_stages",
                                                                   "tma_npt", "rounding")})
        rest = {k: v for k, v in kw.items() if k in ("device", "stream")}
        return cls(p, theta0=cav.theta0(), theta_hot_profile=cav.theta_hot_profile, **rest)

    def step(self, n: int):
        dmrt_step(self.h, n)

    def check(self):
        dmrt_check(self.h)

    @property
    def steps_done(self) -> int:
        return dmrt_steps_done(self.h)

    def fields(self):
        """(u, v, theta) as float32 CUDA tensors [ny][nx]."""
        import torch

        out = [torch.empty((self.ny, self.nx), dtype=torch.float32, device=self.device) for _ in range(3)]
        dmrt_fields(self.h, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), True)
        return tuple(out)

    def fields_host(self, pinned=None):
        """(u, v, theta) as float32 numpy arrays [ny][nx], copied by the library."""
        if pinned is None:
            out = [np.empty((self.ny, self.nx), dtype=np.float32) for _ in range(3)]
            ptrs = [a.ctypes.data for a in out]
        else:
            out = pinned
            ptrs = [t.data_ptr() for t in pinned]
        dmrt_fields(self.h, ptrs[0], ptrs[1], ptrs[2], False)
        return tuple(out) if pinned is None else tuple(t.numpy() for t in pinned)

    def adjoint(self, nsteps: int, avg_last: int, overlap: bool = True, store: str = "auto"):
        """Advance nsteps and return (J, dJ/dtheta_w [ny], dJ/dRa): J = mean hot-wall Nu
        over the last avg_last steps. The adjoint workspace is allocated with torch.
        store="all": every forward state kept (cluster-kernel contexts only; no
        segment recompute); "checkpoints": sqrt(N) checkpoints, the segment
        recompute overlapped with the reverse sweep or, with overlap=False,
        alternating with it (the smallest workspace); "auto": "all" when the
        context allows it and the states take at most half of the free device
        memory, else "checkpoints"."""
        import torch

        if store not in ("auto", "all", "checkpoints"):
            raise ValueError("store must be 'auto', 'all' or 'checkpoints'")
        lib = load()
        nbytes = ctypes.c_size_t()
        if store != "checkpoints":
            _check(lib.dmrt_adjoint_workspace_all(self.h, int(nsteps), ctypes.byref(nbytes)), self.h)
            if store == "all" and nbytes.value == 0:
                raise ValueError("this context does not step with the cluster kernel: store='all' is unavailable")
            if store == "auto" and (nbytes.value == 0 or nbytes.value > torch.cuda.mem_get_info(self.device)[0] // 2):
                nbytes.value = 0
        if nbytes.value == 0:
            size_fn = lib.dmrt_adjoint_workspace_size if overlap else lib.dmrt_adjoint_workspace_min
            _check(size_fn(self.h, int(nsteps), ctypes.byref(nbytes)), self.h)
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        J = ctypes.c_double()
        dth = np.zeros(self.ny)
        dRa = ctypes.c_double()
        _check(lib.dmrt_adjoint(self.h, int(nsteps), int(avg_last), _VP(ws.data_ptr()), nbytes.value,
                                ctypes.byref(J), _dptr(dth), ctypes.byref(dRa)), self.h)
        del ws
        return J.value, dth, dRa.value

    def get_state(self) -> np.ndarray:
        """Post-collision populations [14][ny][nx] (f_1..f_9, g_1..g_5), float32."""
        return dmrt_get_state(self.h, self.nx, self.ny)

    def set_state(self, state):
        dmrt_set_state(self.h, state)

    def save(self, path=None) -> bytes:
        """Checkpoint (bytes; also written to ``path`` when given)."""
        blob = dmrt_save(self.h)
        if path is not None:
            tmp = str(path) + ".tmp"
            with open(tmp, "wb") as fh:
                fh.write(blob)
            os.replace(tmp, path)
        return blob

    def load(self, blob_or_path):
        """Resume from a checkpoint made by ``save`` (bytes or a file path)."""
        if isinstance(blob_or_path, (bytes, bytearray, memoryview)):
            blob = bytes(blob_or_path)
        else:
            with open(blob_or_path, "rb") as fh:
                blob = fh.read()
        dmrt_load(self.h, blob)

    def nusselt(self, series_cap: int = 0):
        return dmrt_nusselt(self.h, self.ny, series_cap)

    def energy(self):
        """(sum of theta, wall heat input of the next step) of the current state."""
        return dmrt_energy(self.h)

    def nusselt_flux(self):
        """(mean, per-row array) of the link-flux Nusselt estimator of the current state."""
        local = np.zeros(self.ny)
        mean = ctypes.c_double(0.0)
        _check(load().dmrt_nusselt_flux(self.h, ctypes.byref(mean), local.ctypes.data_as(_DP)), self.h)
        return mean.value, local

    def close(self):
        if getattr(self, "h", None):
            dmrt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slab(Cavity2D):
    """Rows y0 .. y0 + rows - 1 of the cavity ``params`` as a context with two
    halo rows, plus its four face messages (torch uint8 device tensors of
    ``halo_bytes`` each): ``to_below`` / ``to_above`` (what this slab sends) and
    ``from_below`` / ``from_above`` (what it receives)."""

    def __init__(self, params: Params, y0: int, rows: int, theta0=None, device="cuda", stream=None,
                 theta_hot_profile=None):
        import torch

        self.p = params
        self.nx, self.ny = params.nx, int(rows)
        self.y0, self.H = int(y0), params.ny
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = dmrt_slab_workspace_size(params, rows)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.h = dmrt_create_slab(params, y0, rows, theta0, self.workspace.data_ptr(), nbytes,
                                  self.stream.cuda_stream)
        self.consts = dmrt_get_consts(self.h)
        self.launch = dmrt_get_launch(self.h).as_dict()
        self.halo_bytes = dmrt_slab_halo_bytes(self.h)
        self.has_below = self.y0 > 0
        self.has_above = self.y0 + self.ny < self.H
        mk = lambda: torch.zeros(self.halo_bytes, dtype=torch.uint8, device=self.device)  # noqa: E731
        self.to_below, self.to_above, self.from_below, self.from_above = mk(), mk(), mk(), mk()
        if theta_hot_profile is not None:
            dmrt_set_wall_profiles(self.h, hot=theta_hot_profile)

    def _ptr(self, t, use):
        return t.data_ptr() if use else 0

    def pack(self):
        dmrt_slab_pack(self.h, self._ptr(self.to_below, self.has_below), self._ptr(self.to_above, self.has_above))

    def unpack(self):
        dmrt_slab_unpack(self.h, self._ptr(self.from_below, self.has_below),
                         self._ptr(self.from_above, self.has_above))

    def step_one(self):
        """One time step, then the new boundary rows packed into to_below / to_above."""
        dmrt_slab_step(self.h, self._ptr(self.to_below, self.has_below), self._ptr(self.to_above, self.has_above))

    def finish(self):
        """Sum the last step's Nusselt rows into the ring (dmrt_step(c, 0))."""
        dmrt_step(self.h, 0)


class _Member(Cavity2D):
    """A batch member as a context (borrowed: the batch owns it)."""

    def __init__(self, batch, i, params):
        self.p = params
        self.nx, self.ny = params.nx, params.ny
        self.device = batch.device
        self.stream = batch.stream
        self.h = _VP(load().dmrt_batch_context(batch.b, i))
        self.consts = dmrt_get_consts(self.h)
        self.launch = dmrt_get_launch(self.h).as_dict()

    def close(self):
        self.h = None


class Batch:
    """Independent cavities stepped together by the batched kernel (one launch
    per time step); ``members[i]`` exposes each as a context."""

    def __init__(self, params_list, theta0_list=None, opts=None, device="cuda", stream=None):
        import torch

        n = len(params_list)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = (Params * n)(*params_list)
        nbytes = ctypes.c_size_t()
        _check_batch(load().dmrt_batch_workspace_size(arr, n, ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        keep = []
        th_ptrs = None
        if theta0_list is not None:
            th_ptrs = (_DP * n)()
            for i, th in enumerate(theta0_list):
                if th is not None:
                    a = np.ascontiguousarray(th, dtype=np.float64)
                    keep.append(a)
                    th_ptrs[i] = a.ctypes.data_as(_DP)
        o = None
        if opts is not None:
            o = BatchOpts(*[int(opts.get(k, 0)) for k in ("tma_npt", "tma_rows", "tma_stages", "graph_steps",
                                                          "group_bytes", "steps_per_launch", "tensor_store",
                                                          "strip_fill")])
        b = _VP()
        _check_batch(load().dmrt_batch_create(arr, n, th_ptrs, ctypes.byref(o) if o else None,
                                              _VP(self.workspace.data_ptr()), nbytes.value,
                                              _VP(self.stream.cuda_stream), ctypes.byref(b)))
        self.b = b
        self.n = n
        lk = Launch()
        _check_batch(load().dmrt_batch_get_launch(b, ctypes.byref(lk)), b)
        self.launch = lk.as_dict()
        self.groups = load().dmrt_batch_group_count(b)
        self.members = [_Member(self, i, params_list[i]) for i in range(n)]

    @classmethod
    def from_inputs(cls, cavities, opts=None, nu_capacity=1 << 16, storage=DMRT_FP32,
                    rounding=DMRT_ROUND_AUTO, **kw):
        """Every cavity stored alike: DMRT_FP32, or DMRT_MIXED with either rounding
        (AUTO: stochastic for mixed storage)."""
        ps = [make_params(c.nx, c.ny, c.Ra, c.Pr, c.alpha, theta_hot=c.theta_hot, theta_cold=c.theta_cold,
                          theta_init=c.theta_init, nu_capacity=nu_capacity, storage=storage, rounding=rounding)
              for c in cavities]
        return cls(ps, [c.theta0() for c in cavities], opts=opts, **kw)

    @property
    def nodes(self) -> int:
        return sum(m.nx * m.ny for m in self.members)

    def step(self, n: int):
        _check_batch(load().dmrt_batch_step(self.b, int(n)), self.b)

    def check(self):
        _check_batch(load().dmrt_batch_check(self.b), self.b)

    def close(self):
        if getattr(self, "b", None):
            for m in self.members:
                m.close()
            load().dmrt_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _nusselt_objective_class():
    import torch

    class NusseltObjective(torch.autograd.Function):
        """J(theta_w, Ra) = mean hot-wall Nusselt number over the last ``avg_last`` of
        ``nsteps`` steps of a cavity started from ``cavity`` (an ``inputs.Cavity``), as
        a differentiable function of the hot-wall profile theta_w [ny] and Ra; the
        backward pass returns the discrete adjoint's gradients."""

        @staticmethod
        def forward(ctx, theta_w, Ra, cavity, nsteps, avg_last):
            import copy

            cav = copy.copy(cavity)
            cav.Ra = float(Ra.detach().cpu())
            cav.theta_hot_profile = theta_w.detach().cpu().double().numpy()
            sim = Cavity2D.from_inputs(cav, nu_capacity=max(int(avg_last), 1))
            J, dth, dRa = sim.adjoint(int(nsteps), int(avg_last))
            sim.close()
            ctx.save_for_backward(torch.as_tensor(dth, dtype=theta_w.dtype, device=theta_w.device),
                                  torch.as_tensor(dRa, dtype=Ra.dtype, device=Ra.device))
            return torch.as_tensor(J, dtype=theta_w.dtype, device=theta_w.device)

        @staticmethod
        def backward(ctx, gJ):
            dth, dRa = ctx.saved_tensors
            return gJ * dth, gJ * dRa, None, None, None

    return NusseltObjective


def nusselt_objective(theta_w, Ra, cavity, nsteps: int, avg_last: int):
    """Differentiable J(theta_w, Ra) (see ``NusseltObjective``)."""
    return _nusselt_objective_class().apply(theta_w, Ra, cavity, nsteps, avg_last)
