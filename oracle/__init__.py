"""FP64 CPU oracle of the double-MRT thermal LBM step (arXiv 1601.04633, Sec. 3).

TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path (the CUDA library
and its binding) never does, and shares no code with it.

The arithmetic lives in ``dmrt_oracle.c`` (plain C, fp64). This module builds
it with gcc on first use and wraps it with ctypes and numpy arrays of shape
``(planes, ny, nx)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmrt_oracle.c")
_HDR = os.path.join(_HERE, "dmrt_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

WALL_FIXED = 0
WALL_ADIABATIC = 1


class Model(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("left_bc", ctypes.c_int32), ("right_bc", ctypes.c_int32),
        ("rho0", ctypes.c_double), ("H", ctypes.c_double),
        ("alpha", ctypes.c_double), ("nu", ctypes.c_double),
        ("s_rho", ctypes.c_double), ("s_j", ctypes.c_double),
        ("s_e", ctypes.c_double), ("s_nu", ctypes.c_double),
        ("s_q", ctypes.c_double), ("s_eps", ctypes.c_double),
        ("sig_0", ctypes.c_double), ("sig_k", ctypes.c_double),
        ("sig_e", ctypes.c_double), ("sig_nu", ctypes.c_double),
        ("a", ctypes.c_double),
        ("theta_hot", ctypes.c_double), ("theta_cold", ctypes.c_double),
        ("theta_ref", ctypes.c_double), ("dT", ctypes.c_double),
        ("gbeta", ctypes.c_double), ("abb_coef", ctypes.c_double),
    ]

    def copy(self) -> "Model":
        m = Model()
        ctypes.memmove(ctypes.byref(m), ctypes.byref(self), ctypes.sizeof(Model))
        return m


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            mp = ctypes.POINTER(Model)
            L.orc_derive.argtypes = [ctypes.c_int32, ctypes.c_int32] + [ctypes.c_double] * 6 + [mp]
            L.orc_derive.restype = ctypes.c_int
            for name in ("orc_moments9", "orc_moments5", "orc_from_moments9", "orc_from_moments5"):
                getattr(L, name).argtypes = [dp, dp]
                getattr(L, name).restype = None
            L.orc_meq9.argtypes = [ctypes.c_double] * 4 + [dp]
            L.orc_neq5.argtypes = [ctypes.c_double] * 4 + [dp]
            L.orc_force9.argtypes = [ctypes.c_double] * 5 + [dp]
            L.orc_collide_node.argtypes = [mp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_init.argtypes = [mp, dp, dp, dp]
            L.orc_stream.argtypes = [mp, dp, dp, dp, dp, dp, dp]
            L.orc_step.argtypes = [mp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_step.restype = ctypes.c_int
            L.orc_run.argtypes = [mp, ctypes.c_int64, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_run.restype = ctypes.c_int
            L.orc_fields_from_post.argtypes = [mp, dp, dp, dp, dp, dp]
            L.orc_stream_transpose.argtypes = [mp, dp, dp, dp]
            L.orc_nu_flux.argtypes = [mp, dp, dp, dp]
            L.orc_nu_flux.restype = ctypes.c_double
            L.orc_collide_vjp.argtypes = [mp, dp, dp, dp, dp]
            L.orc_adjoint.argtypes = [mp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp, dp, dp]
            L.orc_adjoint.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    assert a.shape == (n,)
    return a


def set_threads(n: int) -> int:
    """Number of OpenMP threads the per-node loop uses (0 = leave as is)."""
    return lib().orc_set_threads(int(n))


def derive(nx, ny, Ra, Pr, alpha, theta_hot=0.5, theta_cold=-0.5, theta_ref=None,
           left_bc=WALL_FIXED, right_bc=WALL_FIXED) -> Model:
    """Model constants from the problem statement (Eqs. 9, 31-32, 38-40, 43)."""
    if theta_ref is None:
        theta_ref = 0.5 * (theta_hot + theta_cold)
    m = Model()
    rc = lib().orc_derive(int(nx), int(ny), float(Ra), float(Pr), float(alpha),
                          float(theta_hot), float(theta_cold), float(theta_ref),
                          ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"invalid oracle parameters (rc={rc})")
    m.left_bc = left_bc
    m.right_bc = right_bc
    return m


# ---- per-node pieces ------------------------------------------------------

def moments9(f):
    f = _vec(f, 9)
    out = np.zeros(9)
    lib().orc_moments9(_p(f), _p(out))
    return out


def moments5(g):
    g = _vec(g, 5)
    out = np.zeros(5)
    lib().orc_moments5(_p(g), _p(out))
    return out


def from_moments9(m):
    m = _vec(m, 9)
    out = np.zeros(9)
    lib().orc_from_moments9(_p(m), _p(out))
    return out


def from_moments5(n):
    n = _vec(n, 5)
    out = np.zeros(5)
    lib().orc_from_moments5(_p(n), _p(out))
    return out


def meq9(rho0, drho, u, v):
    out = np.zeros(9)
    lib().orc_meq9(float(rho0), float(drho), float(u), float(v), _p(out))
    return out


def neq5(a, theta, u, v):
    out = np.zeros(5)
    lib().orc_neq5(float(a), float(theta), float(u), float(v), _p(out))
    return out


def force9(rho0, u, v, Gx, Gy):
    out = np.zeros(9)
    lib().orc_force9(float(rho0), float(u), float(v), float(Gx), float(Gy), _p(out))
    return out


def collide_node(model: Model, f, g):
    """One node's D2Q9 collision + force and D2Q5 collision; returns (f*, g*, u, v, theta)."""
    f = _vec(f, 9)
    g = _vec(g, 5)
    fo, go = np.zeros(9), np.zeros(5)
    u, v, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    lib().orc_collide_node(ctypes.byref(model), _p(f), _p(g), _p(fo), _p(go),
                           ctypes.cast(ctypes.byref(u), dp), ctypes.cast(ctypes.byref(v), dp),
                           ctypes.cast(ctypes.byref(t), dp))
    return fo, go, u.value, v.value, t.value


# ---- whole grid -------------------------------------------------------------

def init(model: Model, theta0):
    """Initial post-collision state: f = 0 (rest, delta-rho = 0), g = g_eq(theta0, u = 0)."""
    nx, ny = model.nx, model.ny
    th = np.ascontiguousarray(np.asarray(theta0, dtype=np.float64)).reshape(ny, nx)
    f = np.zeros((9, ny, nx))
    g = np.zeros((5, ny, nx))
    lib().orc_init(ctypes.byref(model), _p(th), _p(f), _p(g))
    return f, g


def _profile(x, ny):
    return None if x is None else _vec(x, ny)


def stream(model: Model, fs, gs, theta_hot_profile=None, theta_cold_profile=None):
    nx, ny = model.nx, model.ny
    f = np.zeros((9, ny, nx))
    g = np.zeros((5, ny, nx))
    hp, cp = _profile(theta_hot_profile, ny), _profile(theta_cold_profile, ny)
    lib().orc_stream(ctypes.byref(model), _p(fs), _p(gs), _p(hp), _p(cp), _p(f), _p(g))
    return f, g


def step(model: Model, fs, gs, theta_hot_profile=None, theta_cold_profile=None):
    """One time step. Returns dict(f, g, u, v, theta, nu_local, nu) (new arrays)."""
    nx, ny = model.nx, model.ny
    fo = np.zeros((9, ny, nx))
    go = np.zeros((5, ny, nx))
    u, v, t = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    nl = np.zeros(ny)
    nu = ctypes.c_double()
    hp, cp = _profile(theta_hot_profile, ny), _profile(theta_cold_profile, ny)
    rc = lib().orc_step(ctypes.byref(model), _p(fs), _p(gs), _p(hp), _p(cp), _p(fo), _p(go),
                        _p(u), _p(v), _p(t), _p(nl),
                        ctypes.cast(ctypes.byref(nu), ctypes.POINTER(ctypes.c_double)))
    if rc:
        raise RuntimeError(f"orc_step failed rc={rc}")
    return dict(f=fo, g=go, u=u, v=v, theta=t, nu_local=nl, nu=nu.value)


def run(model: Model, nsteps: int, f, g, theta_hot_profile=None, theta_cold_profile=None):
    """Advance (f, g) in place by nsteps. Returns dict(nu_series, u, v, theta, nu_local)
    where the fields and the local Nusselt profile are those of the last step."""
    nx, ny = model.nx, model.ny
    assert f.shape == (9, ny, nx) and g.shape == (5, ny, nx)
    series = np.zeros(max(int(nsteps), 0))
    u, v, t = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    nl = np.zeros(ny)
    hp, cp = _profile(theta_hot_profile, ny), _profile(theta_cold_profile, ny)
    if nsteps > 0:
        rc = lib().orc_run(ctypes.byref(model), int(nsteps), _p(f), _p(g), _p(hp), _p(cp),
                           _p(series), _p(u), _p(v), _p(t), _p(nl))
        if rc:
            raise RuntimeError(f"orc_run failed rc={rc}")
    return dict(nu_series=series, u=u, v=v, theta=t, nu_local=nl)


def fields_from_post(model: Model, fs, gs):
    """(u, v, theta) at the time level of a post-collision state."""
    nx, ny = model.nx, model.ny
    u, v, t = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    lib().orc_fields_from_post(ctypes.byref(model), _p(fs), _p(gs), _p(u), _p(v), _p(t))
    return u, v, t


def stream_transpose(model: Model, lam):
    """S^T lam for the linear part S of ``stream`` (lam: 14 planes, f then g), and
    the hot-wall temperature derivative it carries. Returns (lprev, dthw)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    assert lam.shape == (14, model.ny, model.nx)
    out = np.zeros_like(lam)
    dthw = np.zeros(model.ny)
    lib().orc_stream_transpose(ctypes.byref(model), _p(lam), _p(out), _p(dthw))
    return out, dthw


def nu_flux(model: Model, gs, theta_hot_profile=None):
    """Secondary hot-wall Nusselt number of a post-collision thermal state
    ``gs`` (5, ny, nx): the heat the next streaming carries across the hot wall's
    links (Eq. 45), Nu_j = H (abb theta_w(j) - 2 g*_3(0, j)) / (alpha dT).
    Returns (mean over rows, per-row array)."""
    ny = model.ny
    local = np.zeros(ny)
    hp = _profile(theta_hot_profile, ny)
    mean = lib().orc_nu_flux(ctypes.byref(model), _p(np.ascontiguousarray(gs, dtype=np.float64)), _p(hp),
                             _p(local))
    return float(mean), local


def collide_vjp(model: Model, x, lam):
    """nu = C'(x)^T lam for one node (x, lam: 14 values, f then g) and lam . dC/dgbeta."""
    x = _vec(x, 14)
    lam = _vec(lam, 14)
    nu = np.zeros(14)
    dgb = ctypes.c_double(0.0)
    lib().orc_collide_vjp(ctypes.byref(model), _p(x), _p(lam), _p(nu),
                          ctypes.cast(ctypes.byref(dgb), ctypes.POINTER(ctypes.c_double)))
    return nu, dgb.value


def adjoint(model: Model, nsteps: int, avg_last: int, f0, g0, theta_hot_profile=None):
    """J = mean hot-wall Nu over the last avg_last of nsteps steps from (f0, g0), and
    (dJ/dtheta_w[ny], dJ/dgbeta). Keeps every forward state: small grids only."""
    ny = model.ny
    hp = _profile(theta_hot_profile, ny)
    if hp is None:
        hp = np.full(ny, model.theta_hot)
    J = ctypes.c_double()
    dth = np.zeros(ny)
    dgb = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().orc_adjoint(ctypes.byref(model), int(nsteps), int(avg_last),
                           _p(np.ascontiguousarray(f0, dtype=np.float64)),
                           _p(np.ascontiguousarray(g0, dtype=np.float64)), _p(hp),
                           ctypes.cast(ctypes.byref(J), dp), _p(dth), ctypes.cast(ctypes.byref(dgb), dp))
    if rc:
        raise RuntimeError(f"orc_adjoint failed rc={rc}")
    return J.value, dth, dgb.value


def objective(model: Model, nsteps: int, avg_last: int, theta0, theta_hot_profile=None):
    """J (as in ``adjoint``) from a forward run started at rest with temperature theta0."""
    f, g = init(model, theta0)
    r = run(model, nsteps, f, g, theta_hot_profile=theta_hot_profile)
    return float(r["nu_series"][-avg_last:].mean())
