"""The bounds-checked build (libdmrt_bc.so, compiled with DMRT_BOUNDS_CHECK):
every index the kernels compute is range-checked before its access, and a
violation is recorded in the context's error word and reported as
DMRT_E_BOUNDS. These runs are in bounds: over small and ragged grids, every
kernel, storage mode, batched schedule, slab split and the cluster kernel, the
bounds-checked build must report no violation and give the same bits as the
regular build. (The checked build runs in a child process: the library is
chosen when the binding loads it.)"""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu

# (name, nx, ny, keyword arguments of Cavity2D.from_inputs)
SINGLE = [
    ("2x2_auto", 2, 2, {}), ("5x3_auto", 5, 3, {}), ("37x23_direct", 37, 23, {"kernel": 1}),
    ("67x45_tma", 67, 45, {"kernel": 2}), ("130x17_tma_r4", 130, 17, {"kernel": 2, "tma_rows": 4}),
    ("1000x301_tma", 1000, 301, {"kernel": 2}), ("1000x301_npt4", 1000, 301, {"kernel": 2, "tma_npt": 4,
                                                                           "tma_rows": 2, "tma_stages": 2}),
    ("481x8_fp16", 481, 8, {"storage": 1}), ("300x70_bf16", 300, 70, {"storage": 2, "rounding": 1}),
    ("1000x301_mixed", 1000, 301, {"storage": 3}), ("67x45_mixed", 67, 45, {"storage": 3, "rounding": 0}),
    ("64x64_cluster", 64, 64, {"kernel": 3}), ("37x23_cluster", 37, 23, {"kernel": 3}),
    ("1000x301_theta32", 1000, 301, {"storage": 4}), ("5x3_theta32", 5, 3, {"storage": 4, "rounding": 0}),
    ("481x8_theta32_r4", 481, 8, {"storage": 4, "tma_npt": 2, "tma_rows": 4, "tma_stages": 2}),
]
STEPS = 21


def run_cases(out_path):
    """Run every case with the library the environment selects; save the states
    and the status of each case's check to out_path (npz)."""
    import torch  # noqa: F401

    from paper_1601_04633_gb300 import dmrt as D
    from paper_1601_04633_gb300 import inputs, slabs

    res, status = {}, {}

    def chk(name, fn):
        try:
            fn()
            status[name] = 0
        except D.DmrtError as e:
            status[name] = e.code

    for name, nx, ny, kw in SINGLE:
        cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=1e-3, seed=71)
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=STEPS, **kw)
        sim.step(STEPS)
        chk(name, sim.check)
        res[name] = sim.get_state()
        res[name + "_nu"] = sim.nusselt(STEPS)[2]
        sim.close()
    cavs = [inputs.Cavity(nx, ny, 1e5, 0.005, noise_amp=1e-3, seed=80 + k)
            for k, (nx, ny) in enumerate([(128, 128), (200, 150), (67, 45), (500, 9), (2, 2)])]
    for name, storage, opts in (("batch_fp32", 0, dict(tma_npt=2, tma_rows=2, tma_stages=2)),
                                ("batch_mixed", 3, dict(tma_npt=4, tma_rows=2, tma_stages=2)),
                                ("batch_mstep", 0, dict(tma_npt=2, tma_rows=2, tma_stages=2, steps_per_launch=4)),
                                ("batch_groups", 3, dict(tma_npt=4, tma_rows=4, tma_stages=2,
                                                         group_bytes=1 << 20))):
        b = D.Batch.from_inputs(cavs, opts=opts, nu_capacity=STEPS, storage=storage)
        b.step(STEPS)
        chk(name, b.check)
        for i, m in enumerate(b.members):
            res[f"{name}_{i}"] = m.get_state()
        b.close()
    cav = inputs.Cavity(300, 200, 1e5, 0.01, noise_amp=1e-3, seed=90)
    p = D.make_params(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha, nu_capacity=STEPS)
    run = slabs.LocalSlabs(p, 3, theta0=cav.theta0())
    run.step(STEPS)
    chk("slabs", run.check)
    res["slabs"] = run.get_state()
    run.close()
    np.savez(out_path, **res, status_names=np.array(list(status)), status_codes=np.array(list(status.values())))


def _child(out_path, variant):
    env = dict(os.environ)
    if variant:
        env["DMRT_LIBRARY"] = variant
    else:
        env.pop("DMRT_LIBRARY", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(out_path)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(out_path)


def test_bounds_checked_build_reports_nothing_and_gives_the_same_bits(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import build as B

    assert os.path.exists(B.LIB_BC)
    bc = _child(tmp_path / "bc.npz", "bounds_check")
    reg = _child(tmp_path / "reg.npz", None)
    for name, code in zip(bc["status_names"], bc["status_codes"]):
        assert code == 0, (str(name), int(code))  # no DMRT_E_BOUNDS, nothing else either
    keys = [k for k in reg.files if not k.startswith("status")]
    assert len(keys) > 30
    for k in keys:
        assert np.array_equal(bc[k], reg[k]), k


if __name__ == "__main__":
    run_cases(sys.argv[1])
