"""The benchmark workloads at their full stated lengths, against the fp64 oracle.

* 64 x 64, Ra 1e4, Pr 0.01, 20,000 steps: float32 fields within 1e-5 (max
  relative error per field) and the mean-Nu history within 1e-4.
* 256 x 256 oscillatory (Ra 1e5, Pr 0.005): fields at step 1e4 for every
  storage mode (float32 within 1e-4, the 1e-3-step tolerance grown linearly;
  the 16-bit and mixed errors are reported with loose bounds); over 1e6 steps
  the float32 Nu history sample by sample and the mixed-storage histories'
  mean, period and amplitude against the oracle's record (golden file from
  tests/golden/make_baseline_goldens.py).
* The 64-cavity sweep, 50,000 steps in one batch: three sampled members' Nu
  histories within 1e-3 of the oracle's (same golden script).
* 4096 x 4096, Ra 1e7, Pr 0.001, 20,000 steps: the mixed-storage run's mean-Nu
  history within 1e-3 of the float32 run's.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1601_04633_gb300 import analysis as A
from paper_1601_04633_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import dmrt

    return dmrt


def _gold(name):
    path = os.path.join(GOLD, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated (tests/golden/make_baseline_goldens.py)")
    with open(path) as fh:
        return json.load(fh)


def _field_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _gpu_run(D, cav, steps, **kw):
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=steps, **kw)
    sim.step(steps)
    sim.check()
    u, v, th = (x.cpu().numpy().astype(np.float64) for x in sim.fields())
    series = sim.nusselt(steps)[2]
    sim.close()
    return u, v, th, series


def test_cavity_64_20000_steps(D):
    cav = inputs.cavity_64()
    steps = 20_000
    u, v, th, nu = _gpu_run(D, cav, steps)
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
    f, g = O.init(m, cav.theta0())
    ref = O.run(m, steps, f, g)
    for name, a in (("u", u), ("v", v), ("theta", th)):
        assert _field_err(a, ref[name]) <= 1e-5, name
    assert np.abs(nu - ref["nu_series"]).max() <= 1e-4 * np.abs(ref["nu_series"]).max()
    print(f"64^2 x 20000: steady mean Nu {nu[-1]:.6f} (oracle {ref['nu_series'][-1]:.6f})")


def test_cavity_256_fields_at_step_10000(D):
    cav = inputs.cavity_256_oscillatory()
    steps = 10_000
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
    f, g = O.init(m, cav.theta0())
    ref = O.run(m, steps, f, g)
    # float32: the 1e-5 tolerance holds at 1e3 steps; rounding errors grow at
    # most linearly with the step count, so 1e-4 at 1e4 steps. The other modes
    # are reported, with bounds that only catch a broken path.
    # Mixed storage keeps theta within ~3e-5 and Nu within ~5e-7 but the
    # velocities only to ~1.5 % (the float16 resolution of the flow populations
    # while the flow is still weak).
    bounds = {(0, 0): 1e-4, (3, 0): 0.05, (3, 1): 0.05, (1, 1): 0.5, (1, 0): 10.0, (2, 0): 10.0, (2, 1): 10.0}
    for (storage, rounding), bound in bounds.items():
        u, v, th, nu = _gpu_run(D, cav, steps, storage=storage, rounding=rounding)
        errs = {name: _field_err(a, ref[name]) for name, a in (("u", u), ("v", v), ("theta", th))}
        nu_err = float(np.abs(nu - ref["nu_series"]).max() / np.abs(ref["nu_series"]).max())
        print(f"256^2 step 1e4, storage {storage} rounding {rounding}: field errors "
              + ", ".join(f"{k} {e:.2e}" for k, e in errs.items()) + f", Nu {nu_err:.2e}")
        assert max(errs.values()) <= bound, (storage, rounding, errs)


def test_cavity_256_one_million_steps_statistics(D):
    # The oscillatory cavity over 1e6 steps (Fo 1.53) against the oracle's
    # record. float32 follows the oracle sample by sample for the whole run.
    # Mixed storage leaves it after Fo ~0.11 (the oscillation's phase drifts),
    # so its statistics are compared: with stochastic rounding of the flow
    # populations the mean over the second half stays within 1e-3 (measured
    # 1.4e-4); with rounding to nearest it is biased low (measured -3.1e-3:
    # increments below half a float16 unit are lost), which is recorded here
    # with a bound that only catches a broken path.
    gold = _gold("oracle_config2_256.json")
    cav = inputs.cavity_256_oscillatory()
    steps, every = gold["steps"], gold["every"]
    fo = cav.alpha / cav.ny ** 2 * every
    ref = np.array(gold["nu"])
    half = len(ref) // 2
    so = A.nu_statistics(ref, fo, window_fo=1.0)
    for storage, rounding, bound in ((0, 0, 1e-4), (3, 1, 1e-3), (3, 0, 1e-2)):
        sim = D.Cavity2D.from_inputs(cav, storage=storage, rounding=rounding, nu_capacity=steps)
        sim.step(steps)
        sim.check()
        nu = sim.nusselt(steps)[2][every - 1::every]
        sim.close()
        sg = A.nu_statistics(nu, fo, window_fo=1.0)
        dmean = (nu[half:].mean() - ref[half:].mean()) / ref[half:].mean()
        print(f"256^2 x 1e6, storage {storage} rounding {rounding}: second-half mean {nu[half:].mean():.5f} "
              f"(oracle {ref[half:].mean():.5f}, {dmean:+.2e}), period {sg.period_fo:.4f} ({so.period_fo:.4f}), "
              f"amplitude {sg.amplitude:.4f} ({so.amplitude:.4f})")
        assert abs(dmean) <= bound, (storage, rounding, dmean)
        assert not sg.steady and not so.steady
        if storage == 0:
            assert np.abs(nu - ref).max() <= 1e-3 * np.abs(ref).max()
        if rounding == 1 or storage == 0:
            assert sg.period_fo == pytest.approx(so.period_fo, rel=0.05)
            assert sg.amplitude == pytest.approx(so.amplitude, rel=0.1)


def test_sweep_50000_steps_sampled_members(D):
    gold = _gold("oracle_config3_members.json")
    cavs = inputs.batch_sweep()
    steps, every = gold["steps"], gold["every"]
    b = D.Batch.from_inputs(cavs, nu_capacity=steps)
    b.step(steps)
    b.check()
    for mem in gold["members"]:
        nu = b.members[mem["index"]].nusselt(steps)[2][every - 1::every]
        ref = np.array(mem["nu"])
        err = float(np.abs(nu - ref).max() / np.abs(ref).max())
        print(f"sweep member {mem['index']} ({mem['nx']}^2, Ra {mem['Ra']:.3g}, Pr {mem['Pr']}): "
              f"max Nu error {err:.2e} over {steps} steps")
        assert err <= 1e-3
    b.close()


def test_cavity_4096_20000_steps_mixed_against_float32(D):
    cav = inputs.cavity_4096()
    steps = 20_000
    runs = {}
    for name, kw in (("fp32", {}), ("mixed", dict(storage=3)), ("fp16_sr", dict(storage=1, rounding=1))):
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=steps, **kw)
        sim.step(steps)
        sim.check()
        runs[name] = sim.nusselt(steps)[2]
        sim.close()
    ref = runs["fp32"]
    errs = {k: float(np.abs(v - ref).max() / np.abs(ref).max()) for k, v in runs.items() if k != "fp32"}
    print("4096^2 x 20000: max Nu deviation from float32:", {k: f"{e:.2e}" for k, e in errs.items()})
    assert errs["mixed"] <= 1e-3
