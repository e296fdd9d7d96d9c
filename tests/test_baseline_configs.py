"""The benchmark workloads at their full stated lengths, against the fp64 oracle.

* 64 x 64, Ra 1e4, Pr 0.01, 20,000 steps: float32 fields within 1e-5 (max
  relative error per field) and the mean-Nu history within 1e-4.
* 256 x 256 oscillatory (Ra 1e5, Pr 0.005): fields at step 1e4 for every
  storage mode (float32 within 1e-4, the 1e-3-step tolerance grown linearly;
  the 16-bit and mixed errors held to about twice their measured values) and
  the Nusselt gate (1e-3, step by step; strict expected failures for the
  storage modes that miss it); over 1e6 steps the float32 Nu history sample
  by sample, and the reduced-precision histories' mean, period and amplitude
  against the oracle's record (golden file from
  tests/golden/make_baseline_goldens.py), over an ensemble of initial-noise
  seeds where the rounding is stochastic.
* The 64-cavity sweep, 50,000 steps in one batch: three sampled members' Nu
  histories within 1e-3 of the oracle's (same golden script).
* 4096 x 4096, Ra 1e7, Pr 0.001, 20,000 steps: each storage mode's mean-Nu
  history within 1e-3 of the float32 run's, step by step (strict expected
  failures for the modes that miss it).
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


# 256^2 at step 1e4, every storage mode. float32: the 1e-5 tolerance holds at
# 1e3 steps; rounding errors grow at most linearly with the step count, so 1e-4
# at 1e4 steps. The other modes are held to about twice their measured field
# errors (GB300, max over u, v, theta of max |a - b| / max |b|: mixed 1.5e-2,
# mixed SR 1.3e-2, float16 0.12, bfloat16 0.58, float16 SR 1.1e-2, bfloat16 SR
# 7.1e-2, THETA32 1.4e-2, THETA32 SR 1.3e-2); mixed and THETA32 storage keep
# theta within ~3e-5 and the velocities only to ~1.5 % (the float16 resolution
# of the flow populations while the flow is still weak). The Nusselt gate is
# checked step by step over the 1e4 steps.
FIELDS_256_BOUND = {(0, 0): 1e-4, (3, 0): 0.03, (3, 1): 0.03, (1, 0): 0.25, (2, 0): 1.2, (1, 1): 0.025,
                    (2, 1): 0.15, (4, 0): 0.03, (4, 1): 0.03}
_runs_256 = {}


def _run_256(D, storage, rounding):
    key = (storage, rounding)
    if key not in _runs_256:
        cav = inputs.cavity_256_oscillatory()
        steps = 10_000
        if "ref" not in _runs_256:
            m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
            f, g = O.init(m, cav.theta0())
            _runs_256["ref"] = O.run(m, steps, f, g)
        ref = _runs_256["ref"]
        u, v, th, nu = _gpu_run(D, cav, steps, storage=storage, rounding=rounding)
        errs = {name: _field_err(a, ref[name]) for name, a in (("u", u), ("v", v), ("theta", th))}
        nu_pw = float(np.max(np.abs(nu - ref["nu_series"]) / np.abs(ref["nu_series"])))
        print(f"256^2 step 1e4, storage {storage} rounding {rounding}: field errors "
              + ", ".join(f"{k} {e:.2e}" for k, e in errs.items()) + f", Nu step-by-step {nu_pw:.2e}")
        _runs_256[key] = (errs, nu_pw)
    return _runs_256[key]


@pytest.mark.parametrize("storage,rounding", list(FIELDS_256_BOUND),
                         ids=["fp32", "mixed", "mixed_sr", "fp16", "bf16", "fp16_sr", "bf16_sr", "theta32",
                              "theta32_sr"])
def test_cavity_256_fields_at_step_10000(D, storage, rounding):
    errs, nu_pw = _run_256(D, storage, rounding)
    assert max(errs.values()) <= FIELDS_256_BOUND[(storage, rounding)], errs
    if storage == 0:
        assert nu_pw <= 1e-4


def _gate_fails(reason):
    return pytest.mark.xfail(strict=True, reason=reason)


GATE_CASES = [
    pytest.param(3, 0, id="mixed"),
    pytest.param(3, 1, id="mixed_sr"),
    pytest.param(4, 0, id="theta32"),
    pytest.param(4, 1, id="theta32_sr"),
    pytest.param(1, 0, id="fp16", marks=_gate_fails("float16 nearest storage misses the Nu target")),
    pytest.param(2, 0, id="bf16", marks=_gate_fails("bfloat16 nearest storage misses the Nu target")),
    pytest.param(1, 1, id="fp16_sr", marks=_gate_fails("float16 SR storage misses the Nu target")),
    pytest.param(2, 1, id="bf16_sr", marks=_gate_fails("bfloat16 SR storage misses the Nu target")),
]


@pytest.mark.parametrize("storage,rounding", GATE_CASES)
def test_cavity_256_nu_gate_at_step_10000(D, storage, rounding):
    _, nu_pw = _run_256(D, storage, rounding)
    assert nu_pw <= 1e-3


_runs_1e6 = {}
# Initial-noise seeds of the long-run ensemble. The oscillation's statistics do
# not depend on the initial noise (float32 gives the same second-half mean,
# +6.7e-6 .. +7.0e-6 against the oracle's seed-2 record, for seeds 2..7), so
# every member is compared with the oracle's record. With stochastic rounding
# each member's rounding stream is one draw: its second-half mean is a random
# variable (GB300, seeds 2..7: mixed SR -2.2e-3 .. +7.3e-4, THETA32 SR
# -1.2e-3 .. +5.4e-4), so the gate takes the ensemble mean.
SEEDS_1E6 = (2, 3, 4, 5, 6, 7)


def _run_1e6(D, storage, rounding, seed=2):
    key = (storage, rounding, seed)
    if key not in _runs_1e6:
        gold = _gold("oracle_config2_256.json")
        cav = inputs.cavity_256_oscillatory()
        cav = inputs.Cavity(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha, seed=seed)
        steps, every = gold["steps"], gold["every"]
        fo = cav.alpha / cav.ny ** 2 * every
        ref = np.array(gold["nu"])
        half = len(ref) // 2
        sim = D.Cavity2D.from_inputs(cav, storage=storage, rounding=rounding, nu_capacity=steps)
        sim.step(steps)
        sim.check()
        nu = sim.nusselt(steps)[2][every - 1::every]
        sim.close()
        sg = A.nu_statistics(nu, fo, window_fo=1.0)
        so = A.nu_statistics(ref, fo, window_fo=1.0)
        dmean = (nu[half:].mean() - ref[half:].mean()) / ref[half:].mean()
        print(f"256^2 x 1e6, storage {storage} rounding {rounding} seed {seed}: second-half mean "
              f"{nu[half:].mean():.5f} (oracle {ref[half:].mean():.5f}, {dmean:+.2e}), period {sg.period_fo:.4f} "
              f"({so.period_fo:.4f}), amplitude {sg.amplitude:.4f} ({so.amplitude:.4f})")
        _runs_1e6[key] = (nu, ref, sg, so, dmean)
    return _runs_1e6[key]


def _ensemble_1e6(D, storage, rounding):
    runs = [_run_1e6(D, storage, rounding, sd) for sd in SEEDS_1E6]
    dmean = float(np.mean([r[4] for r in runs]))
    amp = float(np.mean([r[2].amplitude for r in runs]))
    print(f"256^2 x 1e6, storage {storage} rounding {rounding}: ensemble of {len(runs)} seeds, mean bias "
          f"{dmean:+.2e} (spread {np.std([r[4] for r in runs]):.2e}), mean amplitude {amp:.4f}")
    return runs, dmean, amp


def test_cavity_256_one_million_steps_float32_follows_the_oracle(D):
    # The oscillatory cavity over 1e6 steps (Fo 1.53): float32 follows the
    # oracle's record sample by sample for the whole run, from every seed's
    # initial noise to the same long-run mean.
    nu, ref, sg, so, dmean = _run_1e6(D, 0, 0)
    assert np.abs(nu - ref).max() <= 1e-3 * np.abs(ref).max()
    assert not sg.steady and not so.steady
    assert sg.period_fo == pytest.approx(so.period_fo, rel=0.05)
    assert sg.amplitude == pytest.approx(so.amplitude, rel=0.1)
    for sd in SEEDS_1E6:
        assert abs(_run_1e6(D, 0, 0, sd)[4]) <= 1e-4


# Mean bias of the nearest-rounding modes (one seed: the bias is systematic),
# held to about twice its measured value (GB300: mixed -3.1e-3, THETA32 -3.5e-3).
MEAN_1E6_NEAREST_BOUND = {(3, 0): 7e-3, (4, 0): 7e-3}


@pytest.mark.parametrize("storage,rounding", list(MEAN_1E6_NEAREST_BOUND), ids=["mixed", "theta32"])
def test_cavity_256_one_million_steps_nearest_bias(D, storage, rounding):
    # Rounding to nearest loses the increments below half a float16 unit: the
    # long-run mean is biased (its gate, below, is an expected failure).
    nu, ref, sg, so, dmean = _run_1e6(D, storage, rounding)
    assert abs(dmean) <= MEAN_1E6_NEAREST_BOUND[(storage, rounding)], dmean
    assert not sg.steady


@pytest.mark.parametrize("storage", [3, 4], ids=["mixed_sr", "theta32_sr"])
def test_cavity_256_one_million_steps_stochastic_statistics(D, storage):
    # Stochastic rounding: every member oscillates with the oracle's period
    # (within 5 %); the ensemble's mean amplitude is within 10 % of the oracle's.
    runs, dmean, amp = _ensemble_1e6(D, storage, 1)
    so = runs[0][3]
    for nu, ref, sg, _, _ in runs:
        assert not sg.steady
        assert sg.period_fo == pytest.approx(so.period_fo, rel=0.05)
    assert amp == pytest.approx(so.amplitude, rel=0.1)


@pytest.mark.parametrize("storage,rounding", [
    pytest.param(3, 1, id="mixed_sr"),
    pytest.param(4, 1, id="theta32_sr"),
    pytest.param(3, 0, id="mixed", marks=_gate_fails("mixed nearest: long-run mean biased by -3.1e-3")),
    pytest.param(4, 0, id="theta32", marks=_gate_fails("THETA32 nearest: long-run mean biased by -3.5e-3")),
])
def test_cavity_256_one_million_steps_mean_gate(D, storage, rounding):
    # The Nusselt target over the long run: the second-half mean within 1e-3 of
    # the oracle's, over the seed ensemble (GB300: mixed SR -8.5e-4, THETA32 SR
    # -2.1e-4; one seed for the nearest modes, whose bias is systematic).
    if rounding == 1:
        dmean = _ensemble_1e6(D, storage, rounding)[1]
    else:
        dmean = _run_1e6(D, storage, rounding)[4]
    assert abs(dmean) <= 1e-3


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


_runs_4096 = {}


def _run_4096(D, storage, rounding):
    key = (storage, rounding)
    if key not in _runs_4096:
        cav = inputs.cavity_4096()
        steps = 20_000
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=steps, storage=storage, rounding=rounding)
        sim.step(steps)
        sim.check()
        _runs_4096[key] = sim.nusselt(steps)[2]
        sim.close()
    return _runs_4096[key]


@pytest.mark.parametrize("storage,rounding", GATE_CASES)
def test_cavity_4096_20000_steps_nu_gate_against_float32(D, storage, rounding):
    # The metric's gate on the large cavity: the mean-Nu history within 1e-3 of
    # the float32 run's, step by step, over the stated 20,000 steps.
    ref = _run_4096(D, 0, 0)
    nu = _run_4096(D, storage, rounding)
    dev = float(np.max(np.abs(nu - ref) / np.abs(ref)))
    print(f"4096^2 x 20000, storage {storage} rounding {rounding}: Nu step-by-step deviation from float32 {dev:.2e}")
    assert dev <= 1e-3
