"""16-bit and mixed population storage (float16 / bfloat16 everywhere, or
float16 flow populations with float32 thermal populations; float32 collision).

One step from a given state is checked element by element against the fp64
oracle run from the same (already rounded) state: the only extra error of a
16-bit plane is the final rounding of each stored value, at most one half unit
in the last place (nearest) or one unit (stochastic), u = 2^-11 (float16) or
2^-8 (bfloat16) of the stored (shifted) value, plus the float32 arithmetic
(~1e-6 of the plane); a float32 plane of the mixed layout has only the latter.
Long runs are compared with the oracle step by step. Plain 16-bit storage
misses the 1e-3 Nusselt target (increments below half an ulp are lost, and the
temperature noise of 16-bit thermal populations remains with stochastic
rounding): those cases are strict expected failures. The mixed layout meets it,
and so does THETA32 (float32 theta, float16 deviations of the moving thermal
populations; tests/test_theta32.py checks its single step).
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_04633_gb300 import inputs, tune

pytestmark = pytest.mark.gpu

UNIT_ROUNDOFF = {1: 2.0 ** -11, 2: 2.0 ** -8, 3: 2.0 ** -11}  # 3: mixed (float16 flow planes)
NU_TARGET = 1e-3


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import dmrt

    return dmrt


def _random_state(nx, ny, seed, theta_mid):
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    r = inputs.uniform01(seed, 4 * nx * ny).reshape(4, ny, nx)
    drho, u, v = 2e-3 * (r[0] - 0.5), 0.1 * (r[1] - 0.5), 0.1 * (r[2] - 0.5)
    th = theta_mid + r[3] - 0.5
    eu = ex[:, None, None] * u + ey[:, None, None] * v
    f = w9[:, None, None] * (drho + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u * u + v * v))
    g = np.empty((5, ny, nx))
    g[0] = 0.3 * th
    g[1:] = 0.175 * th
    g += 1e-2 * (inputs.uniform01(seed + 2, 5 * nx * ny).reshape(5, ny, nx) - 0.5)
    return np.concatenate([f, g]).astype(np.float32)


@pytest.mark.parametrize("rounding", [0, 1], ids=["nearest", "stochastic"])
@pytest.mark.parametrize("storage", [1, 2, 3], ids=["fp16", "bf16", "mixed"])
@pytest.mark.parametrize("walls", [(0.5, -0.5), (1.0, 0.0)], ids=["theta_ref0", "theta_ref0.5"])
@pytest.mark.parametrize("nx,ny", [(1000, 301), (67, 45), (70, 3)])
def test_one_step_matches_oracle_within_rounding(D, storage, walls, nx, ny, rounding):
    # Nearest: at most half a unit in the last place; stochastic: less than one.
    hot, cold = walls
    cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=0.0, theta_hot=hot, theta_cold=cold)
    sim = D.Cavity2D.from_inputs(cav, storage=storage, rounding=rounding)
    sim.set_state(_random_state(nx, ny, 61, 0.5 * (hot + cold)))
    state = sim.get_state()  # the state as stored (rounded to 16 bits)
    sim.step(1)
    sim.check()
    out = sim.get_state()
    nu_mean = sim.nusselt()[0]
    k = sim.consts
    sim.close()

    m = O.derive(nx, ny, cav.Ra, cav.Pr, cav.alpha, theta_hot=hot, theta_cold=cold)
    s64 = state.astype(np.float64)
    r = O.step(m, np.ascontiguousarray(s64[:9]), np.ascontiguousarray(s64[9:]))
    ref = np.concatenate([r["f"], r["g"]])
    u16 = UNIT_ROUNDOFF[storage] * (2.0 if rounding else 1.0)
    theta_ref = 0.5 * (hot + cold) if storage != 3 else 0.0  # float32 thermal planes are not shifted
    shift = np.array([0.0] * 9 + [(1 - k.a) / 5 * theta_ref] + [(4 + k.a) / 20 * theta_ref] * 4)
    for p in range(14):
        u = 0.0 if (storage == 3 and p >= 9) else u16
        bound = u * np.abs(ref[p] - shift[p]) + 1e-5 * np.abs(ref[p]).max() + 1e-12
        err = np.abs(out[p] - ref[p])
        assert np.all(err <= bound), f"plane {p}: worst excess {(err - bound).max():.3e}"
        if rounding and u > 0:
            # Unbiased: the mean signed error is far below one unit in the last
            # place. Each node's rounding error has mean zero and a standard
            # deviation below half its spacing (u |x| / 2), so the mean of n
            # errors is allowed six of its standard deviations on top.
            signed = (out[p] - ref[p]).mean()
            ulps = u * np.abs(ref[p] - shift[p])
            sigma = np.sqrt(np.sum((ulps / 2) ** 2)) / ulps.size
            assert abs(signed) <= 0.02 * ulps.mean() + 6 * sigma + 1e-5 * np.abs(ref[p]).max()
    # The Nusselt number comes from the pre-collision theta of the rounded state.
    assert abs(nu_mean - r["nu"]) <= 1e-5 * abs(r["nu"]) + 1e-9


# Long runs: 64 x 64, Ra 1e4, Pr 0.01 (Case 1), 5000 steps, against the oracle.
# The Nusselt gate is the step-by-step relative deviation of the mean-Nu
# history, max_t |Nu(t) - Nu_oracle(t)| / |Nu_oracle(t)| <= 1e-3. The field
# errors are held to about twice their measured values (GB300; max |a - b| /
# max |b| of theta: float32 1.9e-7, float16 4.4e-2, bfloat16 0.31, float16 SR
# 8.7e-4, bfloat16 SR 8.8e-3, mixed 1.6e-5, mixed SR 2.7e-5, THETA32 2.3e-5,
# THETA32 SR 2.8e-5).
LONG_RUN_THETA_BOUND = {(0, 0): 1e-5, (1, 0): 0.09, (2, 0): 0.6, (1, 1): 2e-3, (2, 1): 2e-2, (3, 0): 5e-5,
                        (3, 1): 6e-5, (4, 0): 5e-5, (4, 1): 6e-5}
_long_runs = {}


def _long_run(D, storage, rounding):
    key = (storage, rounding)
    if key not in _long_runs:
        cav = inputs.cavity_64()
        steps = 5000
        sim = D.Cavity2D.from_inputs(cav, storage=storage, rounding=rounding, nu_capacity=steps)
        sim.step(steps)
        sim.check()
        u, v, th = (x.cpu().numpy().astype(np.float64) for x in sim.fields())
        series = sim.nusselt(steps)[2]
        sim.close()
        if "ref" not in _long_runs:
            m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
            f, g = O.init(m, cav.theta0())
            _long_runs["ref"] = O.run(m, steps, f, g)
        ref = _long_runs["ref"]
        nu_pw = float(np.max(np.abs(series - ref["nu_series"]) / np.abs(ref["nu_series"])))
        th_err = np.abs(th - ref["theta"]).max() / np.abs(ref["theta"]).max()
        print(f"storage {storage} rounding {rounding}: Nu step-by-step error {nu_pw:.3e}, theta error {th_err:.3e}")
        _long_runs[key] = (nu_pw, th_err)
    return _long_runs[key]


@pytest.mark.parametrize("storage,rounding", list(LONG_RUN_THETA_BOUND),
                         ids=["fp32", "fp16", "bf16", "fp16_sr", "bf16_sr", "mixed", "mixed_sr", "theta32",
                              "theta32_sr"])
def test_long_run_field_error_bounds(D, storage, rounding):
    nu_pw, th_err = _long_run(D, storage, rounding)
    assert np.isfinite(nu_pw) and th_err <= LONG_RUN_THETA_BOUND[(storage, rounding)]
    if storage == 0:
        assert nu_pw <= 1e-4


def _gate_fails(reason):
    return pytest.mark.xfail(strict=True, reason=reason)


@pytest.mark.parametrize("storage,rounding", [
    pytest.param(0, 0, id="fp32"),
    pytest.param(3, 0, id="mixed"),
    pytest.param(3, 1, id="mixed_sr"),
    pytest.param(4, 0, id="theta32"),
    pytest.param(4, 1, id="theta32_sr"),
    pytest.param(1, 0, id="fp16", marks=_gate_fails("float16 nearest loses sub-half-ulp thermal increments")),
    pytest.param(2, 0, id="bf16", marks=_gate_fails("bfloat16 nearest: 8-bit mantissa, far off")),
    pytest.param(1, 1, id="fp16_sr", marks=_gate_fails("float16 SR: temperature noise, ~0.7 % on Nu")),
    pytest.param(2, 1, id="bf16_sr", marks=_gate_fails("bfloat16 SR: temperature noise, several % on Nu")),
])
def test_long_run_nu_gate(D, storage, rounding):
    # The metric's target: Nu within 1e-3 of the oracle at every step. Storage
    # modes that miss it are expected failures (strict: passing would be news).
    nu_pw, _ = _long_run(D, storage, rounding)
    assert nu_pw <= NU_TARGET


TILES = {(1, 0): tune.SINGLE_TILES_16, (1, 1): tune.SINGLE_TILES_16_SR, (2, 0): tune.SINGLE_TILES_16,
         (2, 1): tune.SINGLE_TILES_16_SR, (3, 0): tune.SINGLE_TILES_MIXED, (3, 1): tune.SINGLE_TILES_MIXED_SR,
         (4, 0): tune.SINGLE_TILES_THETA, (4, 1): tune.SINGLE_TILES_THETA_SR}


@pytest.mark.parametrize("storage,rounding", list(TILES),
                         ids=["fp16", "fp16_sr", "bf16", "bf16_sr", "mixed", "mixed_sr", "theta32", "theta32_sr"])
@pytest.mark.parametrize("nx,ny", [(1000, 301), (67, 45), (481, 8)])
def test_16bit_tiles_agree_bitwise(D, nx, ny, storage, rounding):
    # Every compiled tile of a storage mode computes the same step (a node's
    # stochastic rounding bits depend on its index and the step only), on
    # ragged strips and row blocks.
    cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=1e-3, seed=8)
    states = []
    for npt, R, S in TILES[(storage, rounding)]:
        sim = D.Cavity2D.from_inputs(cav, storage=storage, rounding=rounding, kernel=D.DMRT_KERNEL_TMA,
                                     tma_npt=npt, tma_rows=R, tma_stages=S, nu_capacity=64)
        sim.step(37)
        sim.check()
        states.append((sim.get_state(), sim.nusselt(37)[2]))
        sim.close()
    for st, nu in states[1:]:
        assert np.array_equal(st, states[0][0]) and np.array_equal(nu, states[0][1])


def test_mixed_long_run_meets_nu_target_at_256(D):
    # The oscillatory 256 x 256 cavity (Ra 1e5, Pr 0.005), 4000 steps, against the oracle.
    cav = inputs.cavity_256_oscillatory()
    steps = 4000
    sim = D.Cavity2D.from_inputs(cav, storage=3, rounding=1, nu_capacity=steps)
    sim.step(steps)
    sim.check()
    series = sim.nusselt(steps)[2]
    sim.close()
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
    f, g = O.init(m, cav.theta0())
    ref = O.run(m, steps, f, g)
    nu_err = float(np.max(np.abs(series - ref["nu_series"]) / np.abs(ref["nu_series"])))
    print(f"mixed stochastic 256^2: Nu step-by-step error {nu_err:.3e}")
    assert nu_err <= NU_TARGET
