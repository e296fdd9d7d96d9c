"""THETA32 storage: flow populations in float16, the temperature theta = sum_i g_i
(Eq. 41) in float32, and the moving thermal populations as float16 deviations
d_k = g_k - w theta (w = (4 + a)/20, the D2Q5 rest weight of Eq. 42); the rest
population is g_0 = w_0 theta - sum_k d_k.

One step from a given state is checked element by element against the fp64
oracle run from the same (already stored) state. The flow planes carry one
float16 rounding of the stored value, as in mixed storage. A moving thermal
population carries one float16 rounding of its deviation d_k, at most half a
unit in the last place (nearest) or one unit (stochastic) of |d_k|, which is
far smaller than |g_k| (plain float16 storage rounds g_k itself); the rest
population carries the four deviations' roundings. The stored populations of
a node sum to its theta up to float32 arithmetic, so the rounding moves heat
between nodes but creates none: with adiabatic walls the heat content stays
constant to float32 rounding, as with float32 storage.
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_04633_gb300 import inputs

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11


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
    # Shifted D2Q9 equilibria of random (delta-rho, u, v), and D2Q5 populations
    # near rest equilibrium around theta_mid +- 0.5, with 1e-2 noise.
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
@pytest.mark.parametrize("walls", [(0.5, -0.5), (1.0, 0.0)], ids=["theta_mid0", "theta_mid0.5"])
@pytest.mark.parametrize("nx,ny", [(1000, 301), (67, 45), (70, 3)])
def test_one_step_matches_oracle_within_rounding(D, nx, ny, walls, rounding):
    hot, cold = walls
    cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=0.0, theta_hot=hot, theta_cold=cold)
    sim = D.Cavity2D.from_inputs(cav, storage=D.DMRT_THETA32, rounding=rounding)
    sim.set_state(_random_state(nx, ny, 67, 0.5 * (hot + cold)))
    state = sim.get_state()  # the populations the stored (theta, d) stand for
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
    u = U16 * (2.0 if rounding else 1.0)
    w = (4.0 + k.a) / 20.0
    dev = ref[10:] - w * ref[9:].sum(axis=0)  # deviations of the exact post-collision state
    for p in range(14):
        if p < 9:
            scale = np.abs(ref[p])
        elif p == 9:
            scale = np.abs(dev).sum(axis=0)
        else:
            scale = np.abs(dev[p - 10])
        bound = u * scale + 1e-5 * np.abs(ref[p]).max() + 1e-12
        err = np.abs(out[p] - ref[p])
        assert np.all(err <= bound), f"plane {p}: worst excess {(err - bound).max():.3e}"
        if rounding and p >= 10:
            # Unbiased deviations: the mean signed error stays within six
            # standard deviations of its expected spread.
            ulps = u * scale
            sigma = np.sqrt(np.sum((ulps / 2) ** 2)) / ulps.size
            assert abs((out[p] - ref[p]).mean()) <= 0.02 * ulps.mean() + 6 * sigma + 1e-5 * np.abs(ref[p]).max()
    # Each node's stored populations sum to its theta (the oracle's) up to float32.
    th_scale = np.abs(r["theta"]).max()
    assert np.abs(out[9:].astype(np.float64).sum(axis=0) - r["theta"]).max() <= 2e-6 * th_scale
    assert abs(nu_mean - r["nu"]) <= 1e-5 * abs(r["nu"]) + 1e-9


def test_state_round_trip_keeps_theta_and_rounds_deviations(D):
    # dmrt_set_state stores theta = sum g in float32 and each deviation rounded
    # to the nearest float16; dmrt_get_state rebuilds the populations from them.
    nx, ny = 130, 17
    cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=0.0)
    sim = D.Cavity2D.from_inputs(cav, storage=D.DMRT_THETA32)
    st = _random_state(nx, ny, 71, 0.0)
    sim.set_state(st)
    back = sim.get_state()
    k = sim.consts
    sim.close()
    assert np.array_equal(back[:9], st[:9].astype(np.float16).astype(np.float32))
    g = st[9:].astype(np.float64)
    th = g.sum(axis=0)
    w = (4.0 + k.a) / 20.0
    dev = g[1:] - w * th
    # Within half a float16 unit of each deviation (plus float32 arithmetic);
    # the rest population carries the four roundings.
    assert np.all(np.abs(back[10:] - g[1:]) <= 2.0 ** -11 * np.abs(dev) + 1e-6)
    assert np.all(np.abs(back[9] - g[0]) <= 2.0 ** -11 * np.abs(dev).sum(axis=0) + 1e-6)
    assert np.abs(back[9:].astype(np.float64).sum(axis=0) - th).max() <= 1e-6


def test_heat_conserved_with_adiabatic_walls(D):
    # All walls adiabatic: the heat content stays constant to float32 rounding
    # over 2000 steps with stochastically rounded deviations (the rounding
    # moves heat between nodes, never in or out).
    cav = inputs.Cavity(100, 60, 1e5, 0.01, noise_amp=0.2, seed=22)
    p = D.make_params(cav.nx, cav.ny, cav.Ra, cav.Pr, left_wall=D.DMRT_WALL_ADIABATIC,
                      right_wall=D.DMRT_WALL_ADIABATIC, storage=D.DMRT_THETA32)
    sim = D.Cavity2D(p, theta0=cav.theta0())
    e0, w0 = sim.energy()
    sim.step(2000)
    sim.check()
    e1, w1 = sim.energy()
    sim.close()
    assert w0 == 0.0 and w1 == 0.0
    assert abs(e0 - cav.theta0().sum()) <= 1e-6 * np.abs(cav.theta0()).sum()
    assert abs(e1 - e0) <= 1e-6 * np.abs(cav.theta0()).sum()


def test_checkpoint_resumes_bit_for_bit(D, tmp_path):
    cav = inputs.Cavity(300, 41, 1e5, 0.01, noise_amp=1e-3, seed=5)
    a = D.Cavity2D.from_inputs(cav, storage=D.DMRT_THETA32, nu_capacity=256)
    a.step(50)
    blob = a.save(str(tmp_path / "t.bin"))
    a.step(70)
    sa = a.get_state()
    b = D.Cavity2D.from_inputs(cav, storage=D.DMRT_THETA32, nu_capacity=256)
    b.load(str(tmp_path / "t.bin"))
    b.step(70)
    sb = b.get_state()
    assert np.array_equal(sa, sb)
    assert np.array_equal(a.nusselt(70)[2], b.nusselt(70)[2])
    a.close()
    b.close()
    assert blob


def test_paths_without_theta32_refuse_it(D):
    cav = inputs.Cavity(64, 64, 1e4, 0.01)
    for kw in (dict(kernel=D.DMRT_KERNEL_DIRECT), dict(kernel=D.DMRT_KERNEL_CLUSTER)):
        with pytest.raises(RuntimeError):
            D.Cavity2D.from_inputs(cav, storage=D.DMRT_THETA32, **kw)
    sim = D.Cavity2D.from_inputs(cav, storage=D.DMRT_THETA32)
    with pytest.raises(RuntimeError):
        sim.adjoint(10, 5)
    sim.close()
    with pytest.raises(RuntimeError):
        D.Batch.from_inputs([cav, cav], storage=D.DMRT_THETA32)
