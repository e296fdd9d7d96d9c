"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (the double-MRT step in float32 against fp64):
  fields u, v, theta: max_x |gpu - oracle| / max_x |oracle| <= 1e-5 per field;
  mean hot-wall Nusselt number, every step: |gpu - oracle| / |oracle| <= 1e-4;
  one step from a given state: every population within 1e-5 of the plane's
  largest magnitude (float32 rounding of ~10 operations is ~1e-6 of that).
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_04633_gb300 import inputs, tune

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
NU_TOL = 1e-4


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import dmrt

    return dmrt


def rel_err(a, b):
    return np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300)


def gpu_run(D, cav, steps, **kw):
    sim = D.Cavity2D.from_inputs(cav, **kw)
    sim.step(steps)
    sim.check()
    u, v, t = (x.cpu().numpy().astype(np.float64) for x in sim.fields())
    mean, local, series = sim.nusselt(series_cap=steps)
    state = sim.get_state()
    sim.close()
    return dict(u=u, v=v, theta=t, nu=mean, nu_local=local, nu_series=series, state=state)


def oracle_run(cav, steps, left_bc=O.WALL_FIXED, right_bc=O.WALL_FIXED):
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha, theta_hot=cav.theta_hot,
                 theta_cold=cav.theta_cold, left_bc=left_bc, right_bc=right_bc)
    f, g = O.init(m, cav.theta0())
    r = O.run(m, steps, f, g, theta_hot_profile=cav.theta_hot_profile)
    r["f"], r["g"], r["model"] = f, g, m
    return r


def assert_parity(gpu, ref, field_tol=FIELD_TOL, nu_tol=NU_TOL):
    for name in ("u", "v", "theta"):
        e = rel_err(gpu[name], ref[name])
        assert e <= field_tol, f"{name}: {e:.3e}"
    nu_ref = ref["nu_series"]
    assert len(gpu["nu_series"]) == len(nu_ref)
    e = (np.abs(gpu["nu_series"] - nu_ref) / np.abs(nu_ref)).max()
    assert e <= nu_tol, f"Nu series: {e:.3e}"
    e = np.abs(gpu["nu_local"] - ref["nu_local"]).max() / np.abs(ref["nu_local"]).max()
    assert e <= nu_tol, f"local Nu: {e:.3e}"


KERNELS = [0, 1, 2]  # DMRT_KERNEL_AUTO, DMRT_KERNEL_DIRECT, DMRT_KERNEL_TMA
KERNEL_IDS = ["auto", "direct", "tma"]


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
def test_parity_cavity_64_1000_steps(D, kernel):
    # 64 x 64, Ra 1e4, Pr 0.01, alpha 0.1, seeded 1e-6 noise (the paper's Case 1).
    cav = inputs.cavity_64()
    assert_parity(gpu_run(D, cav, 1000, kernel=kernel), oracle_run(cav, 1000))


def test_parity_oscillatory_256_1000_steps(D):
    cav = inputs.cavity_256_oscillatory()
    assert_parity(gpu_run(D, cav, 1000), oracle_run(cav, 1000))


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("nx,ny", [(300, 70), (67, 45), (130, 9), (2, 2), (5, 3), (3, 17), (129, 130),
                                   (600, 33), (497, 12)])
def test_parity_ragged_shapes(D, nx, ny, kernel):
    # Several tiles in x and y with ragged tails, and degenerate tiny grids. Ra is
    # chosen for Ma = 0.1 (Ma = sqrt(3) alpha sqrt(Ra Pr) / H, from Eq. 9): the
    # method is a low-Mach scheme, and a fixed Ra in a few-row box would drive
    # Ma far above 0.3, where no lattice Boltzmann result is meaningful.
    Pr, alpha, Ma = 0.01, 0.1, 0.1
    Ra = (Ma * ny / (np.sqrt(3) * alpha)) ** 2 / Pr
    cav = inputs.Cavity(nx, ny, Ra, Pr, alpha, noise_amp=1e-2, seed=nx * 1000 + ny)
    assert_parity(gpu_run(D, cav, 300, kernel=kernel), oracle_run(cav, 300))


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
def test_parity_wall_profile_and_adiabatic_right_wall(D, kernel):
    cav = inputs.Cavity(96, 80, 1e5, 0.005, noise_amp=1e-3, seed=21)
    cav.theta_hot_profile = 0.5 + 0.05 * np.sin(np.linspace(0, 3, 80))
    g = gpu_run(D, cav, 500, right_wall=D.DMRT_WALL_ADIABATIC, kernel=kernel)
    r = oracle_run(cav, 500, right_bc=O.WALL_ADIABATIC)
    assert_parity(g, r)


def test_parity_adjoint_config_shape(D):
    # 128 x 128, Ra 1e5, Pr 0.01 with the perturbed hot-wall profile 0.5 + 0.01 N(0,1).
    cav = inputs.cavity_128_adjoint()
    assert_parity(gpu_run(D, cav, 1000), oracle_run(cav, 1000))


def test_energy_conserved_with_adiabatic_walls(D):
    # All walls adiabatic (bounce-back, Eq. 44) and the collision conserving theta
    # (Q_1 = 0, Eq. 38): the heat content stays constant up to float32 rounding,
    # summed in float64 on the GPU by dmrt_energy, and no heat crosses a wall.
    cav = inputs.Cavity(100, 60, 1e5, 0.01, noise_amp=0.2, seed=22)
    p = D.make_params(cav.nx, cav.ny, cav.Ra, cav.Pr, left_wall=D.DMRT_WALL_ADIABATIC,
                      right_wall=D.DMRT_WALL_ADIABATIC)
    sim = D.Cavity2D(p, theta0=cav.theta0())
    e0, w0 = sim.energy()
    sim.step(2000)
    sim.check()
    e1, w1 = sim.energy()
    sim.close()
    assert w0 == 0.0 and w1 == 0.0
    assert abs(e0 - cav.theta0().sum()) <= 1e-6 * np.abs(cav.theta0()).sum()  # float32 initial state
    assert abs(e1 - e0) <= 1e-6 * np.abs(cav.theta0()).sum()


@pytest.mark.parametrize("storage", [0, 1, 3, 4], ids=["fp32", "fp16", "mixed", "theta32"])
@pytest.mark.parametrize("walls", [(0, 0), (0, 1), (1, 0)], ids=["fixed_fixed", "fixed_adiabatic", "adiabatic_fixed"])
def test_energy_budget_with_fixed_temperature_walls(D, storage, walls):
    # Over one step the heat content changes by exactly the wall heat input of
    # the step before it (Eqs. 44-45), up to float32 rounding of each node's
    # populations; both sums come from dmrt_energy and are checked against the
    # same sums taken in numpy from the state that dmrt_get_state returns.
    cav = inputs.Cavity(300, 70, 1e5, 0.01, noise_amp=1e-3, seed=23)
    cav.theta_hot_profile = 0.5 + 0.05 * np.sin(np.linspace(0, 3, cav.ny))
    sim = D.Cavity2D.from_inputs(cav, storage=storage, left_wall=walls[0], right_wall=walls[1])
    sim.step(300)
    st = sim.get_state().astype(np.float64)
    e0, w0 = sim.energy()
    k = sim.consts
    sim.step(1)
    sim.check()
    e1, _ = sim.energy()
    sim.close()
    g = st[9:]
    hot = cav.theta_hot_profile.astype(np.float32).astype(np.float64)
    w_ref = 0.0
    if walls[0] == 0:
        w_ref += np.sum(k.abb * hot - 2.0 * g[3, :, 0])
    if walls[1] == 0:
        w_ref += np.sum(k.abb * cav.theta_cold - 2.0 * g[1, :, -1])
    n = cav.nx * cav.ny
    scale = np.abs(g).sum()
    # THETA32 sums its stored theta; dmrt_get_state rebuilds the populations
    # from theta and the deviations in float32, which sum to theta to rounding.
    assert abs(e0 - g.sum()) <= (1e-6 if storage == 4 else 1e-12) * scale
    assert abs(w0 - w_ref) <= 1e-6 * (abs(w_ref) + cav.ny)
    # Rounding unit of the stored heat: THETA32 keeps theta in float32.
    u = {0: 2.0 ** -24, 1: 2.0 ** -11, 3: 2.0 ** -24, 4: 2.0 ** -24}[storage]
    tol = 10 * u * scale + 1e-6 * abs(w0)
    assert abs((e1 - e0) - w0) <= tol, (e1 - e0, w0)
    if storage == 0 and walls != (0, 0):
        # One heated wall: the heat input is far above the rounding allowance, so
        # a dropped or mis-signed wall term would fail. (With both walls fixed at
        # +-0.5 the two inputs nearly cancel by the cavity's symmetry.)
        assert abs(w0) > 1e3 * tol


def _random_state(nx, ny, seed):
    # A plausible post-collision state: shifted D2Q9 equilibria of random
    # (delta-rho, u, v) plus noise, and D2Q5 populations around theta in [-0.5, 0.5].
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    r = inputs.uniform01(seed, 4 * nx * ny).reshape(4, ny, nx)
    drho, u, v = 2e-3 * (r[0] - 0.5), 0.1 * (r[1] - 0.5), 0.1 * (r[2] - 0.5)
    th = r[3] - 0.5
    eu = ex[:, None, None] * u + ey[:, None, None] * v
    f = w9[:, None, None] * (drho + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u * u + v * v))
    f += 1e-4 * (inputs.uniform01(seed + 1, 9 * nx * ny).reshape(9, ny, nx) - 0.5)
    g = np.empty((5, ny, nx))
    g[0] = 0.3 * th
    g[1:] = 0.175 * th
    g += 1e-2 * (inputs.uniform01(seed + 2, 5 * nx * ny).reshape(5, ny, nx) - 0.5)
    return np.concatenate([f, g]).astype(np.float32)


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
@pytest.mark.parametrize("nx,ny", [(4096, 4096), (32768, 5), (6, 32768)])
def test_one_step_from_random_state_full_size(D, nx, ny, kernel):
    # The largest single cavity (4096^2, the benchmark's launch configuration) and the
    # maximum extents: every population after one step, from the same float32 state.
    cav = inputs.Cavity(nx, ny, 1e7 if nx == ny else 1e5, 0.001, noise_amp=0.0)
    state = _random_state(nx, ny, seed=31)
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=16, kernel=kernel)
    sim.set_state(state)
    sim.step(1)
    sim.check()
    out = sim.get_state()
    nu_mean, nu_local, _ = sim.nusselt()
    sim.close()

    m = O.derive(nx, ny, cav.Ra, cav.Pr, cav.alpha)
    s64 = state.astype(np.float64)
    del state
    r = O.step(m, np.ascontiguousarray(s64[:9]), np.ascontiguousarray(s64[9:]))
    del s64
    for k in range(9):
        ref = r["f"][k]
        assert np.abs(out[k] - ref).max() <= FIELD_TOL * np.abs(ref).max(), f"f{k + 1}"
    for k in range(5):
        ref = r["g"][k]
        assert np.abs(out[9 + k] - ref).max() <= FIELD_TOL * np.abs(ref).max(), f"g{k + 1}"
    assert abs(nu_mean - r["nu"]) <= NU_TOL * abs(r["nu"])
    assert np.abs(nu_local - r["nu_local"]).max() <= NU_TOL * np.abs(r["nu_local"]).max()


@pytest.mark.parametrize("kernel", KERNELS, ids=KERNEL_IDS)
def test_deterministic_and_graph_equals_single_launches(D, kernel):
    cav = inputs.Cavity(700, 150, 1e5, 0.005, noise_amp=1e-3, seed=23)
    a = D.Cavity2D.from_inputs(cav, kernel=kernel)
    a.step(200)  # graphs of 64 steps plus single launches
    b = D.Cavity2D.from_inputs(cav, kernel=kernel)
    for _ in range(200):
        b.step(1)
    c = D.Cavity2D.from_inputs(cav, kernel=kernel)
    c.step(200)
    sa, sb, sc = a.get_state(), b.get_state(), c.get_state()
    na, nb, nc = a.nusselt(200)[2], b.nusselt(200)[2], c.nusselt(200)[2]
    for s in (a, b, c):
        s.close()
    assert np.array_equal(sa, sb) and np.array_equal(sa, sc)
    assert np.array_equal(na, nb) and np.array_equal(na, nc)


TMA_TILES = tune.SINGLE_TILES_FP32  # every compiled float32 tile


def test_all_kernel_variants_agree_bitwise(D):
    # Every variant computes the same per-node arithmetic on the same pulled values:
    # the direct kernel and every compiled TMA tile give identical bits, including
    # the Nusselt series, over several steps from a random state.
    nx, ny, steps = 1000, 301, 5
    cav = inputs.Cavity(nx, ny, 1e6, 0.005, noise_amp=0.0)
    state = _random_state(nx, ny, seed=41)
    outs = []
    for kernel, (npt, R, S) in [(1, (0, 0, 0))] + [(2, t) for t in TMA_TILES]:
        sim = D.Cavity2D.from_inputs(cav, kernel=kernel, tma_rows=R, tma_stages=S, tma_npt=npt)
        sim.set_state(state)
        sim.step(steps)
        sim.check()
        outs.append((sim.get_state(), sim.nusselt(steps)[2], (kernel, npt, R, S)))
        sim.close()
    ref_state, ref_nu, _ = outs[0]
    for st, nu, tag in outs[1:]:
        assert np.array_equal(st, ref_state), tag
        assert np.array_equal(nu, ref_nu), tag


def test_state_roundtrip_resumes_bitwise(D):
    cav = inputs.Cavity(64, 48, 1e5, 0.01, noise_amp=1e-3, seed=24)
    a = D.Cavity2D.from_inputs(cav)
    a.step(150)
    mid = a.get_state()
    a.step(150)
    end_a = a.get_state()
    b = D.Cavity2D.from_inputs(cav)
    b.set_state(mid)
    b.step(150)
    end_b = b.get_state()
    a.close()
    b.close()
    assert np.array_equal(end_a, end_b)


def test_fields_host_equals_device(D):
    cav = inputs.Cavity(70, 50, 1e5, 0.01, noise_amp=1e-3, seed=25)
    sim = D.Cavity2D.from_inputs(cav)
    sim.step(100)
    dev = [t.cpu().numpy() for t in sim.fields()]
    host = sim.fields_host()
    sim.close()
    for a, b in zip(dev, host):
        assert np.array_equal(a, b)


def test_nusselt_ring_wraps(D):
    cav = inputs.Cavity(32, 32, 1e4, 0.01, noise_amp=1e-3, seed=26)
    a = D.Cavity2D.from_inputs(cav, nu_capacity=50)
    b = D.Cavity2D.from_inputs(cav)
    a.step(123)
    b.step(123)
    sa = a.nusselt(1000)[2]
    sb = b.nusselt(1000)[2]
    s7 = a.nusselt(7)[2]
    a.close()
    b.close()
    assert len(sa) == 50 and len(sb) == 123
    assert np.array_equal(sa, sb[-50:])
    assert np.array_equal(s7, sb[-7:])


def test_non_finite_state_is_reported(D):
    cav = inputs.Cavity(40, 30, 1e4, 0.01, noise_amp=0.0)
    th = cav.theta0()
    th[10, 20] = np.nan
    sim = D.Cavity2D(D.make_params(40, 30, 1e4, 0.01), theta0=th)
    sim.step(3)
    with pytest.raises(D.DmrtError) as ei:
        sim.check()
    assert ei.value.code == D.DMRT_E_DIVERGED
    sim.close()


@pytest.mark.parametrize("storage", [0, 1, 3], ids=["fp32", "fp16", "mixed"])
def test_flux_nusselt_matches_oracle(D, storage):
    # The link-flux estimator (dmrt_nusselt_flux) on the GPU's own state equals
    # the oracle's definition evaluated on that state, and after 500 steps it
    # stays within the Nusselt tolerance of the oracle's own run.
    cav = inputs.Cavity(130, 97, 3e4, 0.01, noise_amp=1e-3, seed=29)
    prof = 0.5 + 0.02 * np.cos(np.arange(97) / 9.0)
    sim = D.Cavity2D.from_inputs(cav, storage=storage, nu_capacity=600)
    D.dmrt_set_wall_profiles(sim.h, hot=prof)
    sim.step(500)
    sim.check()
    mean, local = sim.nusselt_flux()
    state = sim.get_state().astype(np.float64)
    sim.close()
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
    hot32 = prof.astype(np.float32).astype(np.float64)  # the device keeps the wall profile in float32
    ref_mean, ref_local = O.nu_flux(m, state[9:], theta_hot_profile=hot32)
    assert np.abs(local - ref_local).max() <= 1e-9 * np.abs(ref_local).max()
    assert mean == pytest.approx(ref_mean, rel=1e-9)
    if storage == 0:
        f, g = O.init(m, cav.theta0())
        O.run(m, 500, f, g, theta_hot_profile=prof)
        assert mean == pytest.approx(O.nu_flux(m, g, theta_hot_profile=prof)[0], rel=NU_TOL)


def test_flux_nusselt_conduction_limit(D):
    cav = inputs.Cavity(32, 32, 0.0, 0.01, noise_amp=0.0)
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=16)
    sim.step(40000)
    sim.check()
    mean, local = sim.nusselt_flux()
    nu = sim.nusselt()[0]
    sim.close()
    assert mean == pytest.approx(1.0, abs=1e-4) and np.allclose(local, 1.0, atol=1e-4)
    assert nu == pytest.approx(1.0, abs=1e-4)
