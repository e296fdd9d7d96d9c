"""The cluster kernel for small float32 cavities (DMRT_KERNEL_CLUSTER): both
population buffers in the shared memory of one thread-block cluster, many
steps per launch. It runs the same per-node arithmetic on the same pulled
values as the other kernels, so states, Nusselt series and per-row Nusselt
numbers must be equal bit for bit to the TMA and direct kernels', over runs of
odd and even lengths and across calls; and the paper's Case 1 workload (64 x 64,
20,000 steps) must meet the oracle tolerances."""
import numpy as np
import pytest

import oracle as O
from paper_1601_04633_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import dmrt

    return dmrt


def _run(D, cav, calls, **kw):
    total = sum(calls)
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=total, **kw)
    for n in calls:
        sim.step(n)
    sim.check()
    out = (sim.get_state(), sim.nusselt(total), sim.launch)
    sim.close()
    return out


@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 128), (37, 23), (100, 70), (130, 17), (2, 2), (5, 31)])
def test_cluster_kernel_bitwise_equal_to_the_others(D, nx, ny):
    # Ra for Ma <= 0.08 in every box (a fixed Ra in a box of a few rows would
    # put the flow far outside any lattice Boltzmann method's validity).
    Ra = min(1e5, (0.08 * ny / (np.sqrt(3) * 0.1)) ** 2 / 0.01)
    cav = inputs.Cavity(nx, ny, Ra, 0.01, noise_amp=1e-3, seed=61)
    cav.theta_hot_profile = 0.5 + 0.03 * np.sin(np.linspace(0, 2, ny))
    calls = [37, 64, 1, 2, 100]
    st_c, (m_c, loc_c, ser_c), launch = _run(D, cav, calls, kernel=D.DMRT_KERNEL_CLUSTER)
    assert launch["kernel"] == D.DMRT_KERNEL_CLUSTER
    for kernel in (D.DMRT_KERNEL_TMA, D.DMRT_KERNEL_DIRECT):
        st, (m, loc, ser), _ = _run(D, cav, calls, kernel=kernel)
        assert np.array_equal(st_c, st), kernel
        assert np.array_equal(ser_c, ser), kernel
        assert np.array_equal(loc_c, loc) and m_c == m, kernel


@pytest.mark.parametrize("cap", [1, 50, 1000, 3000])
def test_cluster_kernel_ring_wraps_like_the_others(D, cap):
    # A run longer than the ring (and than the kernel's on-chip chunk of 1024
    # means): the ring keeps the last `cap` means, as with the TMA kernel.
    cav = inputs.Cavity(48, 40, 1e4, 0.01, noise_amp=1e-3, seed=64)
    out = []
    for kernel in (D.DMRT_KERNEL_CLUSTER, D.DMRT_KERNEL_TMA):
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=cap, kernel=kernel)
        sim.step(2500)
        sim.step(3)
        sim.check()
        out.append(sim.nusselt(5000)[2])
        sim.close()
    assert len(out[0]) == min(cap, 2503)
    assert np.array_equal(out[0], out[1])


def test_cluster_kernel_adiabatic_walls_conserve_energy(D):
    cav = inputs.Cavity(96, 64, 1e5, 0.01, noise_amp=0.2, seed=62)
    p = D.make_params(cav.nx, cav.ny, cav.Ra, cav.Pr, left_wall=D.DMRT_WALL_ADIABATIC,
                      right_wall=D.DMRT_WALL_ADIABATIC, kernel=D.DMRT_KERNEL_CLUSTER)
    sim = D.Cavity2D(p, theta0=cav.theta0())
    e0, _ = sim.energy()
    sim.step(3000)
    sim.check()
    e1, w1 = sim.energy()
    ref = D.Cavity2D(D.make_params(cav.nx, cav.ny, cav.Ra, cav.Pr, left_wall=D.DMRT_WALL_ADIABATIC,
                                   right_wall=D.DMRT_WALL_ADIABATIC), theta0=cav.theta0())
    ref.step(3000)
    assert np.array_equal(sim.get_state(), ref.get_state())
    sim.close()
    ref.close()
    assert w1 == 0.0 and abs(e1 - e0) <= 1e-6 * np.abs(cav.theta0()).sum()


def test_cluster_kernel_case1_against_the_oracle(D):
    # 64 x 64, Ra 1e4, Pr 0.01 (the paper's Case 1), 20,000 steps.
    cav = inputs.cavity_64()
    steps = 20_000
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=steps, kernel=D.DMRT_KERNEL_CLUSTER)
    sim.step(steps)
    sim.check()
    u, v, th = (x.cpu().numpy().astype(np.float64) for x in sim.fields())
    series = sim.nusselt(steps)[2]
    sim.close()
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
    f, g = O.init(m, cav.theta0())
    ref = O.run(m, steps, f, g)
    for name, a in (("u", u), ("v", v), ("theta", th)):
        assert np.abs(a - ref[name]).max() <= 1e-5 * np.abs(ref[name]).max(), name
    assert np.max(np.abs(series - ref["nu_series"]) / np.abs(ref["nu_series"])) <= 1e-4


def test_cluster_kernel_refuses_what_does_not_fit(D):
    p = D.make_params(512, 512, 1e5, 0.01, kernel=D.DMRT_KERNEL_CLUSTER)
    with pytest.raises(D.DmrtError) as ei:
        D.Cavity2D(p)
    assert ei.value.code == D.DMRT_E_ARG
    p = D.make_params(64, 64, 1e5, 0.01, kernel=D.DMRT_KERNEL_CLUSTER, storage=D.DMRT_MIXED)
    with pytest.raises(D.DmrtError):
        D.Cavity2D(p)
