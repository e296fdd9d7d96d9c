"""Discrete adjoint on the GPU: gradients of the mean hot-wall Nusselt number with
respect to the hot-wall temperature profile and Ra.

Checked against the fp64 oracle adjoint (small grids, every component) and
against central finite differences of the fp64 oracle forward run on the
128 x 128, Ra = 1e5, Pr = 0.01 cavity with a perturbed hot-wall profile
(h = 1e-3 absolute for theta_w, 1e-3 relative for Ra), to 1e-4 relative.
The float32 forward and the fp64 finite differences differ by the float32
trajectory error (~1e-6 of the fields), far inside that tolerance.
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_04633_gb300 import inputs

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import dmrt

    return dmrt


# The last case fills the GPU, so its sweep takes one reverse step per launch;
# the others take two.
@pytest.mark.parametrize("nx,ny,Ra,steps,avg", [(24, 20, 1e5, 60, 20), (33, 17, 3e4, 45, 45), (300, 12, 2e3, 30, 7),
                                                (260, 140, 3e4, 25, 9)])
def test_adjoint_matches_oracle_adjoint(D, nx, ny, Ra, steps, avg):
    cav = inputs.Cavity(nx, ny, Ra, 0.01, noise_amp=1e-2, seed=nx + ny)
    cav.theta_hot_profile = 0.5 + 0.03 * np.sin(np.arange(ny))
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=steps)
    J, dth, dRa = sim.adjoint(steps, avg)
    sim.close()
    m = O.derive(nx, ny, Ra, 0.01, 0.1)
    f0, g0 = O.init(m, cav.theta0())
    Jo, dtho, dgbo = O.adjoint(m, steps, avg, f0, g0, theta_hot_profile=cav.theta_hot_profile)
    dRao = dgbo * m.gbeta / Ra
    assert J == pytest.approx(Jo, rel=1e-5)
    assert np.abs(dth - dtho).max() <= REL * np.abs(dtho).max()
    assert dRa == pytest.approx(dRao, rel=REL)


@pytest.mark.parametrize("steps,avg", [(1, 1), (2, 1), (3, 2), (5, 5)])
def test_adjoint_few_steps_against_oracle(D, steps, avg):
    # Fewer steps than one segment: a pair node whose first step lies beyond the
    # run (odd lengths), and the anti-bounce-back term of step 1 after it.
    nx, ny, Ra = 20, 18, 1e5
    cav = inputs.Cavity(nx, ny, Ra, 0.01, noise_amp=1e-2, seed=5)
    cav.theta_hot_profile = 0.5 + 0.03 * np.cos(np.arange(ny))
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=8)
    J, dth, dRa = sim.adjoint(steps, avg)
    sim.close()
    m = O.derive(nx, ny, Ra, 0.01, 0.1)
    f0, g0 = O.init(m, cav.theta0())
    Jo, dtho, dgbo = O.adjoint(m, steps, avg, f0, g0, theta_hot_profile=cav.theta_hot_profile)
    assert J == pytest.approx(Jo, rel=1e-5)
    assert np.abs(dth - dtho).max() <= REL * np.abs(dtho).max()
    # dJ/dRa is exactly 0 for one and two steps (the force reaches the wall
    # temperatures only from the third) and small after.
    assert dRa == pytest.approx(dgbo * m.gbeta / Ra, rel=1e-3, abs=1e-15)


def test_adjoint_store_all_needs_the_cluster_kernel(D):
    # Every state is recorded by the cluster kernel only: a context on the TMA
    # kernel reports no such workspace, and asking for it is refused.
    cav = inputs.Cavity(64, 48, 1e5, 0.01, noise_amp=1e-3, seed=4)
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=50, kernel=2)
    with pytest.raises(ValueError):
        sim.adjoint(50, 10, store="all")
    J1, d1, r1 = sim.adjoint(50, 10)  # auto: checkpoints
    sim.close()
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=50, kernel=3)
    J2, d2, r2 = sim.adjoint(50, 10, store="all")
    sim.close()
    assert J1 == J2 and r1 == r2 and np.array_equal(d1, d2)


def test_adjoint_advances_like_a_forward_run(D):
    cav = inputs.Cavity(130, 40, 1e5, 0.005, noise_amp=1e-3, seed=5)
    a = D.Cavity2D.from_inputs(cav, nu_capacity=500)
    b = D.Cavity2D.from_inputs(cav, nu_capacity=500)
    J, _, _ = a.adjoint(301, 100)
    b.step(301)
    assert a.steps_done == b.steps_done == 301
    assert np.array_equal(a.get_state(), b.get_state())
    assert J == pytest.approx(b.nusselt(100)[2].mean(), rel=1e-14)
    a.close()
    b.close()


def test_adjoint_is_deterministic(D):
    # Every gradient is accumulated in a fixed order (dJ/dgbeta in per-block
    # slots summed in block order, dJ/dtheta_w by one thread per row), so two
    # runs give the same bits.
    cav = inputs.Cavity(200, 90, 1e5, 0.01, noise_amp=1e-3, seed=6)
    out = []
    for _ in range(2):
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=400)
        out.append(sim.adjoint(400, 150))
        sim.close()
    (J1, d1, r1), (J2, d2, r2) = out
    assert J1 == J2 and r1 == r2 and np.array_equal(d1, d2)


@pytest.mark.parametrize("kernel", [1, 2], ids=["direct", "tma"])
def test_adjoint_same_bits_overlapped_or_alternating(D, kernel):
    # Segment recompute on a second stream beside the reverse sweep (the full
    # workspace) or alternating with it (the smallest workspace): the same
    # launches on the same data, so the same bits; 1000 steps = 32 segments,
    # the last one short.
    cav = inputs.Cavity(128, 96, 1e5, 0.01, noise_amp=1e-3, seed=8)
    cav.theta_hot_profile = 0.5 + 0.02 * np.cos(np.arange(96))
    out = []
    for overlap in (True, False):
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=1000, kernel=kernel)
        out.append(sim.adjoint(1000, 300, overlap=overlap))
        sim.close()
    (J1, d1, r1), (J2, d2, r2) = out
    assert J1 == J2 and r1 == r2 and np.array_equal(d1, d2)


def test_adjoint_same_bits_with_every_state_stored(D):
    # A cluster-kernel context may keep every forward state (recorded by the
    # kernel as it steps) instead of checkpoints and segment recomputes: the
    # reverse sweep reads the same states, so every storage mode, and the
    # direct kernel's checkpoints, give the same bits. 1001 steps: the last
    # segment is short and of odd length.
    cav = inputs.Cavity(128, 96, 1e5, 0.01, noise_amp=1e-3, seed=9)
    cav.theta_hot_profile = 0.5 + 0.02 * np.sin(np.arange(96))
    out = []
    for kernel, store, overlap in ((0, "all", True), (0, "checkpoints", True), (0, "checkpoints", False),
                                   (1, "checkpoints", True)):
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=1001, kernel=kernel)
        out.append(sim.adjoint(1001, 250, overlap=overlap, store=store))
        sim.close()
    J0, d0, r0 = out[0]
    for J, d, r in out[1:]:
        assert J == J0 and r == r0 and np.array_equal(d, d0)


@pytest.mark.parametrize("nx,ny", [(128, 128), (600, 40)])
def test_adjoint_same_bits_with_either_step_kernel(D, nx, ny):
    # The segment recompute runs the context's step kernel (direct, or TMA with
    # load maps for every checkpoint and slot); both give the forward run's bits,
    # so the gradients agree bit for bit.
    cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=1e-3, seed=7)
    out = []
    for kernel in (1, 2):
        sim = D.Cavity2D.from_inputs(cav, nu_capacity=300, kernel=kernel)
        out.append(sim.adjoint(300, 100))
        sim.close()
    (J1, d1, r1), (J2, d2, r2) = out
    assert J1 == J2 and r1 == r2 and np.array_equal(d1, d2)


def test_adjoint_config_128_against_finite_differences(D):
    # 128 x 128, Ra 1e5, Pr 0.01, hot wall 0.5 + 0.01 N(0, 1), 10000 steps, J over the last 2000.
    cav = inputs.cavity_128_adjoint()
    steps, avg = 10000, 2000
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=avg)
    J, dth, dRa = sim.adjoint(steps, avg)
    sim.close()
    O.set_threads(0)
    m = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
    th0 = cav.theta0()

    def Jo(profile, model=m):
        return O.objective(model, steps, avg, th0, profile)

    assert J == pytest.approx(Jo(cav.theta_hot_profile), rel=1e-5)
    h = 1e-3
    # A random direction in theta_w, and two single components.
    v = inputs.normal(77, cav.ny)
    v /= np.linalg.norm(v)
    fd = (Jo(cav.theta_hot_profile + h * v) - Jo(cav.theta_hot_profile - h * v)) / (2 * h)
    assert dth @ v == pytest.approx(fd, rel=REL)
    for jrow in (3, 64):
        e = np.zeros(cav.ny)
        e[jrow] = 1.0
        fd = (Jo(cav.theta_hot_profile + h * e) - Jo(cav.theta_hot_profile - h * e)) / (2 * h)
        assert dth[jrow] == pytest.approx(fd, rel=REL, abs=REL * np.abs(dth).max())
    mp = O.derive(cav.nx, cav.ny, cav.Ra * (1 + h), cav.Pr, cav.alpha)
    mm = O.derive(cav.nx, cav.ny, cav.Ra * (1 - h), cav.Pr, cav.alpha)
    fd = (Jo(cav.theta_hot_profile, mp) - Jo(cav.theta_hot_profile, mm)) / (2 * h * cav.Ra)
    assert dRa == pytest.approx(fd, rel=REL)


def test_autograd_function(D):
    import torch

    cav = inputs.Cavity(48, 40, 1e5, 0.01, noise_amp=1e-3, seed=8)
    theta_w = torch.full((40,), 0.5, dtype=torch.float64, requires_grad=True)
    Ra = torch.tensor(1e5, dtype=torch.float64, requires_grad=True)
    J = D.nusselt_objective(theta_w, Ra, cav, 200, 50)
    (2.0 * J).backward()
    sim = D.Cavity2D.from_inputs(inputs.Cavity(48, 40, 1e5, 0.01, noise_amp=1e-3, seed=8), nu_capacity=50)
    D.dmrt_set_wall_profiles(sim.h, hot=np.full(40, 0.5))
    Jr, dth, dRa = sim.adjoint(200, 50)
    sim.close()
    assert float(J.detach()) == pytest.approx(Jr, rel=1e-12)
    assert np.allclose(theta_w.grad.numpy(), 2.0 * dth, rtol=1e-12, atol=0)
    assert float(Ra.grad) == pytest.approx(2.0 * dRa, rel=1e-12)
