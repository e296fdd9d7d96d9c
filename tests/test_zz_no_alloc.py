"""dmrt_step_noalloc: stepping without any device allocation.

For callers that cannot allocate device memory where they step (a framework
that owns all device memory and hands out only input and output buffers, a
real-time loop in which an allocation would synchronise the device, a plug-in
host that forbids allocation in its callbacks). The entry point keeps its
scratch in a static device array inside the library; these tests call it
through the C ABI and check two calls in a row against the regular entry
points (dmrt_set_state + dmrt_step). Every step kernel of the library computes
the same bits (the parity tests check that across kernels and tiles), so the
states and the Nusselt numbers must be equal exactly, not only within the
parity tolerances. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1601_04633_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1601_04633_gb300 import dmrt

    return torch, dmrt


def _random_state(nx, ny, seed):
    # Shifted D2Q9 equilibria of random (delta-rho, u, v) plus noise, and D2Q5
    # populations around theta in [-0.5, 0.5]; host order f1..f9, g1..g5.
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


def _to_device_layout(torch, D, host):
    _, ny, nx = host.shape
    dev = np.zeros((14, ny, D.device_pitch(nx)), dtype=np.float32)
    for d, h in enumerate(D.DEVICE_PLANE_ORDER):
        dev[d, :, :nx] = host[h]
    return torch.from_numpy(dev).cuda()


def _from_device_layout(D, dev, nx):
    dev = dev.cpu().numpy()
    host = np.empty((14, dev.shape[1], nx), dtype=np.float32)
    for d, h in enumerate(D.DEVICE_PLANE_ORDER):
        host[h] = dev[d, :, :nx]
    return host


def _regular_two_steps(D, cav, state0, hot, cold):
    # The regular entry points: a context with its own workspace.
    sim = D.Cavity2D.from_inputs(cav, nu_capacity=8)
    D.dmrt_set_wall_profiles(sim.h, hot=None if hot is None else hot.astype(np.float64),
                             cold=None if cold is None else cold.astype(np.float64))
    sim.set_state(state0)
    sim.step(1)
    ref1, nu1 = sim.get_state(), sim.nusselt()[0]
    sim.step(1)
    ref2, nu2 = sim.get_state(), sim.nusselt()[0]
    sim.close()
    return ref1, nu1, ref2, nu2


@pytest.mark.parametrize("nx,ny", [(300, 200), (67, 45)])
def test_noalloc_two_calls_match_regular_path(env, nx, ny):
    torch, D = env
    cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=0.0)
    state0 = _random_state(nx, ny, seed=51)
    hot = (0.5 + 0.02 * np.sin(np.linspace(0.0, 3.0, ny))).astype(np.float32)
    ref1, nu1, ref2, nu2 = _regular_two_steps(D, cav, state0, hot, None)

    # No-allocation entry point: caller-owned buffers, two calls in a row (ping-pong).
    p = D.make_params(nx, ny, cav.Ra, cav.Pr, cav.alpha)
    a = _to_device_layout(torch, D, state0)
    b = torch.zeros_like(a)
    hot_dev = torch.from_numpy(hot).cuda()
    nu = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    D.dmrt_step_noalloc(p, a.data_ptr(), b.data_ptr(), nu.data_ptr(), stream, hot_ptr=hot_dev.data_ptr())
    D.dmrt_step_noalloc(p, b.data_ptr(), a.data_ptr(), nu.data_ptr() + 8, stream, hot_ptr=hot_dev.data_ptr())
    torch.cuda.synchronize()
    out1 = _from_device_layout(D, b, nx)
    out2 = _from_device_layout(D, a, nx)
    nus = nu.cpu().numpy()

    assert np.array_equal(out1, ref1)
    assert np.array_equal(out2, ref2)
    assert nus[0] == nu1 and nus[1] == nu2


def test_noalloc_cold_profile_no_output_and_changing_sizes(env):
    # A cold-wall profile given as a device pointer and no Nusselt output (the
    # mean goes to the array's internal sink), then calls on a taller and a
    # shorter cavity in a row: the array keeps the previous call's contents, so
    # each call must reset what its step reads.
    torch, D = env
    stream = torch.cuda.current_stream().cuda_stream
    for nx, ny, want_nu in ((130, 90, False), (96, 400, True), (40, 24, True)):
        cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=0.0)
        state0 = _random_state(nx, ny, seed=52 + ny)
        cold = (-0.5 + 0.03 * np.cos(np.linspace(0.0, 2.0, ny))).astype(np.float32)
        ref1, nu1, ref2, nu2 = _regular_two_steps(D, cav, state0, None, cold)
        p = D.make_params(nx, ny, cav.Ra, cav.Pr, cav.alpha)
        a = _to_device_layout(torch, D, state0)
        b = torch.zeros_like(a)
        cold_dev = torch.from_numpy(cold).cuda()
        nu = torch.zeros(2, dtype=torch.float64, device="cuda")
        out_ptr = (lambda k: nu.data_ptr() + 8 * k) if want_nu else (lambda k: 0)
        D.dmrt_step_noalloc(p, a.data_ptr(), b.data_ptr(), out_ptr(0), stream, cold_ptr=cold_dev.data_ptr())
        D.dmrt_step_noalloc(p, b.data_ptr(), a.data_ptr(), out_ptr(1), stream, cold_ptr=cold_dev.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(_from_device_layout(D, b, nx), ref1), (nx, ny)
        assert np.array_equal(_from_device_layout(D, a, nx), ref2), (nx, ny)
        nus = nu.cpu().numpy()
        if want_nu:
            assert nus[0] == nu1 and nus[1] == nu2, (nx, ny)
        else:
            assert not nus.any()


def test_noalloc_rejects_rows_beyond_its_scratch(env):
    torch, D = env
    ny = D.DMRT_NOALLOC_MAX_NY + 1
    p = D.make_params(8, ny, 1e4, 0.01, 0.1)
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(D.DmrtError) as ei:
        D.dmrt_step_noalloc(p, buf.data_ptr(), buf.data_ptr() + 64, 0, 0)
    assert ei.value.code == D.DMRT_E_ARG
    assert "DMRT_NOALLOC_MAX_NY" in str(ei.value)
