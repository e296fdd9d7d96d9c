"""One cavity split into y-slabs (the multi-GPU decomposition), run as several
slab contexts on one GPU: every slab's state must be bit for bit the same rows
of the whole cavity stepped as one context, for every kernel and storage mode,
with the halo rows delivered between steps; the per-row Nusselt numbers agree
bit for bit and the slabs' shares of the mean add up to the cavity's mean (in a
different summation order: within a few units of float64 rounding)."""
import numpy as np
import pytest

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


def _compare(D, cav, parts, steps, **kw):
    from paper_1601_04633_gb300 import slabs

    whole = D.Cavity2D.from_inputs(cav, nu_capacity=steps, **kw)
    whole.step(steps)
    whole.check()
    ref_state = whole.get_state()
    ref_mean, ref_local, ref_series = whole.nusselt(steps)
    whole.close()

    p = D.make_params(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha, theta_hot=cav.theta_hot,
                      theta_cold=cav.theta_cold, theta_init=cav.theta_init, nu_capacity=steps,
                      **{k: v for k, v in kw.items() if k in ("storage", "rounding", "kernel", "tma_npt",
                                                               "tma_rows", "tma_stages")})
    run = slabs.LocalSlabs(p, parts, theta0=cav.theta0(), theta_hot_profile=cav.theta_hot_profile)
    run.step(steps)
    run.check()
    state = run.get_state()
    mean, local, series = run.nusselt(steps)
    run.close()
    assert np.array_equal(state, ref_state)
    assert np.array_equal(local, ref_local)
    assert np.allclose(series, ref_series, rtol=1e-13, atol=0)
    assert mean == pytest.approx(ref_mean, rel=1e-13)


@pytest.mark.parametrize("kernel", [1, 2], ids=["direct", "tma"])
@pytest.mark.parametrize("parts", [2, 3])
def test_slabs_float32_bitwise(D, kernel, parts):
    cav = inputs.Cavity(300, 200, 1e5, 0.01, noise_amp=1e-3, seed=31)
    cav.theta_hot_profile = 0.5 + 0.02 * np.sin(np.linspace(0, 3, cav.ny))
    _compare(D, cav, parts, 1000, kernel=kernel)


@pytest.mark.parametrize("storage,rounding", [(3, 1), (3, 0), (1, 1), (2, 0)],
                         ids=["mixed_sr", "mixed", "fp16_sr", "bf16"])
def test_slabs_16bit_and_mixed_bitwise(D, storage, rounding):
    # TMA kernel with the tensor-store epilogue; stochastic rounding draws on the
    # cavity's row index, so a slab rounds as the whole cavity does.
    cav = inputs.Cavity(1000, 301, 1e6, 0.01, noise_amp=1e-3, seed=32)
    _compare(D, cav, 3, 300, storage=storage, rounding=rounding)


@pytest.mark.parametrize("tile", [(1, 4, 2), (2, 2, 2), (4, 1, 4)])
def test_slabs_ragged_row_blocks(D, tile):
    # Slab heights that do not fill the last row block of the tile.
    cav = inputs.Cavity(600, 90, 1e5, 0.005, noise_amp=1e-3, seed=33)
    npt, R, S = tile
    _compare(D, cav, 4, 200, kernel=2, tma_npt=npt, tma_rows=R, tma_stages=S)


def test_slab_entry_points_refuse_misuse(D):
    import torch

    p = D.make_params(64, 64, 1e4, 0.01)
    s = D.Slab(p, 10, 20)
    with pytest.raises(D.DmrtError) as ei:
        D.dmrt_step(s.h, 2)  # a slab with neighbours steps one step at a time
    assert ei.value.code == D.DMRT_E_STATE
    with pytest.raises(D.DmrtError):
        s.adjoint(10, 5)
    s.close()
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(D.DmrtError) as ei:
        D.dmrt_create_slab(p, 60, 10, None, ws.data_ptr(), 1 << 20, 0)
    assert ei.value.code == D.DMRT_E_ARG
    whole = D.Cavity2D(p)
    with pytest.raises(D.DmrtError):
        D.dmrt_slab_pack(whole.h, 0, 0)  # not a slab
    whole.close()
