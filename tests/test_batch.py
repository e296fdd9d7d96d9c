"""Batched sweep: many independent cavities stepped by one launch per time step.

The batched kernel runs the same per-node arithmetic as the single-cavity
kernels on the same pulled values, so every member must match, bit for bit,
the same cavity stepped on its own; a sampled subset of the 64-cavity sweep is
also checked against the fp64 oracle with the parity tolerances.
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


def _uneven():
    # Uneven shapes (ragged strips and row blocks), Ra for Ma <= 0.1, three Prandtl numbers.
    shapes = [(128, 128), (200, 150), (67, 45), (300, 70), (33, 257), (500, 9), (2, 2)]
    out = []
    for k, (nx, ny) in enumerate(shapes):
        Pr = (0.001, 0.005, 0.01)[k % 3]
        Ra = min(1e6, (0.08 * ny / (np.sqrt(3) * 0.1)) ** 2 / Pr)
        out.append(inputs.Cavity(nx, ny, Ra, Pr, noise_amp=1e-3, seed=100 + k))
    return out


@pytest.mark.parametrize("tile", [(1, 4, 2), (1, 1, 2), (2, 2, 2), (4, 4, 2), (4, 1, 4), (2, 1, 3), (2, 2, 3)])
def test_batch_members_match_single_contexts_bitwise(D, tile):
    cavs = _uneven()
    npt, R, S = tile
    b = D.Batch.from_inputs(cavs, opts=dict(tma_npt=npt, tma_rows=R, tma_stages=S, graph_steps=16),
                            nu_capacity=128)
    b.step(37)  # graphs of 16 steps plus single launches
    b.check()
    for i, cav in enumerate(cavs):
        single = D.Cavity2D.from_inputs(cav, nu_capacity=128)
        single.step(37)
        single.check()
        m = b.members[i]
        assert m.steps_done == 37
        assert np.array_equal(m.get_state(), single.get_state()), i
        assert np.array_equal(m.nusselt(37)[2], single.nusselt(37)[2]), i
        single.close()
    b.close()


@pytest.mark.parametrize("storage", [0, 3], ids=["fp32", "mixed_sr"])
@pytest.mark.parametrize("group_kb", [1, 4000])
def test_cavity_groups_give_the_same_bits(D, storage, group_kb):
    # Cavities split into groups (each group stepped for the whole call before
    # the next) give exactly the single launch's results, over calls of odd and
    # even lengths (the launch parity and the work-pool counters of each group).
    cavs = _uneven()
    opts = dict(tma_npt=2, tma_rows=2, tma_stages=2, graph_steps=16)
    ref = D.Batch.from_inputs(cavs, opts=opts, nu_capacity=128, storage=storage)
    grp = D.Batch.from_inputs(cavs, opts=dict(opts, group_bytes=group_kb << 10), nu_capacity=128,
                              storage=storage)
    assert ref.groups == 1 and grp.groups > 1
    if group_kb == 1:
        assert grp.groups == len(cavs)  # every cavity exceeds the limit: one group each
    for n in (21, 16, 3):
        ref.step(n)
        grp.step(n)
    ref.check()
    grp.check()
    for i in range(len(cavs)):
        a, b = ref.members[i], grp.members[i]
        assert a.steps_done == b.steps_done == 40
        assert np.array_equal(a.get_state(), b.get_state()), i
        assert np.array_equal(a.nusselt(40)[2], b.nusselt(40)[2]), i
    ref.close()
    grp.close()


MSTEP_TILES = {0: [(1, 2, 2), (2, 1, 2), (2, 2, 2), (2, 2, 3), (4, 2, 2), (4, 4, 2)],
               3: [(2, 2, 2), (4, 2, 2), (4, 4, 2)]}


@pytest.mark.parametrize("storage,rounding", [(0, 0), (3, 0), (3, 1)], ids=["fp32", "mixed", "mixed_sr"])
@pytest.mark.parametrize("K", [2, 8])
def test_multistep_launches_give_the_same_bits(D, storage, rounding, K):
    # K steps per launch, each cavity's next step gated by its own previous step
    # only: exactly the results of one launch per step, for every compiled tile,
    # over calls of odd and even lengths (graphs of 2K steps, single launches
    # for the rest), with and without cavity groups.
    cavs = _uneven()
    for npt, R, S in MSTEP_TILES[storage]:
        base = dict(tma_npt=npt, tma_rows=R, tma_stages=S, graph_steps=16)
        ref = D.Batch.from_inputs(cavs, opts=base, nu_capacity=128, storage=storage, rounding=rounding)
        runs = [D.Batch.from_inputs(cavs, opts=dict(base, steps_per_launch=K), nu_capacity=128, storage=storage,
                                    rounding=rounding),
                D.Batch.from_inputs(cavs, opts=dict(base, steps_per_launch=K, group_bytes=4000 << 10),
                                    nu_capacity=128, storage=storage, rounding=rounding)]
        for n in (37, 16, 3):
            for b in [ref] + runs:
                b.step(n)
        for b in [ref] + runs:
            b.check()
        for b in runs:
            for i in range(len(cavs)):
                a, m = ref.members[i], b.members[i]
                assert m.steps_done == a.steps_done == 56
                assert np.array_equal(m.get_state(), a.get_state()), (npt, R, S, i)
                assert np.array_equal(m.nusselt(56)[2], a.nusselt(56)[2]), (npt, R, S, i)
            b.close()
        ref.close()


TS_TILES = {0: [(2, 1, 2), (2, 2, 2)], 3: [(2, 2, 2), (4, 2, 2), (4, 4, 2)]}


@pytest.mark.parametrize("storage,rounding", [(0, 0), (3, 0), (3, 1)], ids=["fp32", "mixed", "mixed_sr"])
def test_tensor_store_epilogue_gives_the_same_bits(D, storage, rounding):
    # Results through a shared-memory tile and the cavity's own store maps:
    # exactly the register-store results, for every compiled tile, with groups.
    cavs = _uneven()
    for npt, R, S in TS_TILES[storage]:
        base = dict(tma_npt=npt, tma_rows=R, tma_stages=S, graph_steps=16)
        ref = D.Batch.from_inputs(cavs, opts=base, nu_capacity=64, storage=storage, rounding=rounding)
        runs = [D.Batch.from_inputs(cavs, opts=dict(base, tensor_store=1), nu_capacity=64, storage=storage,
                                    rounding=rounding),
                D.Batch.from_inputs(cavs, opts=dict(base, tensor_store=1, group_bytes=4000 << 10), nu_capacity=64,
                                    storage=storage, rounding=rounding)]
        for b in [ref] + runs:
            b.step(37)
            b.check()
        for b in runs:
            for i in range(len(cavs)):
                assert np.array_equal(b.members[i].get_state(), ref.members[i].get_state()), (npt, R, S, i)
                assert np.array_equal(b.members[i].nusselt(37)[2], ref.members[i].nusselt(37)[2]), (npt, R, S, i)
            b.close()
        ref.close()


@pytest.mark.parametrize("storage,rounding", [(0, 0), (3, 1)], ids=["fp32", "mixed_sr"])
def test_strip_policy_gives_the_same_bits(D, storage, rounding):
    # Strips chosen to fill the blocks (narrower strips, more rows per item)
    # give exactly the widest strips' results, with register and tensor stores
    # and several steps per launch.
    cavs = _uneven() + [inputs.Cavity(192, 96, 1e5, 0.01, noise_amp=1e-3, seed=140),
                        inputs.Cavity(384, 40, 1e5, 0.005, noise_amp=1e-3, seed=141)]
    tiles = [(2, 2, 2), (4, 2, 2)] if storage else [(2, 2, 2), (1, 4, 2)]
    for npt, R, S in tiles:
        base = dict(tma_npt=npt, tma_rows=R, tma_stages=S, graph_steps=16)
        ref = D.Batch.from_inputs(cavs, opts=base, nu_capacity=64, storage=storage, rounding=rounding)
        variants = [dict(base, strip_fill=1)]
        if (npt, R, S) in tune.BATCH_MSTEP_TILES[storage]:
            variants.append(dict(base, strip_fill=1, steps_per_launch=4))
        if (npt, R, S) in TS_TILES[storage]:
            variants.append(dict(base, strip_fill=1, tensor_store=1))
        runs = [D.Batch.from_inputs(cavs, opts=o, nu_capacity=64, storage=storage, rounding=rounding)
                for o in variants]
        for b in [ref] + runs:
            b.step(36)
            b.check()
        for b in runs:
            for i in range(len(cavs)):
                assert np.array_equal(b.members[i].get_state(), ref.members[i].get_state()), (npt, R, S, i)
                assert np.array_equal(b.members[i].nusselt(36)[2], ref.members[i].nusselt(36)[2]), (npt, R, S, i)
            b.close()
        ref.close()


def test_multistep_sweep_member_matches_single_context(D):
    # The 64-cavity sweep, 8 steps per launch: sampled members against their own
    # contexts stepped alone.
    cavs = inputs.batch_sweep()
    b = D.Batch.from_inputs(cavs, opts=dict(tma_npt=2, tma_rows=2, tma_stages=2, steps_per_launch=8),
                            nu_capacity=64)
    b.step(50)
    b.check()
    for i in (0, 17, 63):
        single = D.Cavity2D.from_inputs(cavs[i], nu_capacity=64)
        single.step(50)
        assert np.array_equal(b.members[i].get_state(), single.get_state()), i
        assert np.array_equal(b.members[i].nusselt(50)[2], single.nusselt(50)[2]), i
        single.close()
    b.close()


def test_batch_parity_rule_and_member_stepping(D):
    cavs = _uneven()[:3]
    b = D.Batch.from_inputs(cavs, nu_capacity=64)
    b.step(4)
    b.members[1].step(1)  # stepped on its own: the batch must refuse until it is even again
    with pytest.raises(D.DmrtError) as ei:
        b.step(1)
    assert ei.value.code == D.DMRT_E_STATE
    b.members[1].step(1)
    b.step(3)
    b.check()
    ref = D.Cavity2D.from_inputs(cavs[1], nu_capacity=64)
    ref.step(9)
    assert np.array_equal(b.members[1].get_state(), ref.get_state())
    assert b.members[0].steps_done == 7 and b.members[1].steps_done == 9
    ref.close()
    b.close()


def test_sweep_of_64_cavities_sampled_against_oracle(D):
    # The 64-cavity sweep (sides 128..384, Ra log-uniform in [1e4, 1e6], Pr in
    # {0.001, 0.005, 0.01}); 300 steps; three members against the oracle.
    cavs = inputs.batch_sweep()
    steps = 300
    b = D.Batch.from_inputs(cavs, nu_capacity=steps)
    b.step(steps)
    b.check()
    for i in (0, 17, 63):
        cav = cavs[i]
        m = b.members[i]
        u, v, th = (x.cpu().numpy().astype(np.float64) for x in m.fields())
        series = m.nusselt(steps)[2]
        mo = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
        f, g = O.init(mo, cav.theta0())
        ref = O.run(mo, steps, f, g)
        for name, a in (("u", u), ("v", v), ("theta", th)):
            err = np.abs(a - ref[name]).max() / np.abs(ref[name]).max()
            assert err <= FIELD_TOL, (i, name, err)
        nu_err = (np.abs(series - ref["nu_series"]) / np.abs(ref["nu_series"])).max()
        assert nu_err <= NU_TOL, (i, nu_err)
    b.close()


def test_autotuner_picks_a_compiled_tile(D):
    from paper_1601_04633_gb300 import tune

    cavs = _uneven()[:4]
    r = tune.tune_batch(cavs, steps=20, warmup=4, tiles=[(1, 4, 2), (2, 2, 2)])
    # Each tile with each strip policy.
    assert r["opts"]["tma_npt"] in (1, 2) and len(r["trials"]) == 4
    assert {t["opts"]["strip_fill"] for t in r["trials"]} == {0, 1}
    assert all(t["mlups"] > 0 for t in r["trials"])


@pytest.mark.parametrize("rounding", [0, 1], ids=["nearest", "stochastic"])
@pytest.mark.parametrize("tile", [(1, 4, 2), (2, 2, 2), (4, 4, 2), (1, 1, 2), (2, 1, 2), (2, 2, 3)])
def test_mixed_batch_members_match_single_contexts_bitwise(D, tile, rounding):
    # Mixed storage (float16 flow, float32 thermal populations): the batched
    # kernel stores the same rounded values as the single-cavity kernel (for
    # stochastic rounding, the same bits from each cavity's own step count).
    cavs = _uneven()
    npt, R, S = tile
    b = D.Batch.from_inputs(cavs, opts=dict(tma_npt=npt, tma_rows=R, tma_stages=S, graph_steps=16),
                            nu_capacity=128, storage=D.DMRT_MIXED, rounding=rounding)
    b.step(37)
    b.check()
    for i, cav in enumerate(cavs):
        single = D.Cavity2D.from_inputs(cav, nu_capacity=128, storage=D.DMRT_MIXED, rounding=rounding)
        single.step(37)
        single.check()
        m = b.members[i]
        assert np.array_equal(m.get_state(), single.get_state()), i
        assert np.array_equal(m.nusselt(37)[2], single.nusselt(37)[2]), i
        single.close()
    b.close()


def test_mixed_sweep_sampled_against_oracle(D):
    # The 64-cavity sweep in mixed storage, 2000 steps: sampled members' Nu
    # histories within 1e-3 of the oracle's (the mixed-storage target).
    cavs = inputs.batch_sweep()
    steps = 2000
    b = D.Batch.from_inputs(cavs, nu_capacity=steps, storage=D.DMRT_MIXED)
    b.step(steps)
    b.check()
    for i in (0, 17, 63):
        cav = cavs[i]
        series = b.members[i].nusselt(steps)[2]
        mo = O.derive(cav.nx, cav.ny, cav.Ra, cav.Pr, cav.alpha)
        f, g = O.init(mo, cav.theta0())
        ref = O.run(mo, steps, f, g)
        nu_err = (np.abs(series - ref["nu_series"]) / np.abs(ref["nu_series"])).max()
        assert nu_err <= 1e-3, (i, nu_err)
    b.close()


def test_batch_rejects_unsupported_storage(D):
    cavs = _uneven()[:2]
    with pytest.raises(D.DmrtError):
        D.Batch.from_inputs(cavs, storage=D.DMRT_FP16)
