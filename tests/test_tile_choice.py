"""The kernel and tile a context chooses (host logic, checked on the CPU through
dmrt_choose_launch, the function dmrt_create itself calls).

The rules are measured choices on a 152-SM GB300: float32 cavities wider than
496 nodes take the TMA kernel with (1, 4, 2); float32 cavities whose rows split
over 16 blocks give at most 1024 nodes per block (up to 128^2) take the cluster
kernel for runs of steps; other small float32 grids take one-row TMA items
while those number at most four per SM ((1, 1, 2) up to two per SM, (2, 1, 3)
beyond), else the direct kernel; 16-bit storage takes
(2, 4, 2) / (4, 4, 2) by rounding, 2-row items while 4-row items would number
fewer than four per SM, one-row items while those number at most two per SM;
mixed storage takes (2, 1, 2). Every chosen tile must be compiled in.
"""
import pytest

from paper_1601_04633_gb300 import inputs

from test_tile_lists import _tables

SMS = 152
DIRECT, TMA, CLUSTER = 1, 2, 3


@pytest.fixture(scope="module")
def D():
    from paper_1601_04633_gb300 import build

    build.build_library()
    from paper_1601_04633_gb300 import dmrt

    dmrt.load()
    return dmrt


def choose(D, nx, ny, storage=0, rounding=0, sms=SMS, **kw):
    cav = inputs.Cavity(nx, ny, 1e5, 0.01, noise_amp=0.0)
    p = D.make_params(nx, ny, cav.Ra, cav.Pr, cav.alpha)
    p.storage, p.rounding = storage, rounding
    for k, v in kw.items():
        setattr(p, k, v)
    return D.dmrt_choose_launch(p, sms)


@pytest.mark.parametrize("n,expect", [
    (4096, (TMA, 1, 4, 2)), (2048, (TMA, 1, 4, 2)), (1000, (TMA, 1, 4, 2)),
    (16, (CLUSTER, 0, 0, 0)), (64, (CLUSTER, 0, 0, 0)), (96, (CLUSTER, 0, 0, 0)),
    (112, (CLUSTER, 0, 0, 0)), (128, (CLUSTER, 0, 0, 0)), (144, (TMA, 1, 1, 2)), (192, (TMA, 1, 1, 2)),
    (256, (TMA, 2, 1, 3)), (304, (TMA, 2, 1, 3)), (384, (DIRECT, 0, 0, 0)), (496, (DIRECT, 0, 0, 0)),
])
def test_float32_square_cavities(D, n, expect):
    assert choose(D, n, n) == expect


@pytest.mark.parametrize("rounding,n,expect", [
    (0, 4096, (TMA, 2, 4, 2)), (1, 4096, (TMA, 4, 4, 2)), (0, 1024, (TMA, 2, 4, 2)),
    (0, 512, (TMA, 2, 2, 2)), (1, 512, (TMA, 4, 2, 2)), (0, 256, (TMA, 2, 2, 2)), (1, 256, (TMA, 4, 2, 2)),
    (0, 128, (TMA, 1, 1, 2)), (1, 128, (TMA, 1, 1, 2)), (0, 64, (TMA, 1, 1, 2)),
])
@pytest.mark.parametrize("storage", [1, 2], ids=["fp16", "bf16"])
def test_16bit_square_cavities(D, storage, rounding, n, expect):
    assert choose(D, n, n, storage, rounding) == expect


@pytest.mark.parametrize("rounding", [0, 1])
@pytest.mark.parametrize("n", [64, 256, 4096])
def test_mixed_storage(D, rounding, n):
    assert choose(D, n, n, 3, rounding) == (TMA, 2, 1, 2)


def test_explicit_choices_are_kept(D):
    assert choose(D, 4096, 4096, kernel=DIRECT) == (DIRECT, 0, 0, 0)
    # The TMA kernel asked for by name keeps the storage's default tile (the
    # small-grid rules belong to AUTO).
    assert choose(D, 64, 64, kernel=TMA) == (TMA, 1, 4, 2)
    assert choose(D, 64, 64, kernel=TMA, tma_npt=4, tma_rows=2, tma_stages=3) == (TMA, 4, 2, 3)
    # A tile given with AUTO keeps the direct kernel on a small float32 grid.
    assert choose(D, 64, 64, tma_rows=2) == (DIRECT, 0, 0, 0)
    with pytest.raises(D.DmrtError):
        choose(D, 64, 64, 1, 0, kernel=DIRECT)  # the direct kernel stores float32 only
    with pytest.raises(D.DmrtError):
        choose(D, 64, 64, sms=0)


def test_the_rules_scale_with_the_sm_count(D):
    # 256^2 float32: 512 one-row items, at most four per SM on 152 SMs, one-row
    # items on 256 SMs (at most two per SM), the direct kernel on 100 SMs.
    assert choose(D, 256, 256, sms=256) == (TMA, 1, 1, 2)
    assert choose(D, 256, 256, sms=100) == (DIRECT, 0, 0, 0)


@pytest.mark.parametrize("storage,rounding", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)])
def test_every_chosen_tile_is_compiled(D, storage, rounding):
    single, _ = _tables()
    shapes = [(nx, ny) for nx in (2, 5, 67, 130, 248, 249, 300, 497, 600, 1000, 4096, 32768)
              for ny in (2, 3, 4, 5, 17, 64, 301, 1024, 4096)]
    for nx, ny in shapes:
        if nx * ny > 1 << 27:
            continue
        k, npt, R, S = choose(D, nx, ny, storage, rounding)
        if k == TMA:
            assert (storage, rounding, npt, R, S) in single, (nx, ny, storage, rounding, (npt, R, S))
        else:
            assert storage == 0 and (npt, R, S) == (0, 0, 0)


def test_auto_takes_the_cluster_kernel_for_small_float32_cavities(D):
    # At most 1024 nodes per block of a 16-block cluster, float32, no tile asked for.
    assert choose(D, 200, 16) == (CLUSTER, 0, 0, 0)      # 1 row of 200 per block
    assert choose(D, 100, 70) == (CLUSTER, 0, 0, 0)      # 5 rows of 100
    assert choose(D, 130, 80) == (CLUSTER, 0, 0, 0)      # 5 rows of 130 = 650
    assert choose(D, 200, 100) != (CLUSTER, 0, 0, 0)     # 7 rows of 200 = 1400
    assert choose(D, 64, 64, 3, 1) == (TMA, 2, 1, 2)     # mixed storage keeps the TMA kernel
    assert choose(D, 64, 64, tma_npt=1, tma_rows=1, tma_stages=2)[0] != CLUSTER  # a tile asked for


def test_cluster_kernel_choice_by_size():
    # Asked for explicitly, the cluster kernel is taken when both float32 buffers
    # fit the shared memory of 16 blocks (64^2, 128^2) and refused otherwise.
    from paper_1601_04633_gb300 import dmrt as D

    for n in (2, 64, 128):
        p = D.make_params(n, n, 1e4, 0.01, kernel=D.DMRT_KERNEL_CLUSTER)
        assert D.dmrt_choose_launch(p, 152) == (D.DMRT_KERNEL_CLUSTER, 0, 0, 0)
    for kw in (dict(nx=512, ny=512), dict(nx=64, ny=64, storage=D.DMRT_MIXED)):
        nx, ny = kw.pop("nx"), kw.pop("ny")
        p = D.make_params(nx, ny, 1e4, 0.01, kernel=D.DMRT_KERNEL_CLUSTER, **kw)
        with pytest.raises(D.DmrtError):
            D.dmrt_choose_launch(p, 152)
