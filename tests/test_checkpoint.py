"""Checkpoint and resume (dmrt_save / dmrt_load).

A run that is saved, loaded into a fresh context and continued must give the
same bits as the uninterrupted run: the population state in its stored
representation (16-bit and mixed storage included), the step counter that
seeds stochastic rounding, the wall profiles and the Nusselt ring all travel in
the checkpoint. Malformed or mismatched checkpoints are refused without
touching the context.
"""
import ctypes

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


def _cav(seed=31, nx=300, ny=70):
    Ra = (0.08 * ny / (np.sqrt(3) * 0.1)) ** 2 / 0.01  # Ma = 0.08
    return inputs.Cavity(nx, ny, Ra, 0.01, noise_amp=1e-3, seed=seed)


@pytest.mark.parametrize("storage,rounding", [(0, 0), (1, 1), (2, 0), (3, 0), (3, 1)],
                         ids=["fp32", "fp16_sr", "bf16", "mixed", "mixed_sr"])
def test_resume_is_bitwise(D, storage, rounding, tmp_path):
    kw = dict(storage=storage, rounding=rounding, nu_capacity=256)
    if storage:
        kw["kernel"] = D.DMRT_KERNEL_TMA
    a = D.Cavity2D.from_inputs(_cav(), **kw)
    prof = 0.5 + 0.01 * np.sin(np.arange(a.ny) / 7.0)
    D.dmrt_set_wall_profiles(a.h, hot=prof)
    a.step(45)
    blob = a.save(tmp_path / "ckpt.bin")
    a.step(40)
    a.check()
    # A context with another initial field and the default walls: all of it is replaced.
    b = D.Cavity2D.from_inputs(_cav(seed=99), **kw)
    b.load(tmp_path / "ckpt.bin")
    assert b.steps_done == 45
    assert blob == b.save()  # a loaded context saves the same checkpoint
    b.step(40)
    b.check()
    assert b.steps_done == 85
    assert np.array_equal(a.get_state(), b.get_state())
    ma, la, sa = a.nusselt(85)
    mb, lb, sb = b.nusselt(85)
    assert ma == mb and np.array_equal(la, lb) and np.array_equal(sa, sb) and len(sa) == 85
    a.close()
    b.close()


def test_ring_capacities_differ(D):
    a = D.Cavity2D.from_inputs(_cav(), nu_capacity=16)
    a.step(45)
    blob = a.save()
    # Larger ring: only the 16 saved values exist before the load point.
    b = D.Cavity2D.from_inputs(_cav(), nu_capacity=128)
    b.load(blob)
    assert len(b.nusselt(128)[2]) == 16
    b.step(10)
    s = b.nusselt(128)[2]
    assert len(s) == 26
    assert np.array_equal(s[:16], a.nusselt(16)[2])
    # Smaller ring: keeps the last 4.
    c = D.Cavity2D.from_inputs(_cav(), nu_capacity=4)
    c.load(blob)
    assert np.array_equal(c.nusselt(4)[2], a.nusselt(4)[2])
    for x in (a, b, c):
        x.close()


def test_bad_checkpoints_are_refused(D):
    a = D.Cavity2D.from_inputs(_cav(), nu_capacity=64)
    a.step(10)
    blob = a.save()
    before = a.get_state()

    other = D.Cavity2D.from_inputs(_cav(nx=301), nu_capacity=64)
    with pytest.raises(D.DmrtError) as e:
        other.load(blob)
    assert e.value.code == D.DMRT_E_STATE
    other.close()

    mixed = D.Cavity2D.from_inputs(_cav(), storage=3, nu_capacity=64)
    with pytest.raises(D.DmrtError) as e:
        mixed.load(blob)
    assert e.value.code == D.DMRT_E_STATE
    mixed.close()

    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 0x01
    with pytest.raises(D.DmrtError) as e:
        a.load(bytes(bad))
    assert e.value.code == D.DMRT_E_STATE
    with pytest.raises(D.DmrtError) as e:
        a.load(blob[:-9])
    assert e.value.code == D.DMRT_E_ARG
    with pytest.raises(D.DmrtError) as e:
        a.load(b"DMRTCKP0" + blob[8:])
    assert e.value.code == D.DMRT_E_STATE
    assert np.array_equal(a.get_state(), before) and a.steps_done == 10

    # Too small a buffer: DMRT_E_SPACE with the needed size reported.
    L = D.load()
    need = ctypes.c_size_t(0)
    small = ctypes.create_string_buffer(64)
    rc = L.dmrt_save(a.h, ctypes.cast(small, ctypes.c_void_p), 64, ctypes.byref(need))
    assert rc == D.DMRT_E_SPACE and need.value == len(blob)
    a.close()
