"""CPU checks of the C ABI: the library builds, loads and exports every symbol the
header declares, and its host-side parameter logic agrees with the oracle's own
derivation (no GPU work is done here)."""
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def D():
    from paper_1601_04633_gb300 import build

    build.build_library()
    from paper_1601_04633_gb300 import dmrt

    dmrt.load()
    return dmrt


def _declared(header):
    with open(os.path.join(ROOT, "include", header)) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dmrt_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(D):
    names = _declared("dmrt.h")
    assert "dmrt_create" in names and "dmrt_step" in names
    L = D.load()
    for n in names:
        assert hasattr(L, n), n
        assert n in D.SIGNATURES, f"binding lacks {n}"


def test_default_params(D):
    p = D.dmrt_default_params()
    assert (p.nx, p.ny, p.Ra, p.Pr, p.alpha) == (64, 64, 1e4, 0.01, 0.1)
    assert (p.theta_hot, p.theta_cold, p.theta_ref) == (0.5, -0.5, 0.0)
    assert p.storage == D.DMRT_FP32 and p.nu_capacity == 1 << 20
    assert p.rounding == D.DMRT_ROUND_AUTO


def test_auto_rounding_resolves_per_storage(D):
    # AUTO means stochastic rounding for 16-bit and mixed storage (the rounding
    # that keeps the long-run Nusselt number within 1e-3) and nothing for float32:
    # the launch chosen for AUTO is the one chosen for the resolved mode.
    for storage, resolved in ((D.DMRT_FP32, D.DMRT_ROUND_NEAREST), (D.DMRT_FP16, D.DMRT_ROUND_STOCHASTIC),
                              (D.DMRT_BF16, D.DMRT_ROUND_STOCHASTIC), (D.DMRT_MIXED, D.DMRT_ROUND_STOCHASTIC),
                              (D.DMRT_THETA32, D.DMRT_ROUND_STOCHASTIC)):
        for n in (64, 1000, 4096):
            auto = D.make_params(n, n, 1e5, 0.01, storage=storage, rounding=D.DMRT_ROUND_AUTO)
            expl = D.make_params(n, n, 1e5, 0.01, storage=storage, rounding=resolved)
            D.dmrt_derive(auto)
            assert D.dmrt_choose_launch(auto, 152) == D.dmrt_choose_launch(expl, 152)


@pytest.mark.parametrize("nx,ny,Ra,Pr,alpha", [(64, 64, 1e4, 0.01, 0.1), (256, 256, 1e5, 0.005, 0.1),
                                               (4096, 4096, 1e7, 0.001, 0.1), (50, 20, 3e3, 0.7, 0.03)])
def test_derive_matches_oracle(D, nx, ny, Ra, Pr, alpha):
    k = D.dmrt_derive(D.make_params(nx, ny, Ra, Pr, alpha))
    m = O.derive(nx, ny, Ra, Pr, alpha)
    for a, b in ((k.nu, m.nu), (k.s_nu, m.s_nu), (k.s_q, m.s_q), (k.s_e, m.s_e), (k.s_eps, m.s_eps),
                 (k.sig_k, m.sig_k), (k.sig_e, m.sig_e), (k.sig_nu, m.sig_nu), (k.a, m.a),
                 (k.gbeta, m.gbeta), (k.abb, m.abb_coef)):
        assert a == pytest.approx(b, rel=1e-13)
    assert k.fo_per_step == pytest.approx(alpha / ny ** 2, rel=1e-14)


def test_alpha_from_mach(D):
    # Eq. 9: Ma = u_c / c_s with u_c^2 = g beta dT H and g beta dT = Ra nu alpha / H^3.
    k1 = D.dmrt_derive(D.make_params(128, 128, 1e5, 0.01, 0.1))
    k2 = D.dmrt_derive(D.make_params(128, 128, 1e5, 0.01, alpha=0.0, Ma=k1.Ma))
    assert k2.alpha == pytest.approx(0.1, rel=1e-13)
    # Fo = tau Ma / sqrt(3 Ra Pr) (Eq. 21) with tau = t c / H (Eq. 9) equals alpha t / H^2 (Eq. 20).
    t = 1000
    assert (t / 128) * k1.Ma / np.sqrt(3 * 1e5 * 0.01) == pytest.approx(k1.fo_per_step * t, rel=1e-12)


@pytest.mark.parametrize("kw,code", [
    (dict(nx=1), -1), (dict(ny=40000), -1), (dict(Pr=0.0), -1), (dict(Ra=-1.0), -1),
    (dict(alpha=0.0, Ma=0.0), -1), (dict(alpha=0.2), -2), (dict(theta_hot=0.0, theta_cold=0.0), -1),
    (dict(storage=7), -1), (dict(nu_capacity=0), -1), (dict(left_wall=3), -1),
    (dict(rounding=3), -1), (dict(rounding=-1), -1),
    (dict(rounding=1), -1),  # stochastic rounding needs 16-bit storage
    (dict(kernel=4), -1), (dict(kernel=-1), -1),
])
def test_invalid_params_rejected(D, kw, code):
    base = dict(nx=64, ny=64, Ra=1e4, Pr=0.01, alpha=0.1)
    base.update({k: v for k, v in kw.items() if k in base})
    p = D.make_params(**base)
    for k, v in kw.items():
        if k not in base:
            setattr(p, k, v)
    with pytest.raises(D.DmrtError) as ei:
        D.dmrt_derive(p)
    assert ei.value.code == code
    assert D.load().dmrt_last_error(None)


def test_workspace_size(D):
    p = D.make_params(4096, 4096, 1e7, 0.001, 0.1)
    n = D.dmrt_workspace_size(p)
    # Two 14-plane float32 buffers of 4096 x 4096 plus small arrays.
    assert 2 * 14 * 4 * 4096 * 4096 <= n < 2 * 14 * 4 * 4096 * 4096 + (16 << 20)
    p2 = D.make_params(130, 7, 1e4, 0.01, 0.1)
    assert D.dmrt_workspace_size(p2) >= 2 * 14 * 4 * 256 * 7  # rows padded to 128 elements


def test_workspace_size_per_storage(D):
    # Bytes per node and buffer: float32 56, float16 / bfloat16 28, mixed 38
    # (float16 flow, float32 thermal), THETA32 30 (float16 flow and deviations,
    # float32 theta).
    for storage, per_node in ((D.DMRT_FP32, 56), (D.DMRT_FP16, 28), (D.DMRT_BF16, 28), (D.DMRT_MIXED, 38),
                              (D.DMRT_THETA32, 30)):
        p = D.make_params(1024, 512, 1e5, 0.01, 0.1, storage=storage, nu_capacity=1024)
        n = D.dmrt_workspace_size(p)
        assert 2 * per_node * 1024 * 512 <= n < 2 * per_node * 1024 * 512 + (1 << 20), storage


def test_theta32_refused_where_it_has_no_kernel(D):
    # THETA32 runs the single-cavity TMA kernel only: no slabs, no direct kernel.
    p = D.make_params(256, 256, 1e5, 0.01, 0.1, storage=D.DMRT_THETA32)
    with pytest.raises(D.DmrtError) as ei:
        D.dmrt_slab_workspace_size(p, 128)
    assert ei.value.code == D.DMRT_E_ARG
    p.kernel = D.DMRT_KERNEL_DIRECT
    with pytest.raises(D.DmrtError):
        D.dmrt_choose_launch(p, 152)
    p.kernel = D.DMRT_KERNEL_AUTO
    assert D.dmrt_choose_launch(p, 152)[0] == D.DMRT_KERNEL_TMA


def test_create_without_workspace_fails_cleanly(D):
    p = D.make_params(64, 64, 1e4, 0.01, 0.1)
    with pytest.raises(D.DmrtError) as ei:
        D.dmrt_create(p, None, 0, 0, 0)
    assert ei.value.code == D.DMRT_E_ARG


def test_adjoint_workspace_queries_refuse_bad_arguments(D):
    # The three workspace queries (checkpoints overlapped, alternating, every
    # state stored) refuse a missing context or a step count below 1 without
    # touching a GPU; the binding checks its storage-mode argument first.
    import ctypes

    L = D.load()
    n = ctypes.c_size_t()
    for fn in (L.dmrt_adjoint_workspace_size, L.dmrt_adjoint_workspace_min, L.dmrt_adjoint_workspace_all):
        assert fn(None, 10, ctypes.byref(n)) == D.DMRT_E_ARG
    with pytest.raises(ValueError):
        D.Cavity2D.adjoint(object(), 10, 5, store="every")
