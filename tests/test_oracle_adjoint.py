"""Pins of the oracle's discrete adjoint: central finite differences of the fp64
forward run (the definition of the derivative of the discrete objective)."""
import numpy as np
import pytest

import oracle as O
from paper_1601_04633_gb300 import inputs


def test_collide_vjp_matches_finite_differences():
    rng = np.random.default_rng(7)
    m = O.derive(8, 8, 1e6, 0.01, 0.1)
    for _ in range(5):
        f = 0.01 * rng.standard_normal(9)
        g = 0.2 * rng.standard_normal(5)
        x = np.concatenate([f, g])
        lam = rng.standard_normal(14)
        nu, dgb = O.collide_vjp(m, x, lam)
        h = 1e-6
        for c in range(14):
            xp, xm = x.copy(), x.copy()
            xp[c] += h
            xm[c] -= h
            fp, gp, *_ = O.collide_node(m, xp[:9], xp[9:])
            fm, gm, *_ = O.collide_node(m, xm[:9], xm[9:])
            fd = lam @ (np.concatenate([fp, gp]) - np.concatenate([fm, gm])) / (2 * h)
            assert nu[c] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        mp, mm = m.copy(), m.copy()
        mp.gbeta *= 1 + 1e-6
        mm.gbeta *= 1 - 1e-6
        fp, gp, *_ = O.collide_node(mp, f, g)
        fm, gm, *_ = O.collide_node(mm, f, g)
        fd = lam @ (np.concatenate([fp, gp]) - np.concatenate([fm, gm])) / (2e-6 * m.gbeta)
        assert dgb == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("nx,ny,Ra", [(8, 6, 1e5), (5, 7, 3e4)])
def test_adjoint_matches_finite_differences(nx, ny, Ra):
    cav = inputs.Cavity(nx, ny, Ra, 0.01, noise_amp=0.02, seed=9)
    m = O.derive(nx, ny, Ra, 0.01, 0.1)
    steps, avg = 40, 15
    hot = 0.5 + 0.05 * np.cos(np.arange(ny))
    f0, g0 = O.init(m, cav.theta0())
    J, dth, dgb = O.adjoint(m, steps, avg, f0, g0, theta_hot_profile=hot)
    assert J == pytest.approx(O.objective(m, steps, avg, cav.theta0(), hot), rel=1e-14)
    h = 1e-5
    for j in range(ny):
        hp, hm = hot.copy(), hot.copy()
        hp[j] += h
        hm[j] -= h
        fd = (O.objective(m, steps, avg, cav.theta0(), hp) - O.objective(m, steps, avg, cav.theta0(), hm)) / (2 * h)
        assert dth[j] == pytest.approx(fd, rel=1e-6, abs=1e-8), j
    mp, mm = m.copy(), m.copy()
    mp.gbeta *= 1 + 1e-5
    mm.gbeta *= 1 - 1e-5
    fd = (O.objective(mp, steps, avg, cav.theta0(), hot) - O.objective(mm, steps, avg, cav.theta0(), hot)) \
        / (2e-5 * m.gbeta)
    assert dgb == pytest.approx(fd, rel=1e-6, abs=1e-8)
    assert abs(dgb) > 0 and np.abs(dth).max() > 0


def test_transposed_streaming_dot_product():
    # Dot-product test of the adjoint streaming: <S x, y> = <x, S^T y> for the
    # linear part S of the pull-stream with all wall rules (wall temperatures 0),
    # and the hot-wall term: <dS/dtheta_w delta, y> = <delta, dthw(y)>.
    rng = np.random.default_rng(7)
    for nx, ny, left in ((5, 4, O.WALL_FIXED), (7, 3, O.WALL_ADIABATIC)):
        m = O.derive(nx, ny, 1e4, 0.01, 0.1, left_bc=left, right_bc=O.WALL_FIXED)
        lin = m.copy()
        lin.theta_hot = lin.theta_cold = 0.0
        x = rng.standard_normal((14, ny, nx))
        y = rng.standard_normal((14, ny, nx))
        f, g = O.stream(lin, np.ascontiguousarray(x[:9]), np.ascontiguousarray(x[9:]))
        sx = np.concatenate([f, g])
        sty, dthw = O.stream_transpose(m, y)
        assert np.dot(sx.ravel(), y.ravel()) == pytest.approx(np.dot(x.ravel(), sty.ravel()), rel=1e-13)
        delta = rng.standard_normal(ny)
        f1, g1 = O.stream(lin, np.ascontiguousarray(x[:9]), np.ascontiguousarray(x[9:]), theta_hot_profile=delta)
        ds = np.concatenate([f1, g1]) - sx
        lhs = np.dot(ds.ravel(), y.ravel())
        assert lhs == pytest.approx(np.dot(delta, dthw), rel=1e-12, abs=1e-13)
        if left == O.WALL_ADIABATIC:
            assert np.all(dthw == 0.0)
