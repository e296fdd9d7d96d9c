"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: polynomial
definitions of the moments, textbook equilibria (BGK limit), closed-form
moments of the force, exact conservation laws, the conduction limit, a
matrix-form brute force built with numpy.linalg.inv, and the paper's own
Case 1 numbers (Sec. 4).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import bruteforce as BF
from paper_1601_04633_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


E9 = BF.velocities_d2q9()
E5 = BF.velocities_d2q5()


def _oracle_M():
    return np.stack([O.moments9(np.eye(9)[k]) for k in range(9)], axis=1)


def _oracle_N():
    return np.stack([O.moments5(np.eye(5)[k]) for k in range(5)], axis=1)


# ---- lattices and transforms ---------------------------------------------------

def test_eq23_directions():
    # Eq. 23 evaluated; rows 2-3 of M (Eq. 30) must be e_x and e_y of the same order.
    assert E9.tolist() == [[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]]
    M = _oracle_M()
    assert np.array_equal(M[1], E9[:, 0]) and np.array_equal(M[2], E9[:, 1])


def test_M_rows_are_lallemand_luo_polynomials():
    # Moments of Eq. 29 as polynomials of the velocities (Lallemand & Luo 2000, the
    # MRT source the paper cites): 1, ex, ey, 3|e|^2-4, ex^2-ey^2, ex ey,
    # (3|e|^2-5) ex, (3|e|^2-5) ey, (9|e|^4 - 21|e|^2 + 8)/2.
    ex, ey = E9[:, 0].astype(float), E9[:, 1].astype(float)
    e2 = ex ** 2 + ey ** 2
    expected = np.stack([np.ones(9), ex, ey, 3 * e2 - 4, ex ** 2 - ey ** 2, ex * ey,
                         (3 * e2 - 5) * ex, (3 * e2 - 5) * ey, (9 * e2 ** 2 - 21 * e2 + 8) / 2])
    assert np.array_equal(_oracle_M(), expected)
    assert np.array_equal(_oracle_M(), np.array(_gold("paper_matrices.json")["M"], dtype=float))


def test_M_orthogonal():
    M = _oracle_M()
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    assert np.diag(G).tolist() == [9, 6, 6, 36, 4, 4, 12, 12, 36]


def test_N_rows_and_eq37_reading():
    ex, ey = E5[:, 0].astype(float), E5[:, 1].astype(float)
    e2 = ex ** 2 + ey ** 2
    expected = np.stack([np.ones(5), ex, ey, 5 * e2 - 4, ex ** 2 - ey ** 2])
    N = _oracle_N()
    assert np.array_equal(N, expected)
    G = N @ N.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    assert np.diag(G).tolist() == [5, 2, 2, 20, 4]
    # The printed fifth row is not orthogonal to rows 1 and 3: it cannot be a moment basis row.
    Np = np.array(_gold("paper_matrices.json")["N_printed"], dtype=float)
    assert Np[4] @ Np[0] != 0 and Np[4] @ Np[2] != 0
    assert np.array_equal(Np[:4], N[:4])


def test_inverse_transforms():
    rng = np.random.default_rng(0)
    M = np.array(_gold("paper_matrices.json")["M"], dtype=float)
    for _ in range(5):
        m = rng.standard_normal(9)
        assert np.allclose(O.from_moments9(m), np.linalg.inv(M) @ m, rtol=0, atol=1e-14)
        f = rng.standard_normal(9)
        assert np.allclose(O.from_moments9(O.moments9(f)), f, rtol=0, atol=1e-14)
        g = rng.standard_normal(5)
        assert np.allclose(O.from_moments5(O.moments5(g)), g, rtol=0, atol=1e-14)


# ---- equilibria: BGK limit -----------------------------------------------------

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _textbook_feq(drho, u, v, rho0=1.0):
    # Incompressible D2Q9 equilibrium (He & Luo 1997): w [drho + rho0 (3 e.u + 9/2 (e.u)^2 - 3/2 u^2)].
    eu = E9 @ np.array([u, v])
    return W9 * (drho + rho0 * (3 * eu + 4.5 * eu ** 2 - 1.5 * (u * u + v * v)))


def _textbook_geq(theta, u, v, a):
    # D2Q5 advection-diffusion equilibrium w_k theta (1 + e_k.u / cT^2) with
    # cT^2 = (4+a)/10, w_0 = (1-a)/5, w_{1..4} = (4+a)/20.
    cT2 = (4 + a) / 10
    w = np.array([(1 - a) / 5] + [(4 + a) / 20] * 4)
    return w * theta * (1 + (E5 @ np.array([u, v])) / cT2)


def _model_all_rates(s9, s5):
    m = O.derive(8, 8, 0.0, 0.01, 0.1)
    m.s_rho = m.s_j = m.s_e = m.s_nu = m.s_q = m.s_eps = s9
    m.sig_0 = m.sig_k = m.sig_e = m.sig_nu = s5
    m.gbeta = 0.0
    return m


def test_bgk_limit_d2q9_pins_meq():
    # With all rates equal, MRT is BGK: f* = f - s (f - f_eq). This fixes every
    # entry of Eq. 34, including the factor 3 in m4_eq.
    rng = np.random.default_rng(1)
    for s in (0.7, 1.3, 1.95):
        m = _model_all_rates(s, 1.0)
        for _ in range(10):
            f = 0.01 * rng.standard_normal(9)
            g = np.zeros(5)
            fo, _, u, v, _ = O.collide_node(m, f, g)
            feq = _textbook_feq(f.sum(), u, v)
            assert np.allclose(fo, f - s * (f - feq), rtol=0, atol=1e-15)


def test_bgk_limit_d2q9_detects_m4_typo():
    # The printed m4_eq (-2 drho + rho0 |u|^2) violates the BGK limit.
    u, v, drho = 0.03, -0.02, 0.001
    meq_printed = O.meq9(1.0, drho, u, v)
    meq_printed[3] = -2 * drho + (u * u + v * v)
    feq_printed = O.from_moments9(meq_printed)
    assert not np.allclose(feq_printed, _textbook_feq(drho, u, v), rtol=0, atol=1e-6)
    assert np.allclose(O.from_moments9(O.meq9(1.0, drho, u, v)), _textbook_feq(drho, u, v),
                       rtol=0, atol=1e-16)


def test_bgk_limit_d2q5():
    rng = np.random.default_rng(2)
    for s in (0.8, 1.5):
        m = _model_all_rates(1.0, s)
        for _ in range(10):
            f = 0.01 * rng.standard_normal(9)
            g = 0.3 * rng.standard_normal(5)
            _, go, u, v, th = O.collide_node(m, f, g)
            geq = _textbook_geq(th, u, v, m.a)
            assert np.allclose(go, g - s * (g - geq), rtol=0, atol=1e-15)


def test_derived_constants():
    m = O.derive(64, 64, 1e4, 0.01, 0.1)
    assert m.nu == pytest.approx(1e-3, rel=1e-15)
    assert m.s_nu == pytest.approx(2 / (6e-3 + 1), rel=1e-15)
    assert m.s_q == pytest.approx(8 * (2 - m.s_nu) / (8 - m.s_nu), rel=1e-15)
    # Eq. 39: (1/sigma_nu - 1/2)(1/sigma_k - 1/2) = 1/6 follows from Eq. 40.
    assert (1 / m.sig_nu - 0.5) * (1 / m.sig_k - 0.5) == pytest.approx(1 / 6, rel=1e-14)
    # Eq. 43 round trip and a < 1 (stability, Sec. 3.2).
    assert (4 + m.a) / 10 * (1 / m.sig_k - 0.5) == pytest.approx(0.1, rel=1e-14)
    assert m.a == pytest.approx(2 * math.sqrt(3) - 4, rel=1e-14) and m.a < 1
    # Eq. 45's 2 sqrt(3) alpha equals twice the D2Q5 rest-free weight (4+a)/20.
    assert m.abb_coef == pytest.approx((4 + m.a) / 10, rel=1e-14)
    # Eq. 9: Ra = g beta dT H^3 / (nu alpha); Mach number Ma = sqrt(3 g beta dT H).
    assert m.gbeta * m.dT * 64 ** 3 / (m.nu * m.alpha) == pytest.approx(1e4, rel=1e-14)


# ---- force --------------------------------------------------------------------

def test_force_moments_closed_form():
    # Eq. 26 with p = rho0 cs^2 and f_eq(rho0, u): sum F = 0, sum e F = G,
    # sum e_a e_b F = u_a G_b + u_b G_a - 3 (u.G) u_a u_b (exact for D2Q9, rho0 = 1).
    rng = np.random.default_rng(3)
    for _ in range(20):
        u, v = 0.05 * rng.standard_normal(2)
        G = 1e-4 * rng.standard_normal(2)
        F = O.force9(1.0, u, v, G[0], G[1])
        assert abs(F.sum()) < 1e-19
        assert np.allclose(E9.T @ F, G, rtol=1e-13, atol=0)
        U = np.array([u, v])
        second = np.einsum("k,ka,kb->ab", F, E9.astype(float), E9.astype(float))
        expected = np.outer(U, G) + np.outer(G, U) - 3 * (U @ G) * np.outer(U, U)
        assert np.allclose(second, expected, rtol=1e-12, atol=1e-22)


# ---- streaming and walls ------------------------------------------------------

def test_stream_is_a_permutation_with_bounce_back():
    rng = np.random.default_rng(4)
    m = O.derive(7, 5, 0.0, 0.01, 0.1, left_bc=O.WALL_ADIABATIC, right_bc=O.WALL_ADIABATIC)
    fs = rng.random((9, 5, 7))
    gs = rng.random((5, 5, 7))
    f, g = O.stream(m, fs, gs)
    assert np.array_equal(np.sort(f.ravel()), np.sort(fs.ravel()))
    assert np.array_equal(np.sort(g.ravel()), np.sort(gs.ravel()))
    # Every post-collision value lands at its link's head, or reflects at its tail.
    opp9 = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    for k in range(9):
        for j in range(5):
            for i in range(7):
                di, dj = i + E9[k][0], j + E9[k][1]
                if 0 <= di < 7 and 0 <= dj < 5:
                    assert f[k, dj, di] == fs[k, j, i]
                else:
                    assert f[opp9[k], j, i] == fs[k, j, i]


def test_mass_conservation_closed_cavity():
    c = inputs.Cavity(24, 20, 1e5, 0.01, noise_amp=1e-3, seed=11)
    m = O.derive(c.nx, c.ny, c.Ra, c.Pr, c.alpha)
    f, g = O.init(m, c.theta0())
    r = O.run(m, 400, f, g)
    assert np.abs(r["v"]).max() > 1e-5  # the flow is moving
    assert abs(f.sum()) < 1e-13


def test_energy_conserved_with_adiabatic_walls():
    c = inputs.Cavity(20, 16, 1e5, 0.01, noise_amp=0.2, seed=12)
    m = O.derive(c.nx, c.ny, c.Ra, c.Pr, c.alpha, left_bc=O.WALL_ADIABATIC,
                 right_bc=O.WALL_ADIABATIC)
    f, g = O.init(m, c.theta0())
    e0 = g.sum()
    O.run(m, 300, f, g)
    assert abs(g.sum() - e0) < 1e-12 * max(1.0, abs(e0)) + 1e-12


def test_energy_budget_with_anti_bounce_back():
    # Sum theta after streaming = sum theta* plus, on each fixed-temperature wall link,
    # (2 sqrt(3) alpha theta_w - g*_out) - g*_out.
    c = inputs.Cavity(12, 10, 1e5, 0.01, noise_amp=0.1, seed=13)
    m = O.derive(c.nx, c.ny, c.Ra, c.Pr, c.alpha)
    f, g = O.init(m, c.theta0())
    O.run(m, 50, f, g)
    hot = 0.5 + 0.05 * np.sin(np.arange(10))
    fn, gn = O.stream(m, f, g, theta_hot_profile=hot)
    flux = (m.abb_coef * hot - 2 * g[3, :, 0]).sum() + (m.abb_coef * m.theta_cold - 2 * g[1, :, -1]).sum()
    assert gn.sum() == pytest.approx(g.sum() + flux, abs=1e-13)


def test_conduction_limit_square():
    # Ra = 0: no buoyancy, u stays exactly 0; steady theta is linear through the
    # wall values at x = 0 and x = H; Nu = 1 (Eqs. 18-19).
    m = O.derive(16, 16, 0.0, 0.01, 0.1)
    f, g = O.init(m, np.zeros((16, 16)))
    r = O.run(m, 20000, f, g)
    assert np.all(r["u"] == 0.0) and np.all(r["v"] == 0.0) and np.all(f == 0.0)
    x = np.arange(16) + 0.5
    assert np.abs(r["theta"] - (0.5 - x / 16)[None, :]).max() < 1e-12
    assert r["nu_series"][-1] == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(r["nu_local"], 1.0, atol=1e-12)


def test_flux_nusselt_conduction_limit_and_case1():
    # The secondary estimator (heat carried across the hot wall's links, Eq. 45)
    # is exactly 1 in the square conduction limit, H / width in a rectangle, and
    # agrees with the wall-gradient estimator (Eqs. 18-19) at the steady Case 1
    # state to the discretisation level.
    for nx, ny, expect in ((16, 16, 1.0), (24, 16, 16 / 24)):
        m = O.derive(nx, ny, 0.0, 0.01, 0.1)
        f, g = O.init(m, np.zeros((ny, nx)))
        r = O.run(m, 40000, f, g)
        mean, local = O.nu_flux(m, g)
        assert mean == pytest.approx(expect, abs=1e-12)
        assert np.allclose(local, expect, atol=1e-12)
        assert r["nu_series"][-1] == pytest.approx(expect, abs=1e-12)
    m = O.derive(16, 16, 0.0, 0.01, 0.1, left_bc=O.WALL_ADIABATIC)
    f, g = O.init(m, np.zeros((16, 16)))
    O.run(m, 100, f, g)
    assert O.nu_flux(m, g)[0] == 0.0  # an adiabatic wall carries no heat
    c = inputs.cavity_64()
    m = O.derive(c.nx, c.ny, c.Ra, c.Pr, c.alpha)
    f, g = O.init(m, c.theta0())
    r = O.run(m, 20000, f, g)
    assert O.nu_flux(m, g)[0] == pytest.approx(r["nu_series"][-1], rel=1e-3)


def test_conduction_limit_rectangle_and_other_walls():
    # Width 24, height H = 16: -d theta/dX = H dT / width. Wall temperatures 1 and 0.
    m = O.derive(24, 16, 0.0, 0.01, 0.05, theta_hot=1.0, theta_cold=0.0)
    f, g = O.init(m, np.full((16, 24), 0.5))
    r = O.run(m, 60000, f, g)
    x = np.arange(24) + 0.5
    assert np.abs(r["theta"] - (1.0 - x / 24)[None, :]).max() < 1e-11
    assert r["nu_series"][-1] == pytest.approx(16 / 24, abs=1e-11)


# ---- brute force --------------------------------------------------------------

def _bruteforce_for(m):
    gold = _gold("paper_matrices.json")
    N = np.array(gold["N_printed"], dtype=float)
    N[4, 4] = -1.0  # reading of Eq. 37 pinned by test_N_rows_and_eq37_reading
    return BF.BruteForce(gold["M"], N, m.nx, m.ny,
                         [m.s_rho, m.s_j, m.s_j, m.s_e, m.s_nu, m.s_nu, m.s_q, m.s_q, m.s_eps],
                         [m.sig_0, m.sig_k, m.sig_k, m.sig_e, m.sig_nu],
                         m.a, m.gbeta, m.theta_ref, m.theta_hot, m.theta_cold, m.abb_coef)


@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 3)])
def test_bruteforce_matrix_form(nx, ny):
    rng = np.random.default_rng(5)
    # G ~ 1e-2, so that a wrong force term shows; walls at 1 and 0 (theta_ref = 0.5).
    m = O.derive(nx, ny, 1e5, 0.01, 0.1, theta_hot=1.0, theta_cold=0.0)
    bf = _bruteforce_for(m)
    fs = 1e-2 * rng.standard_normal((9, ny, nx))
    gs = 0.1 * rng.standard_normal((5, ny, nx))
    fo, go = fs.copy(), gs.copy()
    fb, gb = fs.copy(), gs.copy()
    for step in range(10):
        r = O.step(m, fo, go)
        fo, go = r["f"], r["g"]
        fb, gb, thb = bf.step(fb, gb)
        assert np.abs(fo - fb).max() <= 1e-14 * max(1.0, np.abs(fb).max()), step
        assert np.abs(go - gb).max() <= 1e-14 * max(1.0, np.abs(gb).max()), step
        assert np.abs(r["theta"] - thb).max() <= 1e-14 * max(1.0, np.abs(thb).max())


def test_uniform_reference_temperature_stays_at_rest():
    # Eq. 27: G vanishes where theta = theta_l. A closed adiabatic box at a uniform
    # theta equal to the reference stays exactly at rest even at large Ra.
    m = O.derive(9, 7, 1e6, 0.01, 0.1, theta_hot=1.2, theta_cold=0.2,
                 left_bc=O.WALL_ADIABATIC, right_bc=O.WALL_ADIABATIC)
    assert m.theta_ref == pytest.approx(0.7) and m.gbeta > 0
    th = np.full((7, 9), m.theta_ref)
    f, g = O.init(m, th)
    r = O.run(m, 100, f, g)
    assert np.abs(f).max() < 1e-13  # only round-off of theta - theta_ref drives it
    assert np.abs(r["theta"] - m.theta_ref).max() < 1e-13


def test_fields_from_post_collision_state():
    c = inputs.Cavity(12, 12, 1e5, 0.01, noise_amp=0.1, seed=14)
    m = O.derive(c.nx, c.ny, c.Ra, c.Pr, c.alpha)
    f, g = O.init(m, c.theta0())
    O.run(m, 30, f, g)
    r = O.step(m, f, g)
    u, v, t = O.fields_from_post(m, r["f"], r["g"])
    assert np.allclose(u, r["u"], rtol=0, atol=1e-15)
    assert np.allclose(v, r["v"], rtol=0, atol=1e-15)
    assert np.allclose(t, r["theta"], rtol=0, atol=1e-15)


# ---- the paper's own numbers --------------------------------------------------

@pytest.mark.slow
def test_paper_case1_nusselt():
    # Sec. 4, Case 1 (Ra = 1e4, Pr = 0.01): mean Nu 1.95 once steady (after Fo = 3),
    # local Nu maximum 3.02 at Y = 0.30. Grid 64x64, alpha = 0.1 (Fo = alpha t / H^2).
    gold = _gold("paper_case1.json")
    c = inputs.cavity_64()
    m = O.derive(c.nx, c.ny, gold["Ra"], gold["Pr"], c.alpha)
    f, g = O.init(m, c.theta0())
    steps = int(round(gold["steady_after_Fo"] * c.ny ** 2 / c.alpha))
    r = O.run(m, steps, f, g)
    nu = r["nu_series"]
    assert nu[-1] == pytest.approx(gold["nu_avg_steady"], rel=0.02)
    assert abs(nu[-1] - nu[-1000]) < 2e-3  # close to steady
    nl = r["nu_local"]
    Y = (np.arange(c.ny) + 0.5) / c.ny
    assert nl.max() == pytest.approx(gold["nu_local_max"], rel=0.02)
    assert abs(Y[nl.argmax()] - gold["Y_of_nu_local_max"]) <= 1.0 / c.ny
