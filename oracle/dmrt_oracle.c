/*
 * FP64 CPU oracle for the double-MRT thermal lattice Boltzmann time step of
 * Li, Yang & Zhang, "Double MRT thermal lattice Boltzmann method for
 * simulating natural convection of low Prandtl number fluids" (arXiv 1601.04633).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file. The product (CUDA) path never calls
 * it, and the two share no code, headers, tables or constants.
 *
 * Everything here is deliberately plain: dense 9x9 / 5x5 matrices typed from
 * the paper, inverses computed by Gauss-Jordan elimination, one loop per stage
 * of the algorithm, fp64 throughout, a fresh temporary array per stage.
 *
 * Stage order of one time step (Sec. 3; the initial arrays are a
 * post-collision state, so each step starts with streaming):
 *   1. stream f  (Eq. 25, left-hand side), half-way bounce-back at walls
 *   2. stream g  (Eq. 36, left-hand side), bounce-back (Eq. 44) on adiabatic
 *      walls, anti-bounce-back (Eq. 45) on fixed-temperature walls
 *   3. macroscopic moments  delta-rho, j = rho0 u (Eq. 33), theta (Eq. 41)
 *   4. D2Q9 MRT collision  (Eqs. 28-32, 34)
 *   5. buoyancy force      (Eqs. 26-27) added to the post-collision f
 *   6. D2Q5 MRT collision  (Eqs. 36-43)
 *   7. hot-wall Nusselt number from the pre-collision theta (Eqs. 18-19)
 *
 * Readings of the paper taken here (each one also listed in the design notes):
 *   - Eq. 23 evaluated: e2..e5 = (1,0),(0,1),(-1,0),(0,-1);
 *     e6..e9 = (1,1),(-1,1),(-1,-1),(1,-1).
 *   - Eq. 34: m4_eq = -2 drho + 3 rho0 |u|^2 (the printed formula lacks the 3).
 *   - Eq. 37: fifth row of N is (0,1,-1,1,-1) (the printed last entry is +1).
 *   - Eq. 26: p = rho0 cs^2 and f_eq = f_eq(rho0, u) (full, unshifted
 *     equilibrium at the reference density); G = (0, gbeta (theta - theta_ref)).
 *   - gbeta * dT = Ra nu alpha / H^3 with H = ny (from Eq. 9).
 *   - Eq. 43 solved for a: a = 10 alpha / (1/sigma_k - 1/2) - 4.
 *   - Eq. 45: 2 sqrt(3) alpha theta_w, used as printed.
 *   - Nu_j = H (8 theta_w - 9 theta(0,j) + theta(1,j)) / (3 dT): the
 *     second-order one-sided derivative through the wall value and the first
 *     two node values (Eq. 18), mean over rows (Eq. 19, midpoint rule).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "dmrt_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* Lattices (Eq. 23, Eq. 35). Index k = paper index i - 1.                 */

static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int EX5[5] = {0, 1, 0, -1, 0};
static const int EY5[5] = {0, 0, 1, 0, -1};

/* Transform matrix M, Eq. 30, rows m = (rho, jx, jy, e, pxx, pxy, qx, qy, eps). */
static const double M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
};

/* Transform matrix N, Eq. 37, with the fifth row read as (0,1,-1,1,-1). */
static const double N5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1},
};

static double M9inv[9][9];
static double N5inv[5][5];
static int inverses_ready = 0;

/* Plain Gauss-Jordan elimination with partial pivoting; returns 0 on success. */
static int invert(int n, const double *a, double *out) {
    double w[9][18];
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < n; ++c) {
            w[r][c] = a[r * n + c];
            w[r][n + c] = (r == c) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(w[r][c]) > fabs(w[piv][c])) piv = r;
        if (w[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) {
                double t = w[c][k];
                w[c][k] = w[piv][k];
                w[piv][k] = t;
            }
        double d = w[c][c];
        for (int k = 0; k < 2 * n; ++k) w[c][k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double fct = w[r][c];
            if (fct == 0.0) continue;
            for (int k = 0; k < 2 * n; ++k) w[r][k] -= fct * w[c][k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) out[r * n + c] = w[r][n + c];
    return 0;
}

static void ensure_inverses(void) {
    if (inverses_ready) return;
    invert(9, &M9[0][0], &M9inv[0][0]);
    invert(5, &N5[0][0], &N5inv[0][0]);
    inverses_ready = 1;
}

static int opposite9(int k) {
    for (int q = 0; q < 9; ++q)
        if (EX9[q] == -EX9[k] && EY9[q] == -EY9[k]) return q;
    return -1;
}

static int opposite5(int k) {
    for (int q = 0; q < 5; ++q)
        if (EX5[q] == -EX5[k] && EY5[q] == -EY5[k]) return q;
    return -1;
}

/* ---------------------------------------------------------------------- */
/* Parameters (Eqs. 9, 31-32, 38-40, 43).                                  */

int orc_derive(int32_t nx, int32_t ny, double Ra, double Pr, double alpha,
               double theta_hot, double theta_cold, double theta_ref,
               orc_model *m) {
    if (nx < 2 || ny < 2 || !(alpha > 0.0) || !(Pr > 0.0) || !(Ra >= 0.0)) return -1;
    memset(m, 0, sizeof(*m));
    m->nx = nx;
    m->ny = ny;
    m->rho0 = 1.0;
    m->H = (double)ny;
    m->alpha = alpha;
    m->nu = Pr * alpha;                                 /* Pr = nu / alpha */
    m->s_rho = 0.0;
    m->s_j = 1.0;
    m->s_e = m->s_eps = m->s_nu = 2.0 / (6.0 * m->nu + 1.0); /* Eq. 32 */
    m->s_q = 8.0 * (2.0 - m->s_nu) / (8.0 - m->s_nu);        /* Eq. 32 */
    m->sig_0 = 0.0;
    m->sig_k = 1.0 / (0.5 + sqrt(3.0) / 6.0);                /* Eq. 40 */
    m->sig_e = 1.0 / (0.5 + sqrt(3.0) / 3.0);                /* Eq. 40 */
    m->sig_nu = m->sig_e;
    m->a = 10.0 * alpha / (1.0 / m->sig_k - 0.5) - 4.0;      /* Eq. 43 */
    m->theta_hot = theta_hot;
    m->theta_cold = theta_cold;
    m->theta_ref = theta_ref;
    m->dT = theta_hot - theta_cold;
    /* Ra = g beta dT H^3 / (nu alpha), Eq. 9; gbeta is per unit theta. */
    m->gbeta = (m->dT != 0.0) ? Ra * m->nu * alpha / (m->H * m->H * m->H) / m->dT : 0.0;
    m->abb_coef = 2.0 * sqrt(3.0) * alpha;                   /* Eq. 45 */
    m->left_bc = ORC_WALL_FIXED;
    m->right_bc = ORC_WALL_FIXED;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Per-node pieces.                                                        */

void orc_moments9(const double f[9], double m[9]) {
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += M9[r][k] * f[k];
        m[r] = s;
    }
}

void orc_moments5(const double g[5], double n[5]) {
    for (int r = 0; r < 5; ++r) {
        double s = 0.0;
        for (int k = 0; k < 5; ++k) s += N5[r][k] * g[k];
        n[r] = s;
    }
}

void orc_from_moments9(const double m[9], double f[9]) {
    ensure_inverses();
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += M9inv[r][k] * m[k];
        f[r] = s;
    }
}

void orc_from_moments5(const double n[5], double g[5]) {
    ensure_inverses();
    for (int r = 0; r < 5; ++r) {
        double s = 0.0;
        for (int k = 0; k < 5; ++k) s += N5inv[r][k] * n[k];
        g[r] = s;
    }
}

/* Eq. 34 (with m4 read as -2 drho + 3 rho0 |u|^2). */
void orc_meq9(double rho0, double drho, double u, double v, double meq[9]) {
    double uu = u * u + v * v;
    meq[0] = drho;
    meq[1] = rho0 * u;
    meq[2] = rho0 * v;
    meq[3] = -2.0 * drho + 3.0 * rho0 * uu;
    meq[4] = rho0 * (u * u - v * v);
    meq[5] = rho0 * u * v;
    meq[6] = -rho0 * u;
    meq[7] = -rho0 * v;
    meq[8] = drho - 3.0 * rho0 * uu;
}

/* Eq. 42. */
void orc_neq5(double a, double theta, double u, double v, double neq[5]) {
    neq[0] = theta;
    neq[1] = u * theta;
    neq[2] = v * theta;
    neq[3] = a * theta;
    neq[4] = 0.0;
}

/* Eqs. 26-27 with p = rho0 cs^2, cs^2 = 1/3, and f_eq(rho0, u). */
void orc_force9(double rho0, double u, double v, double Gx, double Gy, double F[9]) {
    static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    double cs2 = 1.0 / 3.0;
    double p = rho0 * cs2;
    for (int k = 0; k < 9; ++k) {
        double eu = EX9[k] * u + EY9[k] * v;
        double feq = W9[k] * rho0 * (1.0 + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) -
                                     (u * u + v * v) / (2.0 * cs2));
        double Gdot = Gx * (EX9[k] - u) + Gy * (EY9[k] - v);
        F[k] = Gdot / p * feq;
    }
}

/* One node: collision (Eq. 28) + force (Eq. 26) + thermal collision (Eq. 36). */
void orc_collide_node(const orc_model *md, const double f[9], const double g[5],
                      double fout[9], double gout[5], double *out_u, double *out_v,
                      double *out_theta) {
    double rates9[9] = {md->s_rho, md->s_j,  md->s_j,  md->s_e, md->s_nu,
                        md->s_nu,  md->s_q,  md->s_q,  md->s_eps};
    double rates5[5] = {md->sig_0, md->sig_k, md->sig_k, md->sig_e, md->sig_nu};
    double drho = 0.0, jx = 0.0, jy = 0.0, theta = 0.0;
    for (int k = 0; k < 9; ++k) {
        drho += f[k];
        jx += f[k] * EX9[k];
        jy += f[k] * EY9[k];
    }
    for (int k = 0; k < 5; ++k) theta += g[k];
    double u = jx / md->rho0, v = jy / md->rho0;

    double m[9], meq[9], mstar[9], fc[9], F[9];
    orc_moments9(f, m);
    orc_meq9(md->rho0, drho, u, v, meq);
    for (int r = 0; r < 9; ++r) mstar[r] = m[r] - rates9[r] * (m[r] - meq[r]);
    orc_from_moments9(mstar, fc);
    double Gx = 0.0, Gy = md->gbeta * (theta - md->theta_ref);
    orc_force9(md->rho0, u, v, Gx, Gy, F);
    for (int k = 0; k < 9; ++k) fout[k] = fc[k] + F[k];

    double n[5], neq[5], nstar[5];
    orc_moments5(g, n);
    orc_neq5(md->a, theta, u, v, neq);
    for (int r = 0; r < 5; ++r) nstar[r] = n[r] - rates5[r] * (n[r] - neq[r]);
    orc_from_moments5(nstar, gout);

    if (out_u) *out_u = u;
    if (out_v) *out_v = v;
    if (out_theta) *out_theta = theta;
}

/* ---------------------------------------------------------------------- */
/* Whole-grid pieces. Layout: f[k][j][i] (k plane, j row, i column), dense. */

#define F_AT(arr, k, j, i) (arr)[((size_t)(k) * ny + (j)) * nx + (i)]

void orc_init(const orc_model *md, const double *theta0, double *f, double *g) {
    int nx = md->nx, ny = md->ny;
    for (size_t q = 0; q < (size_t)9 * nx * ny; ++q) f[q] = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double th = theta0[(size_t)j * nx + i];
            double neq[5], geq[5];
            orc_neq5(md->a, th, 0.0, 0.0, neq);
            orc_from_moments5(neq, geq);
            for (int k = 0; k < 5; ++k) F_AT(g, k, j, i) = geq[k];
        }
}

static double wall_theta(const double *prof, double dflt, int j) {
    return prof ? prof[j] : dflt;
}

void orc_stream(const orc_model *md, const double *fs, const double *gs,
                const double *theta_hot_prof, const double *theta_cold_prof,
                double *f, double *g) {
    int nx = md->nx, ny = md->ny;
    /* Eq. 25: f_k(x) <- f*_k(x - e_k); half-way bounce-back where x - e_k is
     * outside the cavity (no-slip walls, Sec. 3.1). */
    for (int k = 0; k < 9; ++k) {
        int kb = opposite9(k);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int si = i - EX9[k], sj = j - EY9[k];
                if (si >= 0 && si < nx && sj >= 0 && sj < ny)
                    F_AT(f, k, j, i) = F_AT(fs, k, sj, si);
                else
                    F_AT(f, k, j, i) = F_AT(fs, kb, j, i);
            }
    }
    /* Eq. 36: g_k(x) <- g*_k(x - u_k). Walls: Eq. 44 on adiabatic walls,
     * Eq. 45 on fixed-temperature walls. */
    for (int k = 0; k < 5; ++k) {
        int kb = opposite5(k);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int si = i - EX5[k], sj = j - EY5[k];
                if (si >= 0 && si < nx && sj >= 0 && sj < ny) {
                    F_AT(g, k, j, i) = F_AT(gs, k, sj, si);
                    continue;
                }
                double back = F_AT(gs, kb, j, i);
                int wall_bc;
                double thw;
                if (si < 0) {
                    wall_bc = md->left_bc;
                    thw = wall_theta(theta_hot_prof, md->theta_hot, j);
                } else if (si >= nx) {
                    wall_bc = md->right_bc;
                    thw = wall_theta(theta_cold_prof, md->theta_cold, j);
                } else {
                    wall_bc = ORC_WALL_ADIABATIC; /* top and bottom, Eq. 44 */
                    thw = 0.0;
                }
                if (wall_bc == ORC_WALL_FIXED)
                    F_AT(g, k, j, i) = md->abb_coef * thw - back; /* Eq. 45 */
                else
                    F_AT(g, k, j, i) = back;                     /* Eq. 44 */
            }
    }
}

int orc_step(const orc_model *md, const double *fs, const double *gs,
             const double *theta_hot_prof, const double *theta_cold_prof,
             double *fs_out, double *gs_out, double *u_out, double *v_out,
             double *theta_out, double *nu_local, double *nu_mean) {
    int nx = md->nx, ny = md->ny;
    size_t n = (size_t)nx * ny;
    double *f = (double *)malloc(9 * n * sizeof(double));
    double *g = (double *)malloc(5 * n * sizeof(double));
    double *th = (double *)malloc(n * sizeof(double));
    if (!f || !g || !th) {
        free(f);
        free(g);
        free(th);
        return -2;
    }
    ensure_inverses();
    orc_stream(md, fs, gs, theta_hot_prof, theta_cold_prof, f, g);

#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double fl[9], gl[5], fo[9], go[5], u, v, t;
            for (int k = 0; k < 9; ++k) fl[k] = F_AT(f, k, j, i);
            for (int k = 0; k < 5; ++k) gl[k] = F_AT(g, k, j, i);
            orc_collide_node(md, fl, gl, fo, go, &u, &v, &t);
            for (int k = 0; k < 9; ++k) F_AT(fs_out, k, j, i) = fo[k];
            for (int k = 0; k < 5; ++k) F_AT(gs_out, k, j, i) = go[k];
            size_t q = (size_t)j * nx + i;
            th[q] = t;
            if (u_out) u_out[q] = u;
            if (v_out) v_out[q] = v;
            if (theta_out) theta_out[q] = t;
        }

    /* Eqs. 18-19 on the pre-collision temperature. */
    double sum = 0.0;
    for (int j = 0; j < ny; ++j) {
        double thw = wall_theta(theta_hot_prof, md->theta_hot, j);
        double t0 = th[(size_t)j * nx + 0];
        double t1 = th[(size_t)j * nx + 1];
        double nuj = (md->dT != 0.0) ? md->H * (8.0 * thw - 9.0 * t0 + t1) / (3.0 * md->dT) : 0.0;
        if (nu_local) nu_local[j] = nuj;
        sum += nuj;
    }
    if (nu_mean) *nu_mean = sum / ny;
    free(f);
    free(g);
    free(th);
    return 0;
}

int orc_run(const orc_model *md, int64_t nsteps, double *fs, double *gs,
            const double *theta_hot_prof, const double *theta_cold_prof,
            double *nu_series, double *u_out, double *v_out, double *theta_out,
            double *nu_local) {
    size_t n = (size_t)md->nx * md->ny;
    double *fb = (double *)malloc(9 * n * sizeof(double));
    double *gb = (double *)malloc(5 * n * sizeof(double));
    if (!fb || !gb) {
        free(fb);
        free(gb);
        return -2;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        int last = (s == nsteps - 1);
        double nu;
        int rc = orc_step(md, fs, gs, theta_hot_prof, theta_cold_prof, fb, gb,
                          last ? u_out : NULL, last ? v_out : NULL,
                          last ? theta_out : NULL, last ? nu_local : NULL, &nu);
        if (rc) {
            free(fb);
            free(gb);
            return rc;
        }
        memcpy(fs, fb, 9 * n * sizeof(double));
        memcpy(gs, gb, 5 * n * sizeof(double));
        if (nu_series) nu_series[s] = nu;
    }
    free(fb);
    free(gb);
    return 0;
}

/* Post-collision state -> macroscopic fields at the same time level.
 * theta = sum g* (the thermal collision conserves theta, Q_1 = 0) and the
 * pre-collision momentum is sum e f* minus the force's momentum rho0 G. */
/* Secondary Nusselt estimator. Over one streaming, the left wall's link of row
 * j brings g_1(0, j) = 2 sqrt(3) alpha theta_w(j) - g*_3(0, j) into the cavity
 * (anti-bounce-back, Eq. 45) and takes g*_3(0, j) out, so the heat entering per
 * row and step is abb theta_w - 2 g*_3. Fourier's law (Eqs. 18-19 in flux form)
 * gives the local Nusselt number Nu_j = H q_j / (alpha dT); an adiabatic left
 * wall (Eq. 44) returns its link unchanged and carries no heat. */
double orc_nu_flux(const orc_model *md, const double *gs, const double *theta_hot_prof, double *local) {
    int ny = md->ny, nx = md->nx;
    double sum = 0.0;
    for (int j = 0; j < ny; ++j) {
        double q = 0.0;
        if (md->left_bc == ORC_WALL_FIXED)
            q = md->abb_coef * wall_theta(theta_hot_prof, md->theta_hot, j) - 2.0 * F_AT(gs, 3, j, 0);
        double nuj = (md->dT != 0.0) ? md->H * q / (md->alpha * md->dT) : 0.0;
        if (local) local[j] = nuj;
        sum += nuj;
    }
    (void)nx;
    return sum / ny;
}

void orc_fields_from_post(const orc_model *md, const double *fs, const double *gs,
                          double *u, double *v, double *theta) {
    int nx = md->nx, ny = md->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double jx = 0.0, jy = 0.0, t = 0.0;
            for (int k = 0; k < 9; ++k) {
                jx += EX9[k] * F_AT(fs, k, j, i);
                jy += EY9[k] * F_AT(fs, k, j, i);
            }
            for (int k = 0; k < 5; ++k) t += F_AT(gs, k, j, i);
            double Gy = md->gbeta * (t - md->theta_ref);
            size_t q = (size_t)j * nx + i;
            u[q] = jx / md->rho0;
            v[q] = (jy - md->rho0 * Gy) / md->rho0;
            theta[q] = t;
        }
}


/* ---------------------------------------------------------------------- */
/* Discrete adjoint of the step (test infrastructure for the GPU adjoint).  */
/*
 * Objective: J = sum_k w_k Nu(k), with Nu(k) the mean hot-wall Nusselt number
 * of step k (Eqs. 18-19) and w_k = 1 / avg_last for the last avg_last steps.
 * Parameters: the hot-wall temperature profile theta_w(j) (Eq. 45 and the Nu
 * stencil) and the buoyancy scale gbeta (Eq. 27; Ra enters only through it).
 *
 * Reverse sweep, step k = N..1, with all forward states kept:
 *   nu     = C'(q_k)^T lambda_k + w_k dNu(k)/dq_k      (q_k: pulled state of step k)
 *   lambda_{k-1} = P^T nu                              (transposed streaming, walls)
 * The local Jacobian C' of the collision (Eqs. 26-36) is formed column by
 * column by complex-step differentiation (Squire & Trapp, SIAM Rev. 1998):
 * dC/dx_m = Im C(x + i h e_m) / h, exact to rounding for this polynomial map.
 */
typedef double complex cplx;

static void collide_cx(const orc_model *md, const cplx f[9], const cplx g[5], cplx gbeta,
                       cplx fout[9], cplx gout[5]) {
    double rates9[9] = {md->s_rho, md->s_j,  md->s_j,  md->s_e, md->s_nu,
                        md->s_nu,  md->s_q,  md->s_q,  md->s_eps};
    double rates5[5] = {md->sig_0, md->sig_k, md->sig_k, md->sig_e, md->sig_nu};
    static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    cplx drho = 0, jx = 0, jy = 0, theta = 0;
    for (int k = 0; k < 9; ++k) {
        drho += f[k];
        jx += f[k] * EX9[k];
        jy += f[k] * EY9[k];
    }
    for (int k = 0; k < 5; ++k) theta += g[k];
    double rho0 = md->rho0;
    cplx u = jx / rho0, v = jy / rho0, uu = u * u + v * v;
    cplx m[9], meq[9], mstar[9];
    for (int r = 0; r < 9; ++r) {
        m[r] = 0;
        for (int k = 0; k < 9; ++k) m[r] += M9[r][k] * f[k];
    }
    meq[0] = drho;
    meq[1] = rho0 * u;
    meq[2] = rho0 * v;
    meq[3] = -2.0 * drho + 3.0 * rho0 * uu;
    meq[4] = rho0 * (u * u - v * v);
    meq[5] = rho0 * u * v;
    meq[6] = -rho0 * u;
    meq[7] = -rho0 * v;
    meq[8] = drho - 3.0 * rho0 * uu;
    for (int r = 0; r < 9; ++r) mstar[r] = m[r] - rates9[r] * (m[r] - meq[r]);
    double cs2 = 1.0 / 3.0, p = rho0 * cs2;
    cplx Gy = gbeta * (theta - md->theta_ref);
    for (int r = 0; r < 9; ++r) {
        cplx acc = 0;
        for (int k = 0; k < 9; ++k) acc += M9inv[r][k] * mstar[k];
        cplx eu = EX9[r] * u + EY9[r] * v;
        cplx feq = W9[r] * rho0 * (1.0 + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
        fout[r] = acc + Gy * (EY9[r] - v) / p * feq;
    }
    cplx n[5], neq[5], nstar[5];
    for (int r = 0; r < 5; ++r) {
        n[r] = 0;
        for (int k = 0; k < 5; ++k) n[r] += N5[r][k] * g[k];
    }
    neq[0] = theta;
    neq[1] = u * theta;
    neq[2] = v * theta;
    neq[3] = md->a * theta;
    neq[4] = 0;
    for (int r = 0; r < 5; ++r) nstar[r] = n[r] - rates5[r] * (n[r] - neq[r]);
    for (int r = 0; r < 5; ++r) {
        cplx acc = 0;
        for (int k = 0; k < 5; ++k) acc += N5inv[r][k] * nstar[k];
        gout[r] = acc;
    }
}

/* Jacobian-transpose product at one node: nu = C'(x)^T lam (x = 9 f then 5 g),
 * and *dgb += lam . dC/dgbeta. */
void orc_collide_vjp(const orc_model *md, const double x[14], const double lam[14], double nu[14],
                     double *dgb) {
    const double h = 1e-30;
    ensure_inverses();
    for (int col = 0; col <= 14; ++col) {
        cplx f[9], g[5], fo[9], go[5];
        for (int k = 0; k < 9; ++k) f[k] = x[k];
        for (int k = 0; k < 5; ++k) g[k] = x[9 + k];
        cplx gb = md->gbeta;
        if (col < 9) f[col] += I * h;
        else if (col < 14) g[col - 9] += I * h;
        else gb += I * h;
        collide_cx(md, f, g, gb, fo, go);
        double acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += lam[k] * cimag(fo[k]) / h;
        for (int k = 0; k < 5; ++k) acc += lam[9 + k] * cimag(go[k]) / h;
        if (col < 14) nu[col] = acc;
        else *dgb += acc;
    }
}

/* Transposed streaming: lprev = S^T nu for the linear part S of orc_stream
 * (Eqs. 25 and 36 with the bounce-back rules, Eqs. 44-45): every pulled entry
 * goes back to where it came from; a bounced link goes back to the node's
 * opposite direction, with a minus sign on a fixed-temperature wall (Eq. 45).
 * There the pulled value also depends on theta_w(j) with coefficient abb_coef,
 * which is added to dthw[j] (left wall only; dthw may be NULL). */
void orc_stream_transpose(const orc_model *md, const double *nu, double *lprev, double *dthw) {
    int nx = md->nx, ny = md->ny;
    size_t n = (size_t)nx * ny, sz = 14 * n;
    for (size_t c = 0; c < sz; ++c) lprev[c] = 0.0;
    for (int k9 = 0; k9 < 9; ++k9) {
        int kb = opposite9(k9);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int si = i - EX9[k9], sj = j - EY9[k9];
                double val = nu[(size_t)k9 * n + (size_t)j * nx + i];
                if (si >= 0 && si < nx && sj >= 0 && sj < ny)
                    lprev[(size_t)k9 * n + (size_t)sj * nx + si] += val;
                else
                    lprev[(size_t)kb * n + (size_t)j * nx + i] += val;
            }
    }
    for (int k5 = 0; k5 < 5; ++k5) {
        int kb = opposite5(k5);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int si = i - EX5[k5], sj = j - EY5[k5];
                double val = nu[(size_t)(9 + k5) * n + (size_t)j * nx + i];
                if (si >= 0 && si < nx && sj >= 0 && sj < ny) {
                    lprev[(size_t)(9 + k5) * n + (size_t)sj * nx + si] += val;
                    continue;
                }
                int bc = si < 0 ? md->left_bc : si >= nx ? md->right_bc : ORC_WALL_ADIABATIC;
                if (bc == ORC_WALL_FIXED) {
                    lprev[(size_t)(9 + kb) * n + (size_t)j * nx + i] -= val; /* Eq. 45 */
                    if (si < 0 && dthw) dthw[j] += md->abb_coef * val;
                } else {
                    lprev[(size_t)(9 + kb) * n + (size_t)j * nx + i] += val; /* Eq. 44 */
                }
            }
    }
}

int orc_adjoint(const orc_model *md, int64_t nsteps, int64_t avg_last, const double *f0,
                const double *g0, const double *theta_hot_prof, double *J, double *dJ_dthw,
                double *dJ_dgbeta) {
    int nx = md->nx, ny = md->ny;
    size_t n = (size_t)nx * ny, sz = 14 * n;
    if (nsteps < 1 || avg_last < 1 || avg_last > nsteps) return -1;
    double *S = (double *)malloc((size_t)(nsteps + 1) * sz * sizeof(double));
    double *q = (double *)malloc(sz * sizeof(double));
    double *lam = (double *)calloc(sz, sizeof(double));
    double *nu = (double *)malloc(sz * sizeof(double));
    double *lprev = (double *)malloc(sz * sizeof(double));
    if (!S || !q || !lam || !nu || !lprev) {
        free(S); free(q); free(lam); free(nu); free(lprev);
        return -2;
    }
    ensure_inverses();
    const double scale = md->dT != 0.0 ? md->H / (3.0 * md->dT) : 0.0;
    memcpy(S, f0, 9 * n * sizeof(double));
    memcpy(S + 9 * n, g0, 5 * n * sizeof(double));
    double Jacc = 0.0;
    for (int64_t k = 1; k <= nsteps; ++k) {
        double *prev = S + (size_t)(k - 1) * sz, *next = S + (size_t)k * sz, nu_k;
        orc_step(md, prev, prev + 9 * n, theta_hot_prof, NULL, next, next + 9 * n, NULL, NULL, NULL,
                 NULL, &nu_k);
        if (k > nsteps - avg_last) Jacc += nu_k / (double)avg_last;
    }
    *J = Jacc;
    for (int j = 0; j < ny; ++j) dJ_dthw[j] = 0.0;
    double dgb = 0.0;
    for (int64_t k = nsteps; k >= 1; --k) {
        const double *prev = S + (size_t)(k - 1) * sz;
        const double w = (k > nsteps - avg_last) ? 1.0 / (double)avg_last : 0.0;
        orc_stream(md, prev, prev + 9 * n, theta_hot_prof, NULL, q, q + 9 * n);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double x[14], l[14], o[14];
                for (int c = 0; c < 14; ++c) {
                    x[c] = q[(size_t)c * n + (size_t)j * nx + i];
                    l[c] = lam[(size_t)c * n + (size_t)j * nx + i];
                }
                orc_collide_vjp(md, x, l, o, &dgb);
                for (int c = 0; c < 14; ++c) nu[(size_t)c * n + (size_t)j * nx + i] = o[c];
            }
        /* Nu(k) = (1/ny) sum_j scale (8 theta_w(j) - 9 theta(0,j) + theta(1,j)), theta = sum g. */
        if (w != 0.0)
            for (int j = 0; j < ny; ++j) {
                for (int c = 9; c < 14; ++c) {
                    nu[(size_t)c * n + (size_t)j * nx + 0] += w * (-9.0 * scale) / ny;
                    nu[(size_t)c * n + (size_t)j * nx + 1] += w * scale / ny;
                }
                dJ_dthw[j] += w * 8.0 * scale / ny;
            }
        orc_stream_transpose(md, nu, lprev, dJ_dthw);
        double *tmp = lam;
        lam = lprev;
        lprev = tmp;
    }
    *dJ_dgbeta = dgb;
    free(S); free(q); free(lam); free(nu); free(lprev);
    return 0;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_abi_version(void) { return 1; }
