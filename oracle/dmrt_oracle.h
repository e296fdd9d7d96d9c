/*
 * FP64 CPU oracle of the double-MRT thermal LBM step (arXiv 1601.04633, Sec. 3).
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.
 */
#ifndef DMRT_ORACLE_H
#define DMRT_ORACLE_H
#include <stdint.h>

enum { ORC_WALL_FIXED = 0, ORC_WALL_ADIABATIC = 1 };

typedef struct {
    int32_t nx, ny;
    int32_t left_bc, right_bc; /* ORC_WALL_FIXED (Eq. 45) or ORC_WALL_ADIABATIC (Eq. 44) */
    double rho0, H, alpha, nu;
    double s_rho, s_j, s_e, s_nu, s_q, s_eps; /* S, Eqs. 31-32 */
    double sig_0, sig_k, sig_e, sig_nu;       /* Q, Eqs. 38-40 */
    double a;                                 /* Eq. 43 */
    double theta_hot, theta_cold, theta_ref, dT;
    double gbeta;    /* buoyancy per unit theta: G_y = gbeta (theta - theta_ref) */
    double abb_coef; /* 2 sqrt(3) alpha, Eq. 45 */
} orc_model;

int orc_derive(int32_t nx, int32_t ny, double Ra, double Pr, double alpha,
               double theta_hot, double theta_cold, double theta_ref, orc_model *m);
void orc_moments9(const double f[9], double m[9]);
void orc_moments5(const double g[5], double n[5]);
void orc_from_moments9(const double m[9], double f[9]);
void orc_from_moments5(const double n[5], double g[5]);
void orc_meq9(double rho0, double drho, double u, double v, double meq[9]);
void orc_neq5(double a, double theta, double u, double v, double neq[5]);
void orc_force9(double rho0, double u, double v, double Gx, double Gy, double F[9]);
void orc_collide_node(const orc_model *md, const double f[9], const double g[5],
                      double fout[9], double gout[5], double *u, double *v, double *theta);
void orc_init(const orc_model *md, const double *theta0, double *f, double *g);
void orc_stream(const orc_model *md, const double *fs, const double *gs,
                const double *theta_hot_prof, const double *theta_cold_prof,
                double *f, double *g);
int orc_step(const orc_model *md, const double *fs, const double *gs,
             const double *theta_hot_prof, const double *theta_cold_prof,
             double *fs_out, double *gs_out, double *u_out, double *v_out,
             double *theta_out, double *nu_local, double *nu_mean);
int orc_run(const orc_model *md, int64_t nsteps, double *fs, double *gs,
            const double *theta_hot_prof, const double *theta_cold_prof,
            double *nu_series, double *u_out, double *v_out, double *theta_out,
            double *nu_local);
/* Transposed streaming (the adjoint of the linear part of orc_stream); arrays
 * of 14 planes [14][ny][nx]; adds the hot-wall temperature derivative to dthw. */
void orc_stream_transpose(const orc_model *md, const double *nu, double *lprev, double *dthw);
/* Secondary hot-wall Nusselt number from a post-collision thermal state: the
 * heat the next streaming carries into the cavity across the hot wall's links.
 * local[j] (ny values) and the returned mean over the rows. */
double orc_nu_flux(const orc_model *md, const double *gs, const double *theta_hot_prof, double *local);
void orc_fields_from_post(const orc_model *md, const double *fs, const double *gs,
                          double *u, double *v, double *theta);
/* Discrete adjoint (all forward states kept: small grids). J = mean over the last
 * avg_last steps of the mean hot-wall Nu; gradients w.r.t. the hot-wall profile
 * (ny values) and gbeta. f0/g0: initial post-collision state. */
void orc_collide_vjp(const orc_model *md, const double x[14], const double lam[14], double nu[14],
                     double *dgb);
int orc_adjoint(const orc_model *md, int64_t nsteps, int64_t avg_last, const double *f0,
                const double *g0, const double *theta_hot_prof, double *J, double *dJ_dthw,
                double *dJ_dgbeta);
int orc_set_threads(int n); /* OpenMP threads over rows; returns the count in use */
int orc_abi_version(void);

#endif
