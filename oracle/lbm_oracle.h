/*
 * lbm_oracle.h -- plain FP64 CPU oracle of the coupled central-moment lattice
 * Boltzmann (LB) time step of Elbousefi, Schupbach, Premnath & Welch,
 * "Investigation of Surfactant-Laden Bubble Migration Dynamics in
 * Self-Rewetting Fluids using Lattice Boltzmann Method" (arXiv 2408.00146).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * statement of what the GPU path must compute.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, includes or calls it, and it includes nothing
 * from the product library.
 *
 * Layout conventions (shared by value, not by code, with the GPU path):
 *   - lattice nx (periodic x axis) by ny (y axis); node (x, y) is stored at
 *     index y*nx + x;
 *   - walls != 0: rows y = 0 and y = ny-1 are solid wall nodes, rows 1..ny-2
 *     are fluid; walls == 0: every row is fluid and y is periodic;
 *   - populations: [set][alpha][ny][nx], set 0 = f (phase field, App. B),
 *     1 = g (pressure/velocity, App. C), 2 = h (energy, App. D),
 *     3 = q (surfactant, App. E);
 *   - macroscopic fields: [6][ny][nx] in the order phi, u_x, u_y, p, T, psi.
 *
 * Every function returns 0 on success and a negative code on error.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Problem parameters, named as in Sec. 2 and Sec. 6 of the paper. */
typedef struct {
    int32_t nx, ny;      /* lattice size; nx periodic, ny wall-bounded     */
    int32_t walls;       /* 1: solid rows at y=0 and y=ny-1; 0: periodic y  */
    double R;            /* bubble radius: the length scale of Eq. (8)      */
    double xb, yb;       /* bubble centre (used by input generators only)   */
    double W, M_phi;     /* interface width, ACE mobility (Eq. (12))        */
    double rho_A;        /* ambient density                                 */
    double rho_ratio;    /* rho_A / rho_B (Eq. (9))                         */
    double mu_ratio;     /* mu_A / mu_B (Eq. (9))                           */
    double alpha_ratio;  /* alpha_A / alpha_B (Sec. 6: tilde alpha)         */
    double Re, Ma;       /* Eq. (8) with U = U_o of Eq. (21)                */
    double sigma0, sigma_T, sigma_TT, T_ref;  /* Eq. (6)                     */
    double T_H, T_C;     /* wall temperatures at y=0 and y=ny-1             */
    double beta;         /* Gibbs elasticity, Eq. (6)-(7)                   */
    double Pi, Ex;       /* surfactant groups defined after Eq. (11)        */
    double M_psi;        /* surfactant LB diffusivity                       */
    double psi0;         /* initial surfactant level (input generators)     */
    double Fext_x, Fext_y; /* uniform external body force                   */
    double gravity;      /* buoyancy -(rho-rho_A) g along y (Sec. 5.3)      */
    double nu_A;         /* > 0: ambient kinematic viscosity given directly */
    double alpha_A;      /* > 0: ambient thermal diffusivity given directly */
    double psi_L, psi_R; /* surfactant at the y=0 and y=ny-1 ends (Sec. 2, 6) */
    int32_t psi_bc;      /* 0: zero-flux walls; 1: psi fixed to psi_L, psi_R
                            at the wall planes (Sec. 6 main cases); 2: zero
                            flux with psi_L, psi_R only as the initial
                            profile (the variant at the end of Sec. 6)      */
} orc_params;

/* Lattice parameters derived from orc_params (Step P). */
typedef struct {
    double dT, M1, M2, L, U_o;
    double rho_A, rho_B, mu_A, mu_B, nu_A, nu_B, alpha_A, alpha_B;
    double omega_phi, omega_psi;
    double lambda, s, w, m_psi, D_psi;
} orc_derived;

typedef struct orc_sim orc_sim;

int  orc_derive(const orc_params* p, orc_derived* d);
int  orc_create(const orc_params* p, orc_sim** out);
void orc_destroy(orc_sim* s);
int  orc_set_threads(int n);           /* OpenMP threads; returns threads */

/* Populations set to their equilibria built from the given fields. */
int  orc_init_fields(orc_sim* s, const double* fields);
/* Populations copied in directly ([4][9][ny][nx]). */
int  orc_set_populations(orc_sim* s, const double* pops);
int  orc_get_populations(const orc_sim* s, double* pops);
int  orc_step(orc_sim* s, int64_t nsteps);
int64_t orc_time(const orc_sim* s);
/* Macroscopic fields at the current time ([6][ny][nx]; wall rows are 0). */
int  orc_fields(orc_sim* s, double* fields);
/* out[0..8]: t, mass_phi, mass_psi, x_c, y_c, u_bubble_x, u_bubble_y,
 * U_o, t_star.  phi-weighted means over fluid nodes. */
int  orc_observe(orc_sim* s, double* out);

/* Building blocks, exposed so the tests can pin them individually. */
void orc_matrix_P(double* P81);
void orc_matrix_Pinv(double* Pinv81);
void orc_matrix_F(double ux, double uy, double* F81);
void orc_weights(double* w9);
void orc_velocities(int* ex9, int* ey9);
double orc_sigma_eos(const orc_params* p, double T, double psi);
double orc_G(const orc_derived* d, double W, double phi);
double orc_dG(const orc_derived* d, double W, double phi);
/* Generic central-moment collision of one node (App. B-E):
 * out = P^-1 F(-u) [ k + om (eq - k) + (1 - om/2) src ],  k = F(u) P pop.
 * split != 0 relaxes the (20),(02) pair as trace/deviator with om2s, om2d
 * (App. C). */
void orc_cm_collide(const double* pop, double ux, double uy, const double* eq,
                    const double* om, const double* src, int split,
                    double om2s, double om2d, double* out);
/* Isotropic gradient of an nx*ny periodic field at every node. */
int  orc_gradient_periodic(int nx, int ny, const double* a, double* gx, double* gy);

#ifdef __cplusplus
}
#endif
#endif
