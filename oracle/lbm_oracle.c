/*
 * lbm_oracle.c -- plain FP64 CPU oracle of one time step of the coupled
 * central-moment LB system of arXiv 2408.00146 (four D2Q9 distributions:
 * f for the conservative Allen-Cahn phase field, g for the pressure-based
 * two-fluid flow with capillary and Marangoni forces, h for energy and q for
 * surfactant).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product library.
 *
 * The code follows the paper's algorithm in its own order and notation:
 * raw moments by the matrix P (Eq. (45)), central moments by the binomial
 * frame change F (Eq. (24b), Eq. (46)), relaxation (Eqs. (27), (33), (38),
 * (43)), back-transforms F^-1 = F(-u) and P^-1 (Eqs. (47), (48)), then
 * streaming.  There is no blocking, fusion or reordering: every macroscopic
 * field is a full array, every stencil reads those arrays, and the only
 * concurrency is an OpenMP loop over independent nodes, which does not change
 * any result.
 *
 * Readings where the paper is silent, ambiguous or self-contradictory:
 *   R1  F is built from the binomial expansion of (e-u)^m, as the paper
 *       defines it; the last printed row of F and F^-1 misses two factors 2.
 *   R2  rho = rho_A + phi (rho_B - rho_A), same for mu and alpha: the printed
 *       interpolation (Eq. (17)) returns rho_B at phi = phi_A.
 *   R3  theta = +4 phi (1 - phi) / W: the printed theta has the sign of the
 *       phi_A = 1, phi_B = 0 convention and anti-sharpens with phi_A = 0,
 *       phi_B = 1 (Sec. 3).
 *   R4  the CSF components carry delta_s = 1.5 W |grad phi|^2 (Eq. (15)),
 *       with the -sigma kappa n sign of the printed components (Eq. (16)).
 *   R5  F_p = -grad(p* - rho c_s^2) with p* = sum g of the current step; the
 *       corrected p of Eq. (34) then uses that F_p.
 *   R6  isotropic stencils: grad X = 3 sum_a w_a e_a X(x + e_a); the
 *       curvature is the same stencil applied to the nodal unit normals.
 *   R7  surfactant: the LB diffusivity D_psi is the paper's M_psi, the
 *       adsorption flux coefficient is m_psi = D_psi / lambda, s = 8 sigma0
 *       (so Pi = lambda W^2 / s), w = 4 s / (Ex W^2).
 *   R8  R = G'(phi) grad phi, G the bracket of Eq. (5).
 *   R9  ln(1 - psi) in Eq. (6) uses psi clamped to [0, 1 - 1e-6];
 *       psi (1 - psi) in the surfactant equilibrium uses raw psi.
 *   R10 halfway bounce-back walls for f, g, q; anti-bounce-back (Dirichlet
 *       T_w) for h; stencil ghosts at and beyond the walls are the mirror
 *       images about the wall plane (even for phi, psi, p*, odd about T_w
 *       for T).
 *   R14 the properties rho, mu, alpha are interpolated (R2) with phi clamped
 *       to [0, 1]: the conservative phase field overshoots 1 by ~1e-3 inside
 *       a bubble, and at the paper's density ratio of 1000 an overshoot of
 *       1e-3 already makes rho <= 0 (the step then diverges within tens of
 *       steps).  phi itself, and every other use of it, stays unclamped.
 *   R13 surfactant held at psi_L (y = 0 end) and psi_R (y = ny-1 end), the
 *       paper's setting of its main cases (Sec. 2, Sec. 6): q takes the
 *       anti-bounce-back Dirichlet rule of h with psi_w, and psi's stencil
 *       ghosts are odd about psi_w, as T's about T_w (psi_bc = 1).  The
 *       alternative at the end of Sec. 6 keeps zero-flux walls and uses
 *       psi_L, psi_R only for the initial linear profile (psi_bc = 2), which
 *       the input generators build.
 *   R11 L in U_o (Eq. (21)) is the lattice length ny along the temperature
 *       gradient.
 *   R12 n = grad phi / max(|grad phi|, 1e-4): the paper leaves n undefined
 *       where grad phi vanishes (the centre of a bubble, where the direction
 *       of grad phi is arbitrary while theta = 4 phi (1 - phi)/W can still be
 *       ~1e-2 after internal mixing).  The floor keeps the sharpening flux
 *       M theta n continuous there.  It only acts where phi (1 - phi) is
 *       below ~W 1e-4 / 4 on the equilibrium profile; a larger floor would
 *       make the interface tails diffuse into the bulk (1e-2 fills the bulk
 *       to phi ~ 4e-3 and slowly dissolves bubbles), a smaller one leaves
 *       the bubble centre steered by rounding-level gradients.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- lattice */

/* D2Q9 velocities (App. B).  The printed e_x lists 0 at alpha = 8; the second
 * row of P (Eq. (45)) and the symmetry of the set give e_8 = (1, -1). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* Exponents (m, n) of the moment ordering of Eq. (25):
 * 00, 10, 01, 20, 02, 11, 21, 12, 22. */
static const int MX[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int MY[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
/* Standard D2Q9 weights; a test checks that they are the rest-state
 * equilibrium populations of the energy scheme (App. D) for T = 1. */
static const double WGT[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double CS2 = 1.0 / 3.0; /* c_s^2 (App. B-E) */

static double g_P[81], g_Pinv[81];
static int g_tables_ready = 0;

static double ipow(double b, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

static double binom(int n, int k)
{
    static const double c[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    return c[n][k];
}

/* P (Eq. (23), Eq. (45)): row i holds e_x^m e_y^n of moment i. */
static void build_P(double* P)
{
    for (int i = 0; i < 9; ++i)
        for (int a = 0; a < 9; ++a)
            P[i * 9 + a] = ipow(EX[a], MX[i]) * ipow(EY[a], MY[i]);
}

/* Inverse of a 9x9 matrix by Gauss-Jordan elimination with partial pivoting. */
static int invert9(const double* A, double* Ainv)
{
    double m[9][18];
    for (int i = 0; i < 9; ++i) {
        for (int j = 0; j < 9; ++j) {
            m[i][j] = A[i * 9 + j];
            m[i][9 + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(m[r][c]) > fabs(m[piv][c])) piv = r;
        if (fabs(m[piv][c]) < 1e-300) return -1;
        if (piv != c)
            for (int j = 0; j < 18; ++j) {
                double t = m[c][j];
                m[c][j] = m[piv][j];
                m[piv][j] = t;
            }
        double d = m[c][c];
        for (int j = 0; j < 18; ++j) m[c][j] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == c) continue;
            double fct = m[r][c];
            if (fct != 0.0)
                for (int j = 0; j < 18; ++j) m[r][j] -= fct * m[c][j];
        }
    }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) Ainv[i * 9 + j] = m[i][9 + j];
    return 0;
}

static void ensure_tables(void)
{
    if (g_tables_ready) return;
    build_P(g_P);
    invert9(g_P, g_Pinv);
    g_tables_ready = 1;
}

void orc_matrix_P(double* P81)
{
    ensure_tables();
    memcpy(P81, g_P, sizeof g_P);
}

void orc_matrix_Pinv(double* Pinv81)
{
    ensure_tables();
    memcpy(Pinv81, g_Pinv, sizeof g_Pinv);
}

/* Frame change F(u) of Eq. (24b)/(46), built from its definition: the central
 * moment (m, n) is sum_{a<=m, b<=n} C(m,a) C(n,b) (-u_x)^(m-a) (-u_y)^(n-b)
 * times the raw moment (a, b) (reading R1).  F^-1 = F(-u) (App. F). */
void orc_matrix_F(double ux, double uy, double* F)
{
    for (int i = 0; i < 9; ++i) {
        for (int j = 0; j < 9; ++j) {
            int m = MX[i], n = MY[i], a = MX[j], b = MY[j];
            double v = 0.0;
            if (a <= m && b <= n)
                v = binom(m, a) * binom(n, b) * ipow(-ux, m - a) * ipow(-uy, n - b);
            F[i * 9 + j] = v;
        }
    }
}

void orc_weights(double* w9) { memcpy(w9, WGT, sizeof WGT); }

void orc_velocities(int* ex9, int* ey9)
{
    memcpy(ex9, EX, sizeof EX);
    memcpy(ey9, EY, sizeof EY);
}

static void matvec9(const double* M, const double* x, double* y)
{
    for (int i = 0; i < 9; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 9; ++j) acc += M[i * 9 + j] * x[j];
        y[i] = acc;
    }
}

/* One central-moment collision (App. B-E): k' = P pop (Eq. (24a)),
 * k = F(u) k' (Eq. (24b)), relaxation with source (Eq. (33); Eqs. (27), (38),
 * (43) are the src = 0 case), optional trace/deviator split of the second
 * order diagonal pair (App. C), then k~' = F(-u) k~ and pop~ = P^-1 k~'. */
void orc_cm_collide(const double* pop, double ux, double uy, const double* eq,
                    const double* om, const double* src, int split,
                    double om2s, double om2d, double* out)
{
    double F[81], Fi[81], raw[9], k[9], kt[9], rawt[9];
    ensure_tables();
    orc_matrix_F(ux, uy, F);
    orc_matrix_F(-ux, -uy, Fi);
    matvec9(g_P, pop, raw);
    matvec9(F, raw, k);
    for (int i = 0; i < 9; ++i) {
        double s = src ? src[i] : 0.0;
        kt[i] = k[i] + om[i] * (eq[i] - k[i]) + (1.0 - 0.5 * om[i]) * s;
    }
    if (split) {
        double s20 = src ? src[3] : 0.0, s02 = src ? src[4] : 0.0;
        double k2s = k[3] + k[4], k2d = k[3] - k[4];
        double e2s = eq[3] + eq[4], e2d = eq[3] - eq[4];
        double s2s = s20 + s02, s2d = s20 - s02;
        double t2s = k2s + om2s * (e2s - k2s) + (1.0 - 0.5 * om2s) * s2s;
        double t2d = k2d + om2d * (e2d - k2d) + (1.0 - 0.5 * om2d) * s2d;
        kt[3] = 0.5 * (t2s + t2d);
        kt[4] = 0.5 * (t2s - t2d);
    }
    matvec9(Fi, kt, rawt);
    matvec9(g_Pinv, rawt, out);
}

/* ------------------------------------------------------------ parameters */

/* Surface tension equation of state, Eq. (6): quadratic (self-rewetting) law
 * in T plus the Langmuir term in psi (reading R9 for the clamp). */
double orc_sigma_eos(const orc_params* p, double T, double psi)
{
    double pc = psi;
    if (pc < 0.0) pc = 0.0;
    if (pc > 1.0 - 1e-6) pc = 1.0 - 1e-6;
    double dT = T - p->T_ref;
    return p->sigma0 + p->sigma0 * p->beta * (T / p->T_ref) * log(1.0 - pc) +
           p->sigma_T * dT + p->sigma_TT * dT * dT;
}

/* Bracket of Eq. (5): G(phi) = -(s/2) (4/(phi_o^2 W^2)) (phi_o^2 - (phi -
 * phi_m)^2)^2 + (w/2) (phi - phi_m)^2, phi_m = 1/2, phi_o = -1/2
 * (phi_A = 0, phi_B = 1, Sec. 3). */
double orc_G(const orc_derived* d, double W, double phi)
{
    const double phim = 0.5, phio = -0.5;
    double a = phio * phio - (phi - phim) * (phi - phim);
    return -0.5 * d->s * (4.0 / (phio * phio * W * W)) * a * a +
           0.5 * d->w * (phi - phim) * (phi - phim);
}

/* dG/dphi of the same bracket (reading R8: R = G'(phi) grad phi). */
double orc_dG(const orc_derived* d, double W, double phi)
{
    const double phim = 0.5, phio = -0.5;
    double a = phio * phio - (phi - phim) * (phi - phim);
    return -0.5 * d->s * (4.0 / (phio * phio * W * W)) * 2.0 * a *
               (-2.0 * (phi - phim)) +
           d->w * (phi - phim);
}

/* Step P: lattice parameters from the paper's groups.
 * M1, M2 from Eq. (10); U_o from Eq. (21) with mu_A = rho_A nu_A and
 * nu_A = U_o R / Re (Eq. (8)), i.e. U_o^2 = sigma0 Re |M1 + M2| / (rho_A L);
 * alpha_A = U_o R / Ma (Eq. (8)); ratios from Eq. (9) and Sec. 6;
 * relaxation rates from M = c_s^2 (1/omega - 1/2) (App. B, E);
 * lambda from Pi = lambda W^2 / (8 sigma0), s and w by reading R7. */
int orc_derive(const orc_params* p, orc_derived* d)
{
    memset(d, 0, sizeof *d);
    if (p->nx < 4 || p->ny < (p->walls ? 5 : 4)) return -1;
    if (p->psi_bc < 0 || p->psi_bc > 2 || !(p->psi_L >= 0.0 && p->psi_L < 1.0) ||
        !(p->psi_R >= 0.0 && p->psi_R < 1.0))
        return -1;
    if (!(p->rho_A > 0) || !(p->rho_ratio > 0) || !(p->mu_ratio > 0) ||
        !(p->alpha_ratio > 0) || !(p->W > 0) || !(p->T_ref != 0))
        return -1;
    d->dT = p->T_H - p->T_C;
    d->M1 = (p->sigma0 != 0.0) ? d->dT * p->sigma_T / p->sigma0 : 0.0;
    d->M2 = (p->sigma0 != 0.0) ? d->dT * d->dT * p->sigma_TT / p->sigma0 : 0.0;
    d->L = (double)p->ny;
    d->rho_A = p->rho_A;
    d->rho_B = p->rho_A / p->rho_ratio;
    double mm = fabs(d->M1 + d->M2);
    if (p->nu_A > 0) {
        d->nu_A = p->nu_A;
        d->U_o = (p->sigma0 / (p->rho_A * d->nu_A)) * (p->R / d->L) * mm;
    } else {
        if (!(mm > 0) || !(p->Re > 0) || !(p->R > 0) || !(p->sigma0 > 0)) return -1;
        d->U_o = sqrt(p->sigma0 * p->Re * mm / (p->rho_A * d->L));
        d->nu_A = d->U_o * p->R / p->Re;
    }
    if (p->alpha_A > 0) {
        d->alpha_A = p->alpha_A;
    } else {
        if (!(d->U_o > 0) || !(p->Ma > 0)) return -1;
        d->alpha_A = d->U_o * p->R / p->Ma;
    }
    d->mu_A = d->rho_A * d->nu_A;
    d->mu_B = d->mu_A / p->mu_ratio;
    d->nu_B = d->mu_B / d->rho_B;
    d->alpha_B = d->alpha_A / p->alpha_ratio;
    d->omega_phi = 1.0 / (p->M_phi / CS2 + 0.5);
    d->D_psi = p->M_psi;
    d->omega_psi = 1.0 / (p->M_psi / CS2 + 0.5);
    d->lambda = (p->Pi > 0) ? 8.0 * p->sigma0 * p->Pi / (p->W * p->W) : 0.0;
    d->s = (p->Pi > 0) ? 8.0 * p->sigma0 : 0.0;
    d->w = (p->Pi > 0 && p->Ex > 0) ? 4.0 * d->s / (p->Ex * p->W * p->W) : 0.0;
    d->m_psi = (d->lambda > 0) ? d->D_psi / d->lambda : 0.0;
    /* every relaxation rate must lie in (0, 2) */
    double rates[6] = {d->omega_phi, d->omega_psi, 1.0 / (d->nu_A / CS2 + 0.5),
                       1.0 / (d->nu_B / CS2 + 0.5), 1.0 / (d->alpha_A / CS2 + 0.5),
                       1.0 / (d->alpha_B / CS2 + 0.5)};
    for (int i = 0; i < 6; ++i)
        if (!(rates[i] > 0.0 && rates[i] < 2.0)) return -2;
    return 0;
}

/* ------------------------------------------------------------ simulation */

enum { NSET = 4 };

struct orc_sim {
    orc_params p;
    orc_derived d;
    int nx, ny;
    int64_t t;
    double* pop[NSET];  /* S_t: post-streaming populations [9][ny][nx] */
    double* post[NSET]; /* post-collision populations */
    /* macroscopic fields of the current time level, [ny][nx] */
    double *phi, *T, *psi, *pstar, *jx, *jy;
    double *ux, *uy, *p_corr, *Fpx, *Fpy, *Ftx, *Fty, *nxv, *nyv, *gpx, *gpy;
};

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int fluid_row(const orc_sim* s, int y)
{
    return s->p.walls ? (y >= 1 && y <= s->ny - 2) : (y >= 0 && y < s->ny);
}

static int wrapx(const orc_sim* s, int x) { return ((x % s->nx) + s->nx) % s->nx; }

/* Row holding the value seen at row y by a stencil (reading R10): periodic
 * wrap without walls; with walls, rows at and beyond a wall mirror about the
 * wall plane (y = 1/2 at the bottom, y = ny - 3/2 at the top).  *side is -1
 * for a bottom image, +1 for a top image, 0 for a fluid row. */
static int src_row(const orc_sim* s, int y, int* side)
{
    *side = 0;
    if (!s->p.walls) return ((y % s->ny) + s->ny) % s->ny;
    if (y < 1) {
        *side = -1;
        return 1 - y;
    }
    if (y > s->ny - 2) {
        *side = +1;
        return 2 * s->ny - 3 - y;
    }
    return y;
}

static double even_at(const orc_sim* s, const double* a, int x, int y)
{
    int side;
    int r = src_row(s, y, &side);
    return a[(size_t)r * s->nx + wrapx(s, x)];
}

static double T_at(const orc_sim* s, int x, int y)
{
    int side;
    int r = src_row(s, y, &side);
    double v = s->T[(size_t)r * s->nx + wrapx(s, x)];
    if (side < 0) return 2.0 * s->p.T_H - v;
    if (side > 0) return 2.0 * s->p.T_C - v;
    return v;
}

/* psi at (x, y) with the wall ghosts of R10 / R13. */
static double psi_at(const orc_sim* s, int x, int y)
{
    int side;
    int r = src_row(s, y, &side);
    double v = s->psi[(size_t)r * s->nx + wrapx(s, x)];
    if (s->p.psi_bc == 1 && side < 0) return 2.0 * s->p.psi_L - v;
    if (s->p.psi_bc == 1 && side > 0) return 2.0 * s->p.psi_R - v;
    return v;
}

/* phi for the property interpolation (R14): clamped to [0, 1]. */
static double phi_prop(double phi)
{
    return phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
}

static double rho_of(const orc_sim* s, double phi)
{
    return s->d.rho_A + phi_prop(phi) * (s->d.rho_B - s->d.rho_A); /* Eq. (17), R2, R14 */
}

static double mu_of(const orc_sim* s, double phi)
{
    return s->d.mu_A + phi_prop(phi) * (s->d.mu_B - s->d.mu_A); /* Eq. (17), R2, R14 */
}

static double alpha_of(const orc_sim* s, double phi)
{
    return s->d.alpha_A + phi_prop(phi) * (s->d.alpha_B - s->d.alpha_A);
}

static double sigma_at(const orc_sim* s, int x, int y)
{
    return orc_sigma_eos(&s->p, T_at(s, x, y), psi_at(s, x, y));
}

static double phistar_at(const orc_sim* s, int x, int y)
{
    double ph = even_at(s, s->phi, x, y);
    return even_at(s, s->pstar, x, y) - rho_of(s, ph) * CS2;
}

/* Isotropic gradient (reading R6): grad X = 3 sum_a w_a e_a X(x + e_a). */
typedef double (*field_fn)(const orc_sim*, const void*, int, int);

static double fn_phi(const orc_sim* s, const void* u, int x, int y)
{
    (void)u;
    return even_at(s, s->phi, x, y);
}
static double fn_sigma(const orc_sim* s, const void* u, int x, int y)
{
    (void)u;
    return sigma_at(s, x, y);
}
static double fn_phistar(const orc_sim* s, const void* u, int x, int y)
{
    (void)u;
    return phistar_at(s, x, y);
}

static void grad_at(const orc_sim* s, field_fn fn, const void* u, int x, int y,
                    double* gx, double* gy)
{
    double ax = 0.0, ay = 0.0;
    for (int a = 1; a < 9; ++a) {
        double v = fn(s, u, x + EX[a], y + EY[a]);
        ax += WGT[a] * EX[a] * v;
        ay += WGT[a] * EY[a] * v;
    }
    *gx = ax / CS2;
    *gy = ay / CS2;
}

/* Unit normal n = grad phi / |grad phi| (Sec. 3), regularised where the
 * gradient is small (reading R12): n = grad phi / max(|grad phi|, 1e-4). */
#define ORC_NORMAL_EPS 1e-4
static void normal_at(const orc_sim* s, int x, int y, double* nx, double* ny)
{
    double gx, gy;
    grad_at(s, fn_phi, NULL, x, y, &gx, &gy);
    double g = sqrt(gx * gx + gy * gy);
    if (g < ORC_NORMAL_EPS) g = ORC_NORMAL_EPS;
    *nx = gx / g;
    *ny = gy / g;
}

static double* alloc_d(size_t n)
{
    return (double*)calloc(n, sizeof(double));
}

int orc_create(const orc_params* p, orc_sim** out)
{
    *out = NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof *s);
    if (!s) return -3;
    s->p = *p;
    int rc = orc_derive(p, &s->d);
    if (rc) {
        free(s);
        return rc;
    }
    ensure_tables();
    s->nx = p->nx;
    s->ny = p->ny;
    size_t N = (size_t)s->nx * s->ny;
    for (int k = 0; k < NSET; ++k) {
        s->pop[k] = alloc_d(9 * N);
        s->post[k] = alloc_d(9 * N);
    }
    double** fields[] = {&s->phi, &s->T,   &s->psi, &s->pstar, &s->jx,  &s->jy,
                         &s->ux,  &s->uy,  &s->p_corr, &s->Fpx, &s->Fpy, &s->Ftx,
                         &s->Fty, &s->nxv, &s->nyv, &s->gpx,   &s->gpy};
    for (size_t i = 0; i < sizeof fields / sizeof fields[0]; ++i) *fields[i] = alloc_d(N);
    *out = s;
    return 0;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    for (int k = 0; k < NSET; ++k) {
        free(s->pop[k]);
        free(s->post[k]);
    }
    double* fields[] = {s->phi, s->T,   s->psi, s->pstar, s->jx,  s->jy,
                        s->ux,  s->uy,  s->p_corr, s->Fpx, s->Fpy, s->Ftx,
                        s->Fty, s->nxv, s->nyv, s->gpx,   s->gpy};
    for (size_t i = 0; i < sizeof fields / sizeof fields[0]; ++i) free(fields[i]);
    free(s);
}

int64_t orc_time(const orc_sim* s) { return s->t; }

#define POP(s, k, a, idx) ((s)->pop[k][(size_t)(a) * (size_t)(s)->nx * (s)->ny + (idx)])
#define POST(s, k, a, idx) ((s)->post[k][(size_t)(a) * (size_t)(s)->nx * (s)->ny + (idx)])

/* Zeroth and first moments of the current populations: phi (Eq. (28)),
 * T (Eq. (39)), psi (Eq. (44)), p* = sum g and j = sum g e (Eq. (34)). */
static void moments(orc_sim* s)
{
    const int nx = s->nx, ny = s->ny;
#pragma omp parallel for schedule(static) if ((long)nx * ny >= 2048)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            if (!fluid_row(s, y)) {
                s->phi[i] = s->T[i] = s->psi[i] = s->pstar[i] = s->jx[i] = s->jy[i] = 0.0;
                continue;
            }
            double ph = 0, T = 0, ps = 0, pg = 0, jx = 0, jy = 0;
            for (int a = 0; a < 9; ++a) {
                ph += POP(s, 0, a, i);
                pg += POP(s, 1, a, i);
                T += POP(s, 2, a, i);
                ps += POP(s, 3, a, i);
                jx += POP(s, 1, a, i) * EX[a];
                jy += POP(s, 1, a, i) * EY[a];
            }
            s->phi[i] = ph;
            s->T[i] = T;
            s->psi[i] = ps;
            s->pstar[i] = pg;
            s->jx[i] = jx;
            s->jy[i] = jy;
        }
    }
}

/* Forces, velocity and corrected pressure at every fluid node:
 *   kappa = div n (R6), F_s = 1.5 W |grad phi|^2 [-sigma kappa n
 *   + (I - n n) grad sigma] (Eqs. (15)-(16), R4), F_t = F_s + F_ext
 *   + buoyancy (Sec. 5.3), F_p = -grad(p* - rho c_s^2) (App. C, R5),
 *   rho c_s^2 u = sum g e + c_s^2 F_t / 2 and p = p* + F_p . u / 2
 *   (Eq. (34)). */
static void forces_velocity(orc_sim* s)
{
    const int nx = s->nx, ny = s->ny;
    const double W = s->p.W;
#pragma omp parallel for schedule(static) if ((long)nx * ny >= 2048)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            if (!fluid_row(s, y)) continue;
            double gx, gy;
            grad_at(s, fn_phi, NULL, x, y, &gx, &gy);
            double g2 = gx * gx + gy * gy;
            double n_x, n_y;
            normal_at(s, x, y, &n_x, &n_y);
            /* kappa = d(n_x)/dx + d(n_y)/dy with the isotropic stencil */
            double kap = 0.0;
            for (int a = 1; a < 9; ++a) {
                double mx, my;
                normal_at(s, x + EX[a], y + EY[a], &mx, &my);
                kap += WGT[a] * (EX[a] * mx + EY[a] * my);
            }
            kap /= CS2;
            double sgx, sgy;
            grad_at(s, fn_sigma, NULL, x, y, &sgx, &sgy);
            double sig = sigma_at(s, x, y);
            double ndots = n_x * sgx + n_y * sgy;
            double deltas = 1.5 * W * g2;
            double Fsx = deltas * (-sig * kap * n_x + sgx - n_x * ndots);
            double Fsy = deltas * (-sig * kap * n_y + sgy - n_y * ndots);
            double rho = rho_of(s, s->phi[i]);
            double Ftx = Fsx + s->p.Fext_x;
            double Fty = Fsy + s->p.Fext_y - (rho - s->d.rho_A) * s->p.gravity;
            double pgx, pgy;
            grad_at(s, fn_phistar, NULL, x, y, &pgx, &pgy);
            double Fpx = -pgx, Fpy = -pgy;
            double ux = s->jx[i] / (rho * CS2) + 0.5 * Ftx / rho;
            double uy = s->jy[i] / (rho * CS2) + 0.5 * Fty / rho;
            s->ux[i] = ux;
            s->uy[i] = uy;
            s->p_corr[i] = s->pstar[i] + 0.5 * (Fpx * ux + Fpy * uy);
            s->Fpx[i] = Fpx;
            s->Fpy[i] = Fpy;
            s->Ftx[i] = Ftx;
            s->Fty[i] = Fty;
            s->nxv[i] = n_x;
            s->nyv[i] = n_y;
            s->gpx[i] = gx;
            s->gpy[i] = gy;
        }
    }
}

/* Central-moment equilibria:
 *   f: (phi, M theta n_x, M theta n_y, phi/3, phi/3, 0, 0, 0, phi/9)
 *      (Eq. (26), theta by R3);
 *   g: Eq. (31) with varphi = p - rho c_s^2;
 *   h: (T, 0, 0, T/3, T/3, 0, 0, 0, T/9) (Eq. (37));
 *   q: (psi, -m psi(1-psi) R_x, -m psi(1-psi) R_y, psi/3, psi/3, 0, 0, 0,
 *      psi/9) (Eq. (42), R7, R8, R9). */
static void eq_f(const orc_sim* s, double phi, double n_x, double n_y, double* e)
{
    double theta = 4.0 * phi * (1.0 - phi) / s->p.W;
    e[0] = phi;
    e[1] = s->p.M_phi * theta * n_x;
    e[2] = s->p.M_phi * theta * n_y;
    e[3] = CS2 * phi;
    e[4] = CS2 * phi;
    e[5] = e[6] = e[7] = 0.0;
    e[8] = CS2 * CS2 * phi;
}

static void eq_g(double p, double rho, double ux, double uy, double* e)
{
    double vp = p - rho * CS2;
    e[0] = p;
    e[1] = -vp * ux;
    e[2] = -vp * uy;
    e[3] = p * CS2 + vp * ux * ux;
    e[4] = p * CS2 + vp * uy * uy;
    e[5] = vp * ux * uy;
    e[6] = -vp * (ux * ux + CS2) * uy;
    e[7] = -vp * (uy * uy + CS2) * ux;
    e[8] = CS2 * CS2 * CS2 * rho + vp * (ux * ux + CS2) * (uy * uy + CS2);
}

/* Source central moments of App. C, Eq. (32). */
static void src_g(double Ftx, double Fty, double Fpx, double Fpy, double ux,
                  double uy, double* sg)
{
    double G = Fpx * ux + Fpy * uy;
    sg[0] = G;
    sg[1] = CS2 * Ftx - ux * G;
    sg[2] = CS2 * Fty - uy * G;
    sg[3] = 2.0 * CS2 * Fpx * ux + (ux * ux + CS2) * G;
    sg[4] = 2.0 * CS2 * Fpy * uy + (uy * uy + CS2) * G;
    sg[5] = CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;
    sg[6] = sg[7] = sg[8] = 0.0;
}

static void eq_scalar(double v, double* e)
{
    e[0] = v;
    e[1] = e[2] = 0.0;
    e[3] = e[4] = CS2 * v;
    e[5] = e[6] = e[7] = 0.0;
    e[8] = CS2 * CS2 * v;
}

static void eq_q(const orc_sim* s, double psi, double Rx, double Ry, double* e)
{
    eq_scalar(psi, e);
    e[1] = -s->d.m_psi * psi * (1.0 - psi) * Rx;
    e[2] = -s->d.m_psi * psi * (1.0 - psi) * Ry;
}

/* Collision of the four distributions at every fluid node into post[]. */
static void collide(orc_sim* s)
{
    const int nx = s->nx, ny = s->ny;
    const double one[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
#pragma omp parallel for schedule(static) if ((long)nx * ny >= 2048)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            if (!fluid_row(s, y)) continue;
            double ux = s->ux[i], uy = s->uy[i];
            double phi = s->phi[i], T = s->T[i], psi = s->psi[i];
            double rho = rho_of(s, phi);
            double in[9], out[9], eq[9], om[9], src[9];

            /* f: phase field, App. B */
            for (int a = 0; a < 9; ++a) in[a] = POP(s, 0, a, i);
            eq_f(s, phi, s->nxv[i], s->nyv[i], eq);
            memcpy(om, one, sizeof om);
            om[1] = om[2] = s->d.omega_phi;
            orc_cm_collide(in, ux, uy, eq, om, NULL, 0, 1.0, 1.0, out);
            for (int a = 0; a < 9; ++a) POST(s, 0, a, i) = out[a];

            /* g: two-fluid flow, App. C; omega_2d = omega_11 from the local
             * kinematic viscosity nu = mu / rho, every other rate 1 */
            for (int a = 0; a < 9; ++a) in[a] = POP(s, 1, a, i);
            eq_g(s->p_corr[i], rho, ux, uy, eq);
            src_g(s->Ftx[i], s->Fty[i], s->Fpx[i], s->Fpy[i], ux, uy, src);
            double nu = mu_of(s, phi) / rho;
            double omn = 1.0 / (nu / CS2 + 0.5);
            memcpy(om, one, sizeof om);
            om[5] = omn;
            orc_cm_collide(in, ux, uy, eq, om, src, 1, 1.0, omn, out);
            for (int a = 0; a < 9; ++a) POST(s, 1, a, i) = out[a];

            /* h: energy, App. D, first-order rate from the local alpha */
            for (int a = 0; a < 9; ++a) in[a] = POP(s, 2, a, i);
            eq_scalar(T, eq);
            memcpy(om, one, sizeof om);
            om[1] = om[2] = 1.0 / (alpha_of(s, phi) / CS2 + 0.5);
            orc_cm_collide(in, ux, uy, eq, om, NULL, 0, 1.0, 1.0, out);
            for (int a = 0; a < 9; ++a) POST(s, 2, a, i) = out[a];

            /* q: surfactant, App. E */
            for (int a = 0; a < 9; ++a) in[a] = POP(s, 3, a, i);
            double dG = orc_dG(&s->d, s->p.W, phi);
            eq_q(s, psi, dG * s->gpx[i], dG * s->gpy[i], eq);
            memcpy(om, one, sizeof om);
            om[1] = om[2] = s->d.omega_psi;
            orc_cm_collide(in, ux, uy, eq, om, NULL, 0, 1.0, 1.0, out);
            for (int a = 0; a < 9; ++a) POST(s, 3, a, i) = out[a];
        }
    }
}

/* Streaming f_a(x, t+1) = f~_a(x - e_a) (Eqs. in App. B-E), periodic in x
 * (and in y without walls); a population whose source is a wall node is the
 * one that left this node towards the wall, reversed (halfway bounce-back,
 * R10), for h with the anti-bounce-back Dirichlet term 2 w_a T_w, and for q
 * with 2 w_a psi_w when psi is held at the walls (R13). */
static void stream(orc_sim* s)
{
    const int nx = s->nx, ny = s->ny;
#pragma omp parallel for schedule(static) if ((long)nx * ny >= 2048)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            if (!fluid_row(s, y)) continue;
            for (int a = 0; a < 9; ++a) {
                int sy = y - EY[a];
                int sx = wrapx(s, x - EX[a]);
                if (!s->p.walls) sy = ((sy % ny) + ny) % ny;
                if (fluid_row(s, sy)) {
                    size_t j = (size_t)sy * nx + sx;
                    for (int k = 0; k < NSET; ++k) POP(s, k, a, i) = POST(s, k, a, j);
                } else {
                    double Tw = (sy <= 0) ? s->p.T_H : s->p.T_C;
                    POP(s, 0, a, i) = POST(s, 0, OPP[a], i);
                    POP(s, 1, a, i) = POST(s, 1, OPP[a], i);
                    POP(s, 2, a, i) = -POST(s, 2, OPP[a], i) + 2.0 * WGT[a] * Tw;
                    if (s->p.psi_bc == 1) {
                        double psiw = (sy <= 0) ? s->p.psi_L : s->p.psi_R;
                        POP(s, 3, a, i) = -POST(s, 3, OPP[a], i) + 2.0 * WGT[a] * psiw;
                    } else {
                        POP(s, 3, a, i) = POST(s, 3, OPP[a], i);
                    }
                }
            }
        }
    }
}

static void macroscopic(orc_sim* s)
{
    moments(s);
    forces_velocity(s);
}

int orc_step(orc_sim* s, int64_t nsteps)
{
    if (nsteps < 0) return -1;
    for (int64_t k = 0; k < nsteps; ++k) {
        macroscopic(s);
        collide(s);
        stream(s);
        s->t += 1;
    }
    return 0;
}

/* Populations at their equilibria (P^-1 F(-u) applied to the equilibrium
 * central moments) for given phi, u, p, T, psi; n and R from the stencils
 * of the given phi. */
int orc_init_fields(orc_sim* s, const double* fields)
{
    const int nx = s->nx, ny = s->ny;
    const size_t N = (size_t)nx * ny;
    const double *fphi = fields, *fux = fields + N, *fuy = fields + 2 * N,
                 *fp = fields + 3 * N, *fT = fields + 4 * N, *fpsi = fields + 5 * N;
    for (size_t i = 0; i < N; ++i) {
        int y = (int)(i / nx);
        int fl = fluid_row(s, y);
        s->phi[i] = fl ? fphi[i] : 0.0;
        s->T[i] = fl ? fT[i] : 0.0;
        s->psi[i] = fl ? fpsi[i] : 0.0;
    }
    const double zero[9] = {0}, one[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    for (int k = 0; k < NSET; ++k) memset(s->pop[k], 0, 9 * N * sizeof(double));
#pragma omp parallel for schedule(static) if ((long)nx * ny >= 2048)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            if (!fluid_row(s, y)) continue;
            double ux = fux[i], uy = fuy[i];
            double phi = s->phi[i];
            double n_x, n_y, gx, gy, eq[9], out[9];
            normal_at(s, x, y, &n_x, &n_y);
            grad_at(s, fn_phi, NULL, x, y, &gx, &gy);
            /* collision with every rate 1 and no source returns P^-1 F(-u) eq */
            eq_f(s, phi, n_x, n_y, eq);
            orc_cm_collide(zero, ux, uy, eq, one, NULL, 0, 1.0, 1.0, out);
            for (int a = 0; a < 9; ++a) POP(s, 0, a, i) = out[a];
            eq_g(fp[i], rho_of(s, phi), ux, uy, eq);
            orc_cm_collide(zero, ux, uy, eq, one, NULL, 0, 1.0, 1.0, out);
            for (int a = 0; a < 9; ++a) POP(s, 1, a, i) = out[a];
            eq_scalar(s->T[i], eq);
            orc_cm_collide(zero, ux, uy, eq, one, NULL, 0, 1.0, 1.0, out);
            for (int a = 0; a < 9; ++a) POP(s, 2, a, i) = out[a];
            double dG = orc_dG(&s->d, s->p.W, phi);
            eq_q(s, s->psi[i], dG * gx, dG * gy, eq);
            orc_cm_collide(zero, ux, uy, eq, one, NULL, 0, 1.0, 1.0, out);
            for (int a = 0; a < 9; ++a) POP(s, 3, a, i) = out[a];
        }
    }
    s->t = 0;
    return 0;
}

int orc_set_populations(orc_sim* s, const double* pops)
{
    size_t n = 9 * (size_t)s->nx * s->ny;
    for (int k = 0; k < NSET; ++k) memcpy(s->pop[k], pops + k * n, n * sizeof(double));
    return 0;
}

int orc_get_populations(const orc_sim* s, double* pops)
{
    size_t n = 9 * (size_t)s->nx * s->ny;
    for (int k = 0; k < NSET; ++k) memcpy(pops + k * n, s->pop[k], n * sizeof(double));
    return 0;
}

int orc_fields(orc_sim* s, double* fields)
{
    const size_t N = (size_t)s->nx * s->ny;
    macroscopic(s);
    for (size_t i = 0; i < N; ++i) {
        int fl = fluid_row(s, (int)(i / s->nx));
        fields[i] = fl ? s->phi[i] : 0.0;
        fields[N + i] = fl ? s->ux[i] : 0.0;
        fields[2 * N + i] = fl ? s->uy[i] : 0.0;
        fields[3 * N + i] = fl ? s->p_corr[i] : 0.0;
        fields[4 * N + i] = fl ? s->T[i] : 0.0;
        fields[5 * N + i] = fl ? s->psi[i] : 0.0;
    }
    return 0;
}

/* Observables of Sec. 5.3 and Sec. 6: phase-field and surfactant masses, the
 * bubble centroid ("mass center") and the migration velocity ("average
 * velocity inside the bubble"), both weighted by phi (phi = 1 in the bubble);
 * t* = t U_o / R. */
int orc_observe(orc_sim* s, double* out)
{
    macroscopic(s);
    double m = 0, mpsi = 0, sx = 0, sy = 0, su = 0, sv = 0;
    for (int y = 0; y < s->ny; ++y) {
        if (!fluid_row(s, y)) continue;
        for (int x = 0; x < s->nx; ++x) {
            size_t i = (size_t)y * s->nx + x;
            double ph = s->phi[i];
            m += ph;
            mpsi += s->psi[i];
            sx += ph * x;
            sy += ph * y;
            su += ph * s->ux[i];
            sv += ph * s->uy[i];
        }
    }
    out[0] = (double)s->t;
    out[1] = m;
    out[2] = mpsi;
    out[3] = m != 0 ? sx / m : 0.0;
    out[4] = m != 0 ? sy / m : 0.0;
    out[5] = m != 0 ? su / m : 0.0;
    out[6] = m != 0 ? sv / m : 0.0;
    out[7] = s->d.U_o;
    out[8] = (s->p.R > 0) ? s->t * s->d.U_o / s->p.R : 0.0;
    return 0;
}

/* Isotropic gradient on a fully periodic nx*ny array (used by the stencil
 * tests). */
int orc_gradient_periodic(int nx, int ny, const double* a, double* gx, double* gy)
{
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double ax = 0.0, ay = 0.0;
            for (int k = 1; k < 9; ++k) {
                int xx = ((x + EX[k]) % nx + nx) % nx;
                int yy = ((y + EY[k]) % ny + ny) % ny;
                double v = a[(size_t)yy * nx + xx];
                ax += WGT[k] * EX[k] * v;
                ay += WGT[k] * EY[k] * v;
            }
            gx[(size_t)y * nx + x] = ax / CS2;
            gy[(size_t)y * nx + x] = ay / CS2;
        }
    }
    return 0;
}
