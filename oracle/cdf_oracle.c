/*
 * cdf_oracle.c -- CPU FP64 oracle of the lattice Boltzmann model for the coupled
 * cross-diffusion-fluid (CDF) system of Zhan, Chai & Shi (arXiv:2101.03055).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or helper with the CUDA library; both receive the same seeded
 * inputs (initial moments and parameters) and nothing else.
 *
 * It is written to be checked against the paper by eye: FP64 throughout,
 * array-of-structures storage, one node at a time, and the paper's order of
 * operations for every time step t -> t+1:
 *
 *   1. moments of the pre-collision populations           (Eq. sum-phi, sum-u, sum-p)
 *      and the model closures D(phi), S(phi), F(phi)        (Sec. 3.1 / 3.2 closures)
 *   2. relaxation factors: omega = (D/cs^2 + I/2)^-1      (Eq. omega-D, lambda = I, dt = 1)
 *                          omega_f = 1/(nu/cs^2 + 1/2)      (appendix, nu-omega relation)
 *   3. equilibria f^eq, h^eq                                (Eq. feq-phi, heq)
 *   4. collision with the matrix operator, the source, its
 *      time-derivative correction and the auxiliary source   (Eq. evolution12, source, Gi)
 *      and the fluid collision with the force term          (Eq. evolution3, force)
 *   5. streaming f(x + c_i, t+1) = f*(x, t), with the
 *      boundary rules applied to links that leave the box   (Sec. 3, boundary schemes)
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * design notes of the repository):
 *   - lambda = I and varphi = 0 as in the experiments (Sec. 3); vartheta is a
 *     parameter (default 0, i.e. linear f^eq; Case 2 of Sec. 2.1 lets it be arbitrary).
 *   - D(t) S is discretised by the backward difference of Sec. 2.1, i.e.
 *     + 1/2 (S_i(t) - S_i(t-1)) with gamma = 0.
 *   - Initial populations: f = f^eq(phi0, u0); h = h^eq(u0, p0) - F_i(phi0)/2,
 *     so that the moments at t = 0 reproduce (phi0, u0, p0) exactly; S(t-1) at
 *     t = 0 is S(phi0).
 *   - Half-way walls.  Bounce-back: f_opp(i)(x, t+1) = f*_i(x, t).
 *     Anti-bounce-back (Dirichlet phi_w, wall at rest):
 *       f_opp(i)(x, t+1) = -f*_i(x, t) + 2 W_i phi_w.
 *     Free slip: specular reflection of the normal velocity component; a
 *     diagonal link leaving through a corner is bounced back.
 *   - Chemotaxis closure (Sec. 3.1): D_01 += -chi phi_0 r(phi_1),
 *     consumption S_1 = -k phi_0 r(phi_1); r is the step cut-off
 *     (r = 1 for c >= c*) or its regularised form with width eps.
 *   - Force F = g (F0 + sum_a beta_a (phi_a - phi_ref_a)).
 *   - Case 1 of Sec. 2.1 (case1 = 1): the convection cross-diffusion equations
 *     alone, no fluid populations.  The velocity passed to orc_init is a steady
 *     prescribed field (p = 0, F = 0), and the auxiliary source is
 *       G_{i,a} = sum_b (delta_ab - omega_ab / 2) W_i c_i.d_t(phi_b u) / cs^2
 *     with the first-order explicit difference
 *       d_t(phi_b u) = u (phi_b(t) - phi_b(t - 1));
 *     phi(t - 1) at t = 0 is phi0, so the first step has G = 0.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_M 8

enum { ORC_WEST = 0, ORC_EAST = 1, ORC_SOUTH = 2, ORC_NORTH = 3 };
enum { ORC_PERIODIC = 0, ORC_WALL = 1 };
enum { ORC_NOSLIP = 0, ORC_FREESLIP = 1 };
enum { ORC_NOFLUX = 0, ORC_DIRICHLET = 1 };
enum { ORC_D_CONST = 0, ORC_D_CHEMOTAXIS = 1 };
enum { ORC_S_NONE = 0, ORC_S_CONST = 1, ORC_S_CONSUMPTION = 2 };

typedef struct {
    int nx, ny, m;
    int dkind;
    double D[ORC_MAX_M * ORC_MAX_M]; /* row-major m x m, lattice units */
    double chi, c_star, eps;
    int r_regularised;
    int skind;
    double S[ORC_MAX_M];
    double k;
    double g[2];
    double beta[ORC_MAX_M];
    double phi_ref[ORC_MAX_M];
    double F0;
    double nu, rho0, theta;
    int side_kind[4];
    int fluid_bc[4];
    int scalar_bc[4][ORC_MAX_M];
    double value[4][ORC_MAX_M];
    int case1;              /* Case 1 of Sec. 2.1: prescribed steady velocity, no fluid */
    double varphi;          /* the parameter of the second-order part of Eq. force (0 or 1) */
} orc_params;

/* ---- lattices (Eq. D2Q5 and Eq. D2Q9), c_hat = 1 ---------------------------- */
static const double CS2 = 1.0 / 3.0;
static const int Q5_CX[5] = {0, 1, 0, -1, 0};
static const int Q5_CY[5] = {0, 0, 1, 0, -1};
static const double Q5_W[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
static const int Q9_CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int Q9_CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double Q9_W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static int q5_dir(int cx, int cy) {
    for (int i = 0; i < 5; ++i)
        if (Q5_CX[i] == cx && Q5_CY[i] == cy) return i;
    return -1;
}
static int q9_dir(int cx, int cy) {
    for (int i = 0; i < 9; ++i)
        if (Q9_CX[i] == cx && Q9_CY[i] == cy) return i;
    return -1;
}

/* ---- single-node building blocks (exported for the moment-identity pins) ---- */

/* Eq. feq-phi with lambda = I:
 * f^eq_i = W_i [ phi + c_i.(phi u)/cs^2 + vartheta phi uu:(c_i c_i - cs^2 I)/(2 cs^4) ] */
void orc_feq_scalar(double phi, double ux, double uy, double theta, double out[5]) {
    for (int i = 0; i < 5; ++i) {
        double cu = Q5_CX[i] * ux + Q5_CY[i] * uy;
        double uu_cc = cu * cu - CS2 * (ux * ux + uy * uy); /* uu:(cc - cs^2 I) */
        out[i] = Q5_W[i] * (phi + cu * phi / CS2 + theta * phi * uu_cc / (2.0 * CS2 * CS2));
    }
}

/* Eq. heq: h^eq_i = sigma_i + W_i [ c_i.u/cs^2 + uu:(c_i c_i - cs^2 I)/(2 cs^4) ],
 * sigma_0 = (W_0 - 1) p / cs^2 + rho0, sigma_i = W_i p / cs^2 (i != 0). */
void orc_heq(double p, double ux, double uy, double rho0, double out[9]) {
    for (int i = 0; i < 9; ++i) {
        double cu = Q9_CX[i] * ux + Q9_CY[i] * uy;
        double uu_cc = cu * cu - CS2 * (ux * ux + uy * uy);
        double sigma = (i == 0) ? (Q9_W[0] - 1.0) * p / CS2 + rho0 : Q9_W[i] * p / CS2;
        out[i] = sigma + Q9_W[i] * (cu / CS2 + uu_cc / (2.0 * CS2 * CS2));
    }
}

/* Eq. force: F_i = W_i [ c_i.F / cs^2 + varphi (uF + Fu):(c_i c_i - cs^2 I) / (2 cs^4) ],
 * with (uF + Fu):(c_i c_i - cs^2 I) = 2 (c_i.u)(c_i.F) - 2 cs^2 u.F. */
void orc_force_pop_phi(double Fx, double Fy, double ux, double uy, double varphi, double out[9]) {
    for (int i = 0; i < 9; ++i) {
        double cF = Q9_CX[i] * Fx + Q9_CY[i] * Fy, cu = Q9_CX[i] * ux + Q9_CY[i] * uy;
        double uFFu_cc = 2.0 * cu * cF - 2.0 * CS2 * (ux * Fx + uy * Fy);
        out[i] = Q9_W[i] * (cF / CS2 + varphi * uFFu_cc / (2.0 * CS2 * CS2));
    }
}

/* Eq. force with varphi = 0: F_i = W_i c_i.F / cs^2 */
void orc_force_pop(double Fx, double Fy, double out[9]) { orc_force_pop_phi(Fx, Fy, 0.0, 0.0, 0.0, out); }

/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix.
 * Returns 0 on success, -1 if singular. */
static int gj_inverse(int n, const double *a_in, double *inv) {
    double a[ORC_MAX_M * ORC_MAX_M];
    memcpy(a, a_in, sizeof(double) * n * n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = (r == c) ? 1.0 : 0.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * n + col]) > fabs(a[piv * n + col])) piv = r;
        if (a[piv * n + col] == 0.0) return -1;
        if (piv != col) {
            for (int c = 0; c < n; ++c) {
                double t = a[col * n + c]; a[col * n + c] = a[piv * n + c]; a[piv * n + c] = t;
                t = inv[col * n + c]; inv[col * n + c] = inv[piv * n + c]; inv[piv * n + c] = t;
            }
        }
        double d = a[col * n + col];
        for (int c = 0; c < n; ++c) { a[col * n + c] /= d; inv[col * n + c] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = a[r * n + col];
            if (f == 0.0) continue;
            for (int c = 0; c < n; ++c) {
                a[r * n + c] -= f * a[col * n + c];
                inv[r * n + c] -= f * inv[col * n + c];
            }
        }
    }
    return 0;
}

/* Eq. omega-D with lambda = I and dt = 1: D = (omega^-1 - I/2) cs^2, hence
 * omega = (D / cs^2 + I/2)^-1.  Returns 0, or -1 if the matrix is singular. */
int orc_relaxation_matrix(int m, const double *D, double *omega) {
    double winv[ORC_MAX_M * ORC_MAX_M];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) winv[a * m + b] = D[a * m + b] / CS2 + (a == b ? 0.5 : 0.0);
    return gj_inverse(m, winv, omega);
}

/* Appendix, nu = (1/omega - 1/2) cs^2 dt  ->  omega = 1 / (nu / cs^2 + 1/2) */
double orc_fluid_relaxation(double nu) { return 1.0 / (nu / CS2 + 0.5); }

/* Eq. Gi: G_{i,a} = sum_b (delta_ab - omega_ab / 2) W_i c_i.(u S_b + phi_b F) / cs^2.
 * out[a*5 + i]. */
void orc_aux_source(int m, const double *omega, const double *phi, double ux, double uy,
                    const double *S, double Fx, double Fy, double *out) {
    for (int a = 0; a < m; ++a)
        for (int i = 0; i < 5; ++i) {
            double acc = 0.0;
            for (int b = 0; b < m; ++b) {
                double coef = (a == b ? 1.0 : 0.0) - 0.5 * omega[a * m + b];
                double vx = ux * S[b] + phi[b] * Fx;
                double vy = uy * S[b] + phi[b] * Fy;
                acc += coef * Q5_W[i] * (Q5_CX[i] * vx + Q5_CY[i] * vy) / CS2;
            }
            out[a * 5 + i] = acc;
        }
}

/* Case 1 of Sec. 2.1: G_{i,a} = sum_b (delta_ab - omega_ab / 2) W_i c_i.d_t(phi_b u) / cs^2,
 * d_t(phi_b u) = u (phi_b - phi_prev_b) (steady u, first-order explicit difference).
 * out[a*5 + i]. */
void orc_aux_source_case1(int m, const double *omega, const double *phi_prev, const double *phi, double ux,
                          double uy, double *out) {
    for (int a = 0; a < m; ++a)
        for (int i = 0; i < 5; ++i) {
            double acc = 0.0;
            for (int b = 0; b < m; ++b) {
                double coef = a == b ? 1.0 - 0.5 * omega[a * m + b] : -0.5 * omega[a * m + b];
                double dphi = phi[b] - phi_prev[b];
                acc += coef * Q5_W[i] * (Q5_CX[i] * ux + Q5_CY[i] * uy) * dphi / CS2;
            }
            out[a * 5 + i] = acc;
        }
}

/* Chemotactic cut-off r(c): step form (Sec. 3.1.3) or regularised form (Sec. 3.1.2). */
double orc_cutoff(double c, double c_star, double eps, int regularised) {
    if (regularised) {
        double d = c - c_star;
        return 0.5 * (1.0 + d / sqrt(d * d + eps * eps));
    }
    return c >= c_star ? 1.0 : 0.0;
}

/* Model closures at one node from its scalar moments (Sec. 3.1 and 3.2):
 * diffusion matrix D(phi) (m x m), source S(phi) (m), force F(phi) (2). */
void orc_closures(const orc_params *P, const double *phi, double *D, double *S, double *F) {
    int m = P->m;
    double r = 0.0;
    if (P->dkind == ORC_D_CHEMOTAXIS || P->skind == ORC_S_CONSUMPTION)
        r = orc_cutoff(phi[1], P->c_star, P->eps, P->r_regularised);
    for (int a = 0; a < m * m; ++a) D[a] = P->D[a];
    if (P->dkind == ORC_D_CHEMOTAXIS) D[0 * m + 1] += -P->chi * phi[0] * r;
    for (int a = 0; a < m; ++a) S[a] = 0.0;
    if (P->skind == ORC_S_CONST)
        for (int a = 0; a < m; ++a) S[a] = P->S[a];
    if (P->skind == ORC_S_CONSUMPTION) S[1] = -P->k * phi[0] * r;
    double mag = P->F0;
    for (int a = 0; a < m; ++a) mag += P->beta[a] * (phi[a] - P->phi_ref[a]);
    F[0] = P->g[0] * mag;
    F[1] = P->g[1] * mag;
}

/* ---- the lattice --------------------------------------------------------------- */
typedef struct {
    orc_params P;
    long t;
    double *f;     /* [node][a][5] pre-collision scalar populations at time t */
    double *h;     /* [node][9]    pre-collision fluid populations at time t */
    double *sprev; /* [node][a]    S_a(t-1) */
    double *fpost, *hpost, *fnew, *hnew;
    double *uf;      /* [node][2] prescribed velocity (Case 1) */
    double *phiprev; /* [node][a] phi_a(t-1) (Case 1) */
} orc_sim;

#define NODE(P, x, y) ((long)(y) * (P)->nx + (x))

static int params_ok(const orc_params *P) {
    if (P->nx < 1 || P->ny < 1 || P->m < 1 || P->m > ORC_MAX_M) return 0;
    if ((P->dkind == ORC_D_CHEMOTAXIS || P->skind == ORC_S_CONSUMPTION) && P->m < 2) return 0;
    if ((P->side_kind[ORC_WEST] == ORC_PERIODIC) != (P->side_kind[ORC_EAST] == ORC_PERIODIC)) return 0;
    if ((P->side_kind[ORC_SOUTH] == ORC_PERIODIC) != (P->side_kind[ORC_NORTH] == ORC_PERIODIC)) return 0;
    if (!(P->nu > 0.0)) return 0;
    return 1;
}

orc_sim *orc_create(const orc_params *P) {
    if (!params_ok(P)) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->P = *P;
    long n = (long)P->nx * P->ny;
    s->f = (double *)calloc((size_t)n * P->m * 5, sizeof(double));
    s->fpost = (double *)calloc((size_t)n * P->m * 5, sizeof(double));
    s->fnew = (double *)calloc((size_t)n * P->m * 5, sizeof(double));
    s->h = (double *)calloc((size_t)n * 9, sizeof(double));
    s->hpost = (double *)calloc((size_t)n * 9, sizeof(double));
    s->hnew = (double *)calloc((size_t)n * 9, sizeof(double));
    s->sprev = (double *)calloc((size_t)n * P->m, sizeof(double));
    s->uf = (double *)calloc((size_t)n * 2, sizeof(double));
    s->phiprev = (double *)calloc((size_t)n * P->m, sizeof(double));
    if (!s->f || !s->fpost || !s->fnew || !s->h || !s->hpost || !s->hnew || !s->sprev || !s->uf || !s->phiprev) {
        free(s->f); free(s->fpost); free(s->fnew); free(s->h); free(s->hpost); free(s->hnew);
        free(s->sprev); free(s->uf); free(s->phiprev); free(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->f); free(s->fpost); free(s->fnew);
    free(s->h); free(s->hpost); free(s->hnew); free(s->sprev);
    free(s->uf); free(s->phiprev);
    free(s);
}

long orc_time(const orc_sim *s) { return s->t; }

/* Step 1 of the update: moments of one node's pre-collision populations
 * (Eq. sum-phi, sum-u, and the pressure of the appendix's derivation) and the
 * closures.  The appendix obtains p from h_0 = h_0^eq + h_0^ne with
 * h_0^ne = (1/omega - 1/2) F_0 and F_0 = -W_0 varphi u.F / cs^2, i.e.
 * p = cs^2/(1 - W_0) [sum_{i!=0} h_i - W_0 u.u/(2 cs^2) - W_0 varphi (1/omega - 1/2) u.F / cs^2];
 * the printed Eq. sum-p has the opposite sign and no W_0 on the varphi term, the
 * appendix's last line the sign of the derivation and no W_0 (moot at varphi = 0). */
static void node_moments(const orc_sim *s, long node, double *phi, double *u, double *p,
                         double *D, double *S, double *F) {
    const orc_params *P = &s->P;
    int m = P->m;
    const double *f = s->f + node * m * 5;
    const double *h = s->h + node * 9;
    for (int a = 0; a < m; ++a) {
        phi[a] = 0.0;
        for (int i = 0; i < 5; ++i) phi[a] += f[a * 5 + i];
    }
    orc_closures(P, phi, D, S, F);
    if (P->case1) { /* Case 1: the velocity is prescribed; no fluid, no force */
        u[0] = s->uf[node * 2];
        u[1] = s->uf[node * 2 + 1];
        *p = 0.0;
        F[0] = F[1] = 0.0;
        return;
    }
    double jx = 0.0, jy = 0.0, sum_nonrest = 0.0;
    for (int i = 0; i < 9; ++i) {
        jx += Q9_CX[i] * h[i];
        jy += Q9_CY[i] * h[i];
        if (i != 0) sum_nonrest += h[i];
    }
    u[0] = jx + 0.5 * F[0];
    u[1] = jy + 0.5 * F[1];
    double uu = u[0] * u[0] + u[1] * u[1];
    double uF = u[0] * F[0] + u[1] * F[1];
    double omega_f = orc_fluid_relaxation(P->nu);
    *p = CS2 / (1.0 - Q9_W[0]) *
         ((sum_nonrest - Q9_W[0] * uu / (2.0 * CS2)) - Q9_W[0] * P->varphi * (1.0 / omega_f - 0.5) * uF / CS2);
}

/* Steps 1-4 for one node: writes the post-collision populations and updates S(t-1). */
static int node_collide(orc_sim *s, long node, double *fpost, double *hpost, int update_sprev) {
    const orc_params *P = &s->P;
    int m = P->m;
    double phi[ORC_MAX_M], u[2], p, D[ORC_MAX_M * ORC_MAX_M], S[ORC_MAX_M], F[2];
    node_moments(s, node, phi, u, &p, D, S, F);

    double omega[ORC_MAX_M * ORC_MAX_M];
    if (orc_relaxation_matrix(m, D, omega) != 0) return -1;
    double omega_f = orc_fluid_relaxation(P->nu);

    double feq[ORC_MAX_M][5], G[ORC_MAX_M * 5];
    for (int a = 0; a < m; ++a) orc_feq_scalar(phi[a], u[0], u[1], P->theta, feq[a]);
    if (P->case1)
        orc_aux_source_case1(m, omega, s->phiprev + node * m, phi, u[0], u[1], G);
    else
        orc_aux_source(m, omega, phi, u[0], u[1], S, F[0], F[1], G);

    const double *f = s->f + node * m * 5;
    double *sp = s->sprev + node * m;
    for (int a = 0; a < m; ++a)
        for (int i = 0; i < 5; ++i) {
            double coll = 0.0;
            for (int b = 0; b < m; ++b) coll += omega[a * m + b] * (f[b * 5 + i] - feq[b][i]);
            double Si = Q5_W[i] * S[a];         /* Eq. source */
            double Si_prev = Q5_W[i] * sp[a];
            fpost[a * 5 + i] = f[a * 5 + i] - coll + Si + G[a * 5 + i] + 0.5 * (Si - Si_prev);
        }
    if (update_sprev)
        for (int a = 0; a < m; ++a) sp[a] = S[a];
    if (update_sprev && P->case1)
        for (int a = 0; a < m; ++a) s->phiprev[node * m + a] = phi[a];
    if (P->case1) {
        for (int i = 0; i < 9; ++i) hpost[i] = 0.0;
        return 0;
    }

    const double *h = s->h + node * 9;
    double heq[9], Fi[9];
    orc_heq(p, u[0], u[1], P->rho0, heq);
    orc_force_pop_phi(F[0], F[1], u[0], u[1], P->varphi, Fi);
    for (int i = 0; i < 9; ++i)
        hpost[i] = h[i] - omega_f * (h[i] - heq[i]) + (1.0 - 0.5 * omega_f) * Fi[i];
    return 0;
}

/* Which wall (if any) a target coordinate crosses. */
static int crossed_side_x(const orc_params *P, int tx) {
    if (tx < 0 && P->side_kind[ORC_WEST] == ORC_WALL) return ORC_WEST;
    if (tx >= P->nx && P->side_kind[ORC_EAST] == ORC_WALL) return ORC_EAST;
    return -1;
}
static int crossed_side_y(const orc_params *P, int ty) {
    if (ty < 0 && P->side_kind[ORC_SOUTH] == ORC_WALL) return ORC_SOUTH;
    if (ty >= P->ny && P->side_kind[ORC_NORTH] == ORC_WALL) return ORC_NORTH;
    return -1;
}
static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* Threads of the node and row loops of orc_step (1 unless orc_set_threads asks
 * for more; only the timed CPU baseline does).  Every node's arithmetic is the
 * same whatever the thread count, and the push writes every target slot once,
 * so the results do not depend on it. */
static int g_threads = 1;

/* Sets the thread count (n < 1: all cores); returns the count in use (1 when the
 * oracle was built without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
    g_threads = n < 1 ? omp_get_num_procs() : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* Step 5: push every post-collision population along its link. */
static void stream(orc_sim *s) {
    const orc_params *P = &s->P;
    int m = P->m, nx = P->nx, ny = P->ny;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static)
#endif
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long node = NODE(P, x, y);
            /* scalars, D2Q5 */
            for (int a = 0; a < m; ++a)
                for (int i = 0; i < 5; ++i) {
                    double v = s->fpost[(node * m + a) * 5 + i];
                    int tx = x + Q5_CX[i], ty = y + Q5_CY[i];
                    int sx = crossed_side_x(P, tx), sy = crossed_side_y(P, ty);
                    int side = sx >= 0 ? sx : sy;
                    if (side < 0) {
                        long tn = NODE(P, wrap(tx, nx), wrap(ty, ny));
                        s->fnew[(tn * m + a) * 5 + i] = v;
                    } else {
                        int io = q5_dir(-Q5_CX[i], -Q5_CY[i]);
                        if (P->scalar_bc[side][a] == ORC_DIRICHLET) /* anti-bounce-back */
                            s->fnew[(node * m + a) * 5 + io] = -v + 2.0 * Q5_W[i] * P->value[side][a];
                        else /* half-way bounce-back: no flux */
                            s->fnew[(node * m + a) * 5 + io] = v;
                    }
                }
            /* fluid, D2Q9 */
            for (int i = 0; i < 9; ++i) {
                double v = s->hpost[node * 9 + i];
                int tx = x + Q9_CX[i], ty = y + Q9_CY[i];
                int sx = crossed_side_x(P, tx), sy = crossed_side_y(P, ty);
                int io = q9_dir(-Q9_CX[i], -Q9_CY[i]);
                if (sx < 0 && sy < 0) {
                    s->hnew[NODE(P, wrap(tx, nx), wrap(ty, ny)) * 9 + i] = v;
                } else if (sx >= 0 && sy >= 0) {
                    s->hnew[node * 9 + io] = v; /* corner: bounce-back */
                } else if (sy >= 0 && P->fluid_bc[sy] == ORC_FREESLIP) {
                    /* specular reflection at a horizontal wall: c_y flips, the link
                       lands on the neighbour along x (never beyond a wall here) */
                    int j = q9_dir(Q9_CX[i], -Q9_CY[i]);
                    s->hnew[NODE(P, wrap(tx, nx), y) * 9 + j] = v;
                } else if (sx >= 0 && P->fluid_bc[sx] == ORC_FREESLIP) {
                    int j = q9_dir(-Q9_CX[i], Q9_CY[i]);
                    s->hnew[NODE(P, x, wrap(ty, ny)) * 9 + j] = v;
                } else {
                    s->hnew[node * 9 + io] = v; /* no slip: half-way bounce-back */
                }
            }
        }
}

/* Initial state from moments (layouts [a][y][x], [2][y][x], [y][x]; p may be NULL). */
int orc_init(orc_sim *s, const double *phi0, const double *u0, const double *p0) {
    const orc_params *P = &s->P;
    int m = P->m;
    long n = (long)P->nx * P->ny;
    for (long node = 0; node < n; ++node) {
        double phi[ORC_MAX_M], D[ORC_MAX_M * ORC_MAX_M], S[ORC_MAX_M], F[2];
        for (int a = 0; a < m; ++a) phi[a] = phi0[a * n + node];
        double ux = u0[node], uy = u0[n + node], p = p0 ? p0[node] : 0.0;
        orc_closures(P, phi, D, S, F);
        for (int a = 0; a < m; ++a) {
            orc_feq_scalar(phi[a], ux, uy, P->theta, s->f + (node * m + a) * 5);
            s->sprev[node * m + a] = S[a];
            s->phiprev[node * m + a] = phi[a];
        }
        s->uf[node * 2] = ux;
        s->uf[node * 2 + 1] = uy;
        if (P->case1) {
            for (int i = 0; i < 9; ++i) s->h[node * 9 + i] = 0.0;
            continue;
        }
        double heq[9], Fi[9];
        orc_heq(p, ux, uy, P->rho0, heq);
        orc_force_pop_phi(F[0], F[1], ux, uy, P->varphi, Fi);
        for (int i = 0; i < 9; ++i) s->h[node * 9 + i] = heq[i] - 0.5 * Fi[i];
    }
    s->t = 0;
    return 0;
}

/* Advance n time steps.  Returns 0, or -1 if a relaxation matrix was singular. */
int orc_step(orc_sim *s, long nsteps) {
    const orc_params *P = &s->P;
    long n = (long)P->nx * P->ny;
    int m = P->m;
    for (long it = 0; it < nsteps; ++it) {
        int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(| : bad)
#endif
        for (long node = 0; node < n; ++node)
            bad |= node_collide(s, node, s->fpost + node * m * 5, s->hpost + node * 9, 1) != 0;
        if (bad) return -1;
        stream(s);
        double *t;
        t = s->f; s->f = s->fnew; s->fnew = t;
        t = s->h; s->h = s->hnew; s->hnew = t;
        s->t += 1;
    }
    return 0;
}

/* Moments at the current time: out[(m+3)][ny][nx] = phi_0..phi_{m-1}, u_x, u_y, p. */
void orc_moments(const orc_sim *s, double *out) {
    const orc_params *P = &s->P;
    int m = P->m;
    long n = (long)P->nx * P->ny;
    for (long node = 0; node < n; ++node) {
        double phi[ORC_MAX_M], u[2], p, D[ORC_MAX_M * ORC_MAX_M], S[ORC_MAX_M], F[2];
        node_moments(s, node, phi, u, &p, D, S, F);
        for (int a = 0; a < m; ++a) out[a * n + node] = phi[a];
        out[m * n + node] = u[0];
        out[(m + 1) * n + node] = u[1];
        out[(m + 2) * n + node] = p;
    }
}

/* Pre-collision populations at the current time, planar layouts
 * f[a][i][y][x], h[i][y][x], sprev[a][y][x]. */
void orc_get_state(const orc_sim *s, double *f, double *h, double *sprev) {
    const orc_params *P = &s->P;
    int m = P->m;
    long n = (long)P->nx * P->ny;
    for (long node = 0; node < n; ++node) {
        for (int a = 0; a < m; ++a) {
            for (int i = 0; i < 5; ++i) f[(a * 5 + i) * n + node] = s->f[(node * m + a) * 5 + i];
            if (sprev) sprev[a * n + node] = s->sprev[node * m + a];
        }
        for (int i = 0; i < 9; ++i) h[i * n + node] = s->h[node * 9 + i];
    }
}

void orc_set_state(orc_sim *s, const double *f, const double *h, const double *sprev) {
    const orc_params *P = &s->P;
    int m = P->m;
    long n = (long)P->nx * P->ny;
    for (long node = 0; node < n; ++node) {
        for (int a = 0; a < m; ++a) {
            for (int i = 0; i < 5; ++i) s->f[(node * m + a) * 5 + i] = f[(a * 5 + i) * n + node];
            s->sprev[node * m + a] = sprev ? sprev[a * n + node] : 0.0;
        }
        for (int i = 0; i < 9; ++i) s->h[node * 9 + i] = h[i * n + node];
    }
}

/* Post-collision populations of the current state (steps 1-4 without streaming
 * and without advancing time), planar layouts as in orc_get_state. */
int orc_post_collision(orc_sim *s, double *f, double *h) {
    const orc_params *P = &s->P;
    int m = P->m;
    long n = (long)P->nx * P->ny;
    double fp[ORC_MAX_M * 5], hp[9];
    for (long node = 0; node < n; ++node) {
        if (node_collide(s, node, fp, hp, 0) != 0) return -1;
        for (int a = 0; a < m; ++a)
            for (int i = 0; i < 5; ++i) f[(a * 5 + i) * n + node] = fp[a * 5 + i];
        for (int i = 0; i < 9; ++i) h[i * n + node] = hp[i];
    }
    return 0;
}
