/*
 * cdf_oracle3d.c -- CPU FP64 oracle of the three-dimensional form of the lattice
 * Boltzmann model of Zhan, Chai & Shi (arXiv:2101.03055): D3Q7 for the m scalar
 * sets (Eq. D3Q7, cs^2 = 1/4) and D3Q19 for the fluid (Eq. D3Q19, cs^2 = 1/3).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or helper with the CUDA library (nor with the 2-D oracle).
 *
 * Same order of operations as the 2-D oracle, every time step t -> t+1, node by
 * node in FP64, array-of-structures storage:
 *   1. phi_a = sum_i f_{i,a} (Eq. sum-phi); closures D(phi), S(phi), F(phi);
 *      u = sum_i c_i h_i + F/2 (Eq. sum-u);
 *      p = cs^2/(1 - W0) [sum_{i!=0} h_i - W0 u.u/(2 cs^2)] (Eq. sum-p, varphi = 0)
 *   2. omega = (D/cs_s^2 + I/2)^-1 with the scalar lattice's cs_s^2 = 1/4
 *      (Eq. omega-D, lambda = I); omega_f = 1/(nu/cs^2 + 1/2)
 *   3. f^eq_i = W_i phi (1 + c_i.u/cs_s^2) (Eq. feq-phi, lambda = I, vartheta = 0);
 *      h^eq_i = sigma_i + W_i [c_i.u/cs^2 + uu:(c_i c_i - cs^2 I)/(2 cs^4)] (Eq. heq)
 *   4. f*_{i,a} = f_{i,a} - sum_b omega_ab (f_{i,b} - f^eq_{i,b}) + W_i S_a
 *                 + (W_i S_a - W_i S_a(t-1))/2 + G_{i,a}                (Eq. evolution12)
 *      G_{i,a} = sum_b (delta_ab - omega_ab/2) W_i c_i.(u S_b + phi_b F)/cs_s^2 (Eq. Gi)
 *      h*_i = h_i - omega_f (h_i - h^eq_i) + (1 - omega_f/2) W_i c_i.F/cs^2 (Eqs. evolution3, force)
 *   5. streaming f(x + c_i, t+1) = f*(x, t); a link that leaves through a wall
 *      is bounced back half-way (no slip / no flux) or anti-bounced back
 *      (Dirichlet scalar phi_w: -f* + 2 W_i phi_w); a link that crosses two or
 *      three walls at once (edges, corners) is bounced back.
 * Initial state: f = f^eq(phi0, u0), h = h^eq(u0, p0) - F_i/2, S(t-1) = S(phi0).
 * Closures as in Sec. 3: D_01 += -chi phi_0 r(phi_1) (chemotaxis), S_1 =
 * -k phi_0 r(phi_1) (consumption), F = g (F0 + sum_a beta_a (phi_a - phi_ref_a)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define O3_MAX_M 8

enum { O3_PERIODIC = 0, O3_WALL = 1 };
enum { O3_NOFLUX = 0, O3_DIRICHLET = 1 };

typedef struct {
    int nx, ny, nz, m;
    int dkind; /* 0 const, 1 chemotaxis */
    double D[O3_MAX_M * O3_MAX_M];
    double chi, c_star, eps;
    int r_regularised;
    int skind; /* 0 none, 1 const, 2 consumption */
    double S[O3_MAX_M];
    double k;
    double g[3];
    double beta[O3_MAX_M];
    double phi_ref[O3_MAX_M];
    double F0;
    double nu, rho0;
    int side_kind[6];               /* x-, x+, y-, y+, z-, z+ */
    int scalar_bc[6][O3_MAX_M];
    double value[6][O3_MAX_M];
} o3_params;

/* ---- lattices (Eq. D3Q7, Eq. D3Q19), c_hat = 1 ---------------------------------- */
static const double CS2S = 1.0 / 4.0; /* D3Q7 */
static const int Q7_C[7][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}};
static const double Q7_W[7] = {1.0 / 4.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0};
static const double CS2 = 1.0 / 3.0; /* D3Q19 */
static const int Q19_C[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {-1, 0, 1},
    {1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19_0 = 1.0 / 3.0, W19_1 = 1.0 / 18.0, W19_2 = 1.0 / 36.0;

static double q19_w(int i) { return i == 0 ? W19_0 : (i < 7 ? W19_1 : W19_2); }
static int q7_dir(int cx, int cy, int cz) {
    for (int i = 0; i < 7; ++i)
        if (Q7_C[i][0] == cx && Q7_C[i][1] == cy && Q7_C[i][2] == cz) return i;
    return -1;
}
static int q19_dir(int cx, int cy, int cz) {
    for (int i = 0; i < 19; ++i)
        if (Q19_C[i][0] == cx && Q19_C[i][1] == cy && Q19_C[i][2] == cz) return i;
    return -1;
}

/* ---- single-node building blocks (exported for the pins) -------------------------- */
void o3_feq_scalar(double phi, const double *u, double out[7]) {
    for (int i = 0; i < 7; ++i) {
        double cu = Q7_C[i][0] * u[0] + Q7_C[i][1] * u[1] + Q7_C[i][2] * u[2];
        out[i] = Q7_W[i] * (phi + cu * phi / CS2S);
    }
}

void o3_heq(double p, const double *u, double rho0, double out[19]) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double w = q19_w(i);
        double cu = Q19_C[i][0] * u[0] + Q19_C[i][1] * u[1] + Q19_C[i][2] * u[2];
        double uu_cc = cu * cu - CS2 * uu;
        double sigma = (i == 0) ? (w - 1.0) * p / CS2 + rho0 : w * p / CS2;
        out[i] = sigma + w * (cu / CS2 + uu_cc / (2.0 * CS2 * CS2));
    }
}

void o3_force_pop(const double *F, double out[19]) {
    for (int i = 0; i < 19; ++i)
        out[i] = q19_w(i) * (Q19_C[i][0] * F[0] + Q19_C[i][1] * F[1] + Q19_C[i][2] * F[2]) / CS2;
}

static int gj_inverse(int n, const double *a_in, double *inv) {
    double a[O3_MAX_M * O3_MAX_M];
    memcpy(a, a_in, sizeof(double) * n * n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = (r == c) ? 1.0 : 0.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * n + col]) > fabs(a[piv * n + col])) piv = r;
        if (fabs(a[piv * n + col]) < 1e-300) return -1;
        for (int c = 0; c < n; ++c) {
            double t = a[col * n + c]; a[col * n + c] = a[piv * n + c]; a[piv * n + c] = t;
            t = inv[col * n + c]; inv[col * n + c] = inv[piv * n + c]; inv[piv * n + c] = t;
        }
        double d = a[col * n + col];
        for (int c = 0; c < n; ++c) { a[col * n + c] /= d; inv[col * n + c] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = a[r * n + col];
            for (int c = 0; c < n; ++c) { a[r * n + c] -= f * a[col * n + c]; inv[r * n + c] -= f * inv[col * n + c]; }
        }
    }
    return 0;
}

/* Eq. omega-D on the D3Q7 lattice: omega = (D / cs_s^2 + I / 2)^-1. */
int o3_relaxation_matrix(int m, const double *D, double *omega) {
    double winv[O3_MAX_M * O3_MAX_M];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) winv[a * m + b] = D[a * m + b] / CS2S + (a == b ? 0.5 : 0.0);
    return gj_inverse(m, winv, omega);
}

/* Eq. Gi on D3Q7: G_{i,a} = sum_b (delta_ab - omega_ab/2) W_i c_i.(u S_b + phi_b F)/cs_s^2. */
void o3_aux_source(int m, const double *omega, const double *phi, const double *u, const double *S,
                   const double *F, double *out) {
    for (int a = 0; a < m; ++a)
        for (int i = 0; i < 7; ++i) {
            double acc = 0.0;
            for (int b = 0; b < m; ++b) {
                double coef = (a == b ? 1.0 : 0.0) - 0.5 * omega[a * m + b];
                double v = 0.0;
                for (int d = 0; d < 3; ++d) v += Q7_C[i][d] * (u[d] * S[b] + phi[b] * F[d]);
                acc += coef * Q7_W[i] * v / CS2S;
            }
            out[a * 7 + i] = acc;
        }
}

static double cutoff(const o3_params *P, double c) {
    if (P->r_regularised) {
        double d = c - P->c_star;
        return 0.5 * (1.0 + d / sqrt(d * d + P->eps * P->eps));
    }
    return c >= P->c_star ? 1.0 : 0.0;
}

static void closures(const o3_params *P, const double *phi, double *D, double *S, double *F) {
    int m = P->m;
    double r = 0.0;
    if (P->dkind == 1 || P->skind == 2) r = cutoff(P, phi[1]);
    for (int a = 0; a < m * m; ++a) D[a] = P->D[a];
    if (P->dkind == 1) D[0 * m + 1] += -P->chi * phi[0] * r;
    for (int a = 0; a < m; ++a) S[a] = (P->skind == 1) ? P->S[a] : 0.0;
    if (P->skind == 2) S[1] = -P->k * phi[0] * r;
    double mag = P->F0;
    for (int a = 0; a < m; ++a) mag += P->beta[a] * (phi[a] - P->phi_ref[a]);
    for (int d = 0; d < 3; ++d) F[d] = P->g[d] * mag;
}

/* ---- the lattice ------------------------------------------------------------------ */
typedef struct {
    o3_params P;
    long t;
    double *f, *h, *sprev, *fpost, *hpost, *fnew, *hnew;
} o3_sim;

static long n_nodes(const o3_params *P) { return (long)P->nx * P->ny * P->nz; }
static long node_of(const o3_params *P, int x, int y, int z) { return ((long)z * P->ny + y) * P->nx + x; }

o3_sim *o3_create(const o3_params *P) {
    if (P->nx < 1 || P->ny < 1 || P->nz < 1 || P->m < 1 || P->m > O3_MAX_M || !(P->nu > 0.0)) return NULL;
    if ((P->dkind == 1 || P->skind == 2) && P->m < 2) return NULL;
    for (int a = 0; a < 3; ++a)
        if ((P->side_kind[2 * a] == O3_PERIODIC) != (P->side_kind[2 * a + 1] == O3_PERIODIC)) return NULL;
    o3_sim *s = (o3_sim *)calloc(1, sizeof(o3_sim));
    if (!s) return NULL;
    s->P = *P;
    long n = n_nodes(P);
    s->f = (double *)calloc((size_t)n * P->m * 7, sizeof(double));
    s->fpost = (double *)calloc((size_t)n * P->m * 7, sizeof(double));
    s->fnew = (double *)calloc((size_t)n * P->m * 7, sizeof(double));
    s->h = (double *)calloc((size_t)n * 19, sizeof(double));
    s->hpost = (double *)calloc((size_t)n * 19, sizeof(double));
    s->hnew = (double *)calloc((size_t)n * 19, sizeof(double));
    s->sprev = (double *)calloc((size_t)n * P->m, sizeof(double));
    if (!s->f || !s->fpost || !s->fnew || !s->h || !s->hpost || !s->hnew || !s->sprev) {
        free(s->f); free(s->fpost); free(s->fnew); free(s->h); free(s->hpost); free(s->hnew); free(s->sprev);
        free(s);
        return NULL;
    }
    return s;
}

void o3_destroy(o3_sim *s) {
    if (!s) return;
    free(s->f); free(s->fpost); free(s->fnew); free(s->h); free(s->hpost); free(s->hnew); free(s->sprev);
    free(s);
}

long o3_time(const o3_sim *s) { return s->t; }

static void node_moments(const o3_sim *s, long node, double *phi, double *u, double *p, double *D, double *S,
                         double *F) {
    const o3_params *P = &s->P;
    int m = P->m;
    const double *f = s->f + node * m * 7, *h = s->h + node * 19;
    for (int a = 0; a < m; ++a) {
        phi[a] = 0.0;
        for (int i = 0; i < 7; ++i) phi[a] += f[a * 7 + i];
    }
    closures(P, phi, D, S, F);
    double j[3] = {0.0, 0.0, 0.0}, nonrest = 0.0;
    for (int i = 0; i < 19; ++i) {
        for (int d = 0; d < 3; ++d) j[d] += Q19_C[i][d] * h[i];
        if (i != 0) nonrest += h[i];
    }
    for (int d = 0; d < 3; ++d) u[d] = j[d] + 0.5 * F[d];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    *p = CS2 / (1.0 - W19_0) * (nonrest - W19_0 * uu / (2.0 * CS2));
}

static int node_collide(o3_sim *s, long node, double *fpost, double *hpost, int update_sprev) {
    const o3_params *P = &s->P;
    int m = P->m;
    double phi[O3_MAX_M], u[3], p, D[O3_MAX_M * O3_MAX_M], S[O3_MAX_M], F[3];
    node_moments(s, node, phi, u, &p, D, S, F);
    double omega[O3_MAX_M * O3_MAX_M];
    if (o3_relaxation_matrix(m, D, omega) != 0) return -1;
    double omega_f = 1.0 / (P->nu / CS2 + 0.5);
    double feq[O3_MAX_M][7], G[O3_MAX_M * 7];
    for (int a = 0; a < m; ++a) o3_feq_scalar(phi[a], u, feq[a]);
    o3_aux_source(m, omega, phi, u, S, F, G);
    const double *f = s->f + node * m * 7;
    double *sp = s->sprev + node * m;
    for (int a = 0; a < m; ++a)
        for (int i = 0; i < 7; ++i) {
            double coll = 0.0;
            for (int b = 0; b < m; ++b) coll += omega[a * m + b] * (f[b * 7 + i] - feq[b][i]);
            double Si = Q7_W[i] * S[a], Si_prev = Q7_W[i] * sp[a];
            fpost[a * 7 + i] = f[a * 7 + i] - coll + Si + G[a * 7 + i] + 0.5 * (Si - Si_prev);
        }
    if (update_sprev)
        for (int a = 0; a < m; ++a) sp[a] = S[a];
    const double *h = s->h + node * 19;
    double heq[19], Fi[19];
    o3_heq(p, u, P->rho0, heq);
    o3_force_pop(F, Fi);
    for (int i = 0; i < 19; ++i) hpost[i] = h[i] - omega_f * (h[i] - heq[i]) + (1.0 - 0.5 * omega_f) * Fi[i];
    return 0;
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* Side crossed by coordinate v on axis a (0 x, 1 y, 2 z), or -1. */
static int crossed(const o3_params *P, int a, int v, int n) {
    if (v < 0 && P->side_kind[2 * a] == O3_WALL) return 2 * a;
    if (v >= n && P->side_kind[2 * a + 1] == O3_WALL) return 2 * a + 1;
    return -1;
}

static void stream(o3_sim *s) {
    const o3_params *P = &s->P;
    int m = P->m, N[3] = {P->nx, P->ny, P->nz};
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long node = node_of(P, x, y, z);
                int X[3] = {x, y, z};
                for (int a = 0; a < m; ++a)
                    for (int i = 0; i < 7; ++i) {
                        double v = s->fpost[(node * m + a) * 7 + i];
                        int T[3], side = -1;
                        for (int d = 0; d < 3; ++d) {
                            T[d] = X[d] + Q7_C[i][d];
                            int c = crossed(P, d, T[d], N[d]);
                            if (c >= 0) side = c;
                        }
                        if (side < 0) {
                            long tn = node_of(P, wrap(T[0], N[0]), wrap(T[1], N[1]), wrap(T[2], N[2]));
                            s->fnew[(tn * m + a) * 7 + i] = v;
                        } else {
                            int io = q7_dir(-Q7_C[i][0], -Q7_C[i][1], -Q7_C[i][2]);
                            if (P->scalar_bc[side][a] == O3_DIRICHLET)
                                s->fnew[(node * m + a) * 7 + io] = -v + 2.0 * Q7_W[i] * P->value[side][a];
                            else
                                s->fnew[(node * m + a) * 7 + io] = v;
                        }
                    }
                for (int i = 0; i < 19; ++i) {
                    double v = s->hpost[node * 19 + i];
                    int T[3], walls = 0;
                    for (int d = 0; d < 3; ++d) {
                        T[d] = X[d] + Q19_C[i][d];
                        if (crossed(P, d, T[d], N[d]) >= 0) ++walls;
                    }
                    if (walls == 0) {
                        s->hnew[node_of(P, wrap(T[0], N[0]), wrap(T[1], N[1]), wrap(T[2], N[2])) * 19 + i] = v;
                    } else { /* no slip: half-way bounce-back (also through edges and corners) */
                        int io = q19_dir(-Q19_C[i][0], -Q19_C[i][1], -Q19_C[i][2]);
                        s->hnew[node * 19 + io] = v;
                    }
                }
            }
}

/* Initial state from moments ([a][z][y][x], [3][z][y][x], [z][y][x]; p may be NULL). */
int o3_init(o3_sim *s, const double *phi0, const double *u0, const double *p0) {
    const o3_params *P = &s->P;
    int m = P->m;
    long n = n_nodes(P);
    for (long node = 0; node < n; ++node) {
        double phi[O3_MAX_M], D[O3_MAX_M * O3_MAX_M], S[O3_MAX_M], F[3];
        for (int a = 0; a < m; ++a) phi[a] = phi0[a * n + node];
        double u[3] = {u0[node], u0[n + node], u0[2 * n + node]}, p = p0 ? p0[node] : 0.0;
        closures(P, phi, D, S, F);
        for (int a = 0; a < m; ++a) {
            o3_feq_scalar(phi[a], u, s->f + (node * m + a) * 7);
            s->sprev[node * m + a] = S[a];
        }
        double heq[19], Fi[19];
        o3_heq(p, u, P->rho0, heq);
        o3_force_pop(F, Fi);
        for (int i = 0; i < 19; ++i) s->h[node * 19 + i] = heq[i] - 0.5 * Fi[i];
    }
    s->t = 0;
    return 0;
}

int o3_step(o3_sim *s, long nsteps) {
    const o3_params *P = &s->P;
    long n = n_nodes(P);
    int m = P->m;
    for (long it = 0; it < nsteps; ++it) {
        for (long node = 0; node < n; ++node)
            if (node_collide(s, node, s->fpost + node * m * 7, s->hpost + node * 19, 1) != 0) return -1;
        stream(s);
        double *t;
        t = s->f; s->f = s->fnew; s->fnew = t;
        t = s->h; s->h = s->hnew; s->hnew = t;
        s->t += 1;
    }
    return 0;
}

/* out[(m+4)][nz][ny][nx] = phi_0..phi_{m-1}, u_x, u_y, u_z, p. */
void o3_moments(const o3_sim *s, double *out) {
    const o3_params *P = &s->P;
    int m = P->m;
    long n = n_nodes(P);
    for (long node = 0; node < n; ++node) {
        double phi[O3_MAX_M], u[3], p, D[O3_MAX_M * O3_MAX_M], S[O3_MAX_M], F[3];
        node_moments(s, node, phi, u, &p, D, S, F);
        for (int a = 0; a < m; ++a) out[a * n + node] = phi[a];
        for (int d = 0; d < 3; ++d) out[(m + d) * n + node] = u[d];
        out[(m + 3) * n + node] = p;
    }
}

/* Post-collision populations of the current state, planar f[a][i][...], h[i][...]. */
int o3_post_collision(o3_sim *s, double *f, double *h) {
    const o3_params *P = &s->P;
    int m = P->m;
    long n = n_nodes(P);
    double fp[O3_MAX_M * 7], hp[19];
    for (long node = 0; node < n; ++node) {
        if (node_collide(s, node, fp, hp, 0) != 0) return -1;
        for (int a = 0; a < m; ++a)
            for (int i = 0; i < 7; ++i) f[(a * 7 + i) * n + node] = fp[a * 7 + i];
        for (int i = 0; i < 19; ++i) h[i * n + node] = hp[i];
    }
    return 0;
}
