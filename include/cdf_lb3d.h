/*
 * cdf_lb3d.h -- C ABI of the three-dimensional form of the lattice Boltzmann
 * model for the coupled cross-diffusion-fluid system (Zhan, Chai & Shi,
 * arXiv:2101.03055): D3Q7 for the m scalar sets (Eq. D3Q7, cs^2 = 1/4) and
 * D3Q19 for the fluid (Eq. D3Q19, cs^2 = 1/3), with the collision of Eqs.
 * evolution12/evolution3, the equilibria of Eqs. feq-phi (lambda = I,
 * vartheta = 0) and heq, the force of Eq. force (varphi = 0), the source and
 * auxiliary source of Eqs. source and Gi, and the moments of Eqs. sum-phi,
 * sum-u and sum-p, all in the form the paper writes for d dimensions.
 *
 * Conventions as in cdf_lb.h (status codes, cdf_lb_last_error(), ownership,
 * streams, lattice units with dx = dt = 1): fields are [z][y][x] with x
 * fastest; populations are stored in FP32 only.  Walls are half-way: no slip
 * for the fluid (also through edges and corners), no flux (bounce-back) or
 * Dirichlet (anti-bounce-back) per scalar; there is no free-slip wall in 3-D.
 * The scalar count is 1 <= m <= 3.
 */
#ifndef CDF_LB3D_H
#define CDF_LB3D_H

#include "cdf_lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { int nx, ny, nz; } cdf_grid3;

/* F = g (F0 + sum_a beta_a (phi_a - phi_ref_a)), g a 3-vector. */
typedef struct {
    double g[3];
    double beta[CDF_MAX_M];
    double phi_ref[CDF_MAX_M];
    double F0;
} cdf_force3;

/* Sides in the order x-, x+, y-, y+, z-, z+ (cdf_side.fluid is ignored: walls
 * are no slip).  Opposite sides must both be periodic or both walls. */
typedef struct { cdf_side side[6]; } cdf_boundaries3;

typedef struct {
    double rho0;                 /* the constant of sigma_0 in Eq. heq (> 0) */
    void *cuda_stream;           /* cudaStream_t of the caller, NULL = default */
    double phi_ref[CDF_MAX_M];   /* reference scalar values of the stored deviations */
    double p_ref_grad[3];        /* reference pressure gradient (walled axes only) */
    int block_x, block_y;        /* CTA shape of the step kernel (x, y; one z plane per CTA
                                    row of the grid); 0 = autotuned */
} cdf_options3;

typedef struct {
    int nx, ny, nz, m, pitch;    /* pitch: elements per stored x row */
    int block_x, block_y;
    double bytes_per_lup;        /* algorithmic bytes per node update: 2 (19 + 7m) 4 (+ 8 with S(t-1)) */
    long long t;
} cdf_info3;

typedef struct cdf_lb3d cdf_lb3d;

/* Create a solver for one nx x ny x nz lattice.  Checks as cdf_lb_create;
 * 1 <= m <= 3.  On failure *out is NULL and nothing is leaked. */
cdf_status cdf_lb3d_create(const cdf_grid3 *grid, int m, const cdf_diffusion *diffusion, double nu,
                           const cdf_source *source, const cdf_force3 *force, const cdf_boundaries3 *boundaries,
                           const cdf_options3 *options, cdf_lb3d **out);
/* State at t = 0 from host FP64 moments phi [m][nz][ny][nx], u [3][nz][ny][nx],
 * p [nz][ny][nx] or NULL: f = f^eq(phi, u), h = h^eq(u, p) - F_i/2, S(t-1) = S(phi). */
cdf_status cdf_lb3d_init_moments(cdf_lb3d *h, const double *phi, const double *u, const double *p);
/* Advance n >= 0 steps (one fused kernel per step, CUDA-graph launched). */
cdf_status cdf_lb3d_step(cdf_lb3d *h, long long n);
/* Stop test of cdf_lb_run_to_steady over phi_0..phi_{m-1} and the velocity taken
 * as one field: R_u = sum(|du_x| + |du_y| + |du_z|) / sum(|u_x| + |u_y| + |u_z|). */
cdf_status cdf_lb3d_run_to_steady(cdf_lb3d *h, double tol, long long check_every, long long max_steps,
                                  long long *steps_taken, double *residual);
/* Moments at the current time into a host FP64 stack [m+4][nz][ny][nx]:
 * phi_0..phi_{m-1}, u_x, u_y, u_z, p. */
cdf_status cdf_lb3d_moments(cdf_lb3d *h, double *host_out);
/* FP64 totals sum_x phi_a(x) (m values, host). */
cdf_status cdf_lb3d_mass(cdf_lb3d *h, double *sums);
/* Post-collision populations of the current time (full values, FP64 host):
 * f [m][7][nz][ny][nx], h [19][nz][ny][nx]; either may be NULL. */
cdf_status cdf_lb3d_populations(cdf_lb3d *h, double *f, double *hf);
cdf_status cdf_lb3d_get_info(const cdf_lb3d *h, cdf_info3 *out);
void *cdf_lb3d_stream(const cdf_lb3d *h);
void cdf_lb3d_destroy(cdf_lb3d *h);

#ifdef __cplusplus
}
#endif
#endif /* CDF_LB3D_H */
