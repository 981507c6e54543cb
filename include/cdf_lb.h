/*
 * cdf_lb.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for the
 * coupled cross-diffusion-fluid (CDF) system of Zhan, Chai & Shi,
 * "A lattice Boltzmann model for the coupled cross-diffusion-fluid system"
 * (arXiv:2101.03055).
 *
 * The problem (Eqs. CDE, NS1, NS2 of Sec. 1):
 *   d_t phi_a + div(phi_a u) = div(D_ab grad phi_b) + S_a,   a = 0..m-1
 *   div u = 0,  d_t u + div(u u) = -grad p + div(nu grad u) + F
 * is advanced by the model of Sec. 2 with D2Q5 scalar populations and D2Q9
 * fluid populations (Eqs. D2Q5, D2Q9), lambda = I and varphi = 0 (Sec. 3):
 *   Eq. evolution12 -- scalar update with the matrix collision operator
 *                      omega_ab, the source S_i = W_i S_a (Eq. source), its
 *                      time-derivative correction and the auxiliary source
 *                      G_i (Eq. Gi);
 *   Eq. evolution3  -- fluid update with the force term (Eq. force);
 *   Eq. omega-D     -- omega = (D / cs^2 + I / 2)^-1 (dt = 1);
 *   appendix        -- nu = (1 / omega_f - 1/2) cs^2.
 *
 * Conventions for every call:
 *   - Lattice units: dx = dt = 1.  Fields are row-major [y][x] with x fastest;
 *     a stack of fields is [field][y][x].  Moment stacks hold m + 3 fields:
 *     phi_0 .. phi_{m-1}, u_x, u_y, p.
 *   - Node (i, j) of an axis with walls sits half a spacing inside them
 *     (half-way walls); on a periodic axis node i sits at x = i.
 *   - A handle owns all the device memory it allocates.  Pointers passed in
 *     belong to the caller and are not retained after the call returns.
 *   - Device pointers must be on the device that was current at create time.
 *   - Work is ordered on the caller's stream (options.cuda_stream, NULL = the
 *     legacy default stream): each call waits for earlier work on that stream
 *     and later work on it waits for the call.  Calls that return host data
 *     synchronise before they return.
 *   - Every call returns CDF_OK or an error code; cdf_lb_last_error() gives
 *     a message for the calling thread's last failure.  After CDF_ECUDA the
 *     handle should be destroyed.
 */
#ifndef CDF_LB_H
#define CDF_LB_H

#ifdef __cplusplus
extern "C" {
#endif

#define CDF_MAX_M 4 /* scalar sets supported by the kernels */

typedef enum {
    CDF_OK = 0,
    CDF_EINVAL = 1,        /* invalid argument or parameter set */
    CDF_ENOMEM = 2,        /* device or host allocation failed */
    CDF_ECUDA = 3,         /* a CUDA call failed (message has the CUDA error) */
    CDF_ENOTCONVERGED = 4, /* run_to_steady reached max_steps above tol */
    CDF_EUNSTABLE = 5,     /* a NaN or Inf appeared in the fields */
    CDF_ETIMEOUT = 6,      /* a bounded device-side wait ran out */
    CDF_EIO = 7,           /* checkpoint file could not be read or written */
    CDF_ECHECK = 8         /* checks build only: a step kernel met an out-of-range offset, or a
                              canary pad around a device buffer was overwritten */
} cdf_status;

/* Population storage.  Every mode stores each population as its deviation from
 * a reference state -- W_i phi_ref_a for scalar a; h^eq_i(p_ref(x), u = 0) for
 * the fluid, with the linear reference pressure p_ref(x) = p_ref_grad . (x -
 * centre) -- as FP32, FP16 or BF16; every collision is computed in FP32 on
 * these deviations (paper: silent on precision).  The references change no
 * result in exact arithmetic; chosen near the solution (phi_ref inside the
 * scalar range, p_ref_grad the hydrostatic gradient of the mean force) they
 * keep the stored numbers small and the rounding error with them. */
typedef enum { CDF_FP32 = 0, CDF_FP16_DEV = 1, CDF_BF16_DEV = 2 } cdf_storage;

typedef enum { CDF_BC_PERIODIC = 0, CDF_BC_WALL = 1 } cdf_bckind;
typedef enum { CDF_FL_NOSLIP = 0, CDF_FL_FREESLIP = 1 } cdf_fluid_bc;
typedef enum { CDF_SC_NOFLUX = 0, CDF_SC_DIRICHLET = 1 } cdf_scalar_bc;

/* Diffusion matrix D (Eq. CDE).  CDF_D_CONST: D as given.  CDF_D_CHEMOTAXIS
 * (Sec. 3.1): D_01 gets -chi * phi_0 * r(phi_1) added at every node, with the
 * cut-off r(c) = 1 if c >= c_star else 0 (Sec. 3.1.3), or, when
 * r_regularised != 0, r(c) = (1 + (c - c*) / sqrt((c - c*)^2 + eps^2)) / 2
 * (Sec. 3.1.2).  Needs m >= 2. */
typedef enum { CDF_D_CONST = 0, CDF_D_CHEMOTAXIS = 1 } cdf_dkind;
typedef struct {
    int kind;                          /* cdf_dkind */
    double D[CDF_MAX_M * CDF_MAX_M];   /* row-major m x m, lattice units */
    double chi, c_star, eps;
    int r_regularised;
} cdf_diffusion;

/* Source S (Eq. CDE).  CDF_S_CONST: S_a = S[a].  CDF_S_CONSUMPTION (Sec. 3.1):
 * S_1 = -k * phi_0 * r(phi_1), other components 0 (uses the cut-off of the
 * diffusion struct).  Its time derivative enters Eq. evolution12 as the
 * backward difference (S_i(t) - S_i(t-1)) / 2 (Sec. 2.1, gamma = 0). */
typedef enum { CDF_S_NONE = 0, CDF_S_CONST = 1, CDF_S_CONSUMPTION = 2 } cdf_skind;
typedef struct {
    int kind;                          /* cdf_skind */
    double S[CDF_MAX_M];
    double k;
} cdf_source;

/* Body force F = g * (F0 + sum_a beta[a] * (phi_a - phi_ref[a])) (Eq. NS2;
 * Sec. 3.1: F = -Sc gamma n z; Sec. 3.2: F = Ra Pr (T + Nc C) z).
 * varphi is the parameter of Eq. force: 0 (the paper's experiments, Sec. 3)
 * leaves F_i = W_i c_i.F / cs^2; varphi != 0 adds its second-order part
 * W_i varphi (uF + Fu):(c_i c_i - cs^2 I) / (2 cs^4) and gives the pressure the
 * correction of the appendix's derivation, -W_0 varphi (1/omega - 1/2) u.F / cs^2
 * inside the bracket of Eq. sum-p (with W_0 and this sign; the printed Eq. sum-p
 * differs, see the appendix).  varphi = 1 is Case 2 of the appendix. */
typedef struct {
    double g[2];
    double beta[CDF_MAX_M];
    double phi_ref[CDF_MAX_M];
    double F0;
    double varphi;
} cdf_force;

/* One side of the box (Sec. 3: anti-bounce-back for scalar Dirichlet values,
 * half-way bounce-back for no-flux and no-slip; free slip as specular
 * reflection).  Opposite sides must both be periodic or both be walls. */
typedef struct {
    int kind;                          /* cdf_bckind */
    int fluid;                         /* cdf_fluid_bc (walls) */
    int scalar[CDF_MAX_M];             /* cdf_scalar_bc per scalar (walls) */
    double value[CDF_MAX_M];           /* Dirichlet value per scalar */
} cdf_side;
typedef struct { cdf_side west, east, south, north; } cdf_boundaries;

typedef struct { int nx, ny; } cdf_grid;

typedef struct {
    int storage;                       /* cdf_storage */
    double rho0;                       /* the constant of sigma_0 in Eq. heq (> 0) */
    void *cuda_stream;                 /* cudaStream_t of the caller, NULL = default */
    double phi_ref[CDF_MAX_M];         /* reference scalar values of the stored deviations */
    double p_ref_grad[2];              /* reference pressure gradient (used along walled axes only) */
    int block_x, block_y;              /* step kernel CTA shape; block_x = 0: autotuned;
                                          block_y = 0: flat launch of block_x threads (FP32) */
    int resident;                      /* tile-resident persistent step (FP32, lattices that fit
                                          in shared memory, about 150 k nodes for m = 2):
                                          0 = used when the autotuner measures it faster
                                          (not considered with temporal = 1),
                                          1 = always (CDF_EINVAL if the lattice does not fit),
                                          -1 = never */
    double wait_timeout_s;             /* bound of every wait of the resident step; 0 = 1 s */
    int test_stall_tile;               /* test hook: k > 0 makes tile k - 1 of the resident step
                                          never publish its step, so the waits of its neighbours
                                          run out (CDF_ETIMEOUT); 0 in normal use */
    int prescribed_velocity;           /* 1: Case 1 of Sec. 2.1 -- the convection cross-diffusion
                                          equations alone in a steady prescribed velocity, no fluid
                                          populations.  The u passed to the init calls is that
                                          velocity (p is ignored and reported as 0); nu (still
                                          > 0) is not used and the force must be zero; G comes
                                          from the first-order difference u (phi(t) - phi(t - 1)).
                                          FP32 storage only. */
    int temporal;                      /* two time steps per launch (temporal blocking: each CTA
                                          updates its tile and a one-node halo into shared memory,
                                          then the tile again from there; one pass over global
                                          memory serves two steps), full model and Case 1:
                                          0 = used when the autotuner measures it faster,
                                          1 = always, -1 = never; a fixed block_x with
                                          temporal = 0 keeps one step per launch.  FP32: bitwise
                                          the same as one step per launch.  16-bit storage: the
                                          intermediate step stays in FP32 in shared memory, so
                                          the populations are rounded to 16 bits once per two
                                          steps (results differ from one step per launch by that
                                          saved rounding) */
    int temporal_block_x, temporal_block_y, temporal_tile_y;
                                       /* with temporal = 1: the two-step kernel's CTA shape
                                          (block_x 32 or 64: the halo region is block_x nodes wide,
                                          the output tile block_x - 2) and its output tile height;
                                          0 = autotuned.  CDF_EINVAL if it cannot run the lattice
                                          (periodic axes need nx >= block_x, ny >= tile_y + 2) */
    int halo_rows;                     /* a slab of a lattice split along y (see "split lattice"
                                          below): bit 0 set = row 0 is a halo row, bit 1 set = row
                                          ny - 1 is.  A halo row is not updated by the step; it holds
                                          the neighbouring slab's post-collision populations, written by
                                          cdf_lb_halo_unpack between steps, and the reductions leave it
                                          out.  FP32 storage, full model, one step per launch (resident
                                          and temporal 0 or -1).  0 = a whole lattice */
    int origin_y;                      /* slab: the row of the whole lattice that local row 0 is (-1:
                                          the halo row below row 0 of a periodic axis); 0 otherwise */
    int ny_global;                     /* slab: rows of the whole lattice, whose pressure reference the
                                          slab keeps; 0 = ny (and 0 for a whole lattice) */
    int temporal_lanes;                /* with a given two-step kernel shape: nodes each thread
                                          updates.  2 = the paired-lane kernel (two nodes of a column
                                          collide together on paired FP32 instructions; FP32 storage,
                                          m <= 2, full model, block 32 x 8, tile_y 14 or 30); bitwise
                                          the same as one node per thread.  0 or 1 = one node per
                                          thread.  The autotuner does not time it: it executes 28 %
                                          fewer instructions but needs 126 registers a thread, and at
                                          half the occupancy it measured 20-27 % slower on GB300. */
    int block_lanes;                   /* with a given flat launch (block_x > 0, block_y = 0): nodes
                                          each thread updates.  2 = the paired-lane flat kernel (nodes
                                          t and t + half of the row order collide together on paired
                                          FP32 instructions; FP32 storage, m <= 2, full model); bitwise
                                          the same as one node per thread.  0 or 1 = one.  Not timed by
                                          the autotuner (measured 12 % slower on the 512 x 256 plume,
                                          for the reason given at temporal_lanes). */
} cdf_options;

/* Facts about a handle (for benchmarks and tests). */
typedef struct {
    int nx, ny, m, pitch;              /* pitch: elements per stored row */
    int storage;
    int planes;                        /* population planes per buffer */
    int sprev_planes;                  /* S(t-1) planes (CONSUMPTION: 1) */
    int block_x, block_y;              /* step kernel CTA shape in use */
    int resident;                      /* 1 if the tile-resident persistent step is in use */
    int tile_x, tile_y, tiles;         /* its tile shape (nodes) and number of tiles */
    double bytes_per_lup;              /* minimal HBM bytes moved per node update */
    long long t;                       /* time steps taken since initialisation */
    int temporal;                      /* 1 if two steps run per launch; block_x/y is then that
                                          kernel's CTA shape and tile_x/y its output tile */
    int lanes;                         /* nodes each thread of the step kernel in use updates (1 or 2:
                                          the paired-lane kernels of block_lanes / temporal_lanes) */
} cdf_info;

typedef struct cdf_lb cdf_lb;

/* Create a solver for one nx x ny lattice with m scalar sets (1 <= m <= 4).
 * Checks: nx, ny >= 1; the relaxation matrix of Eq. omega-D exists (D / cs^2 +
 * I / 2 invertible); nu > 0 (so 0 < omega_f < 2); opposite sides both periodic
 * or both walls; chemotaxis and consumption need m >= 2; rho0 > 0.
 * Allocates the device buffers; the populations hold no state until one of
 * the init calls.  On failure *out is NULL and nothing is leaked. */
cdf_status cdf_lb_create(const cdf_grid *grid, int m, const cdf_diffusion *diffusion, double nu,
                         const cdf_source *source, const cdf_force *force,
                         const cdf_boundaries *boundaries, const cdf_options *options,
                         cdf_lb **out);

/* Set the state at t = 0 from moments (host, FP64): phi [m][ny][nx],
 * u [2][ny][nx], p [ny][nx] or NULL (p = 0).  Populations are f = f^eq(phi, u)
 * (Eq. feq-phi), h = h^eq(u, p) - F_i / 2 (Eq. heq, Eq. force) so that the
 * moments of Eqs. sum-phi/u/p return the inputs; S(t-1) = S(phi). */
cdf_status cdf_lb_init_moments(cdf_lb *h, const double *phi, const double *u, const double *p);

/* As cdf_lb_init_moments from a device FP32 stack [m+3][ny][nx]
 * (phi..., u_x, u_y, p), contiguous, on the handle's device. */
cdf_status cdf_lb_init_moments_device(cdf_lb *h, const float *dev_fields);

/* Advance n >= 0 time steps of Eqs. evolution12 and evolution3 with streaming
 * and the boundary rules, one fused kernel per step (CUDA-graph launched). */
cdf_status cdf_lb_step(cdf_lb *h, long long n);

/* Step until the relative change of every field q in {phi_0..phi_{m-1}, u_x,
 * u_y} over `check_every` steps, R = max_q sum|q(t) - q(t - K)| / sum|q(t)|,
 * summed in FP64, is below tol (the stop test of Sec. 3.1.1 with absolute
 * differences).  Returns CDF_ENOTCONVERGED after max_steps more steps,
 * CDF_EUNSTABLE on a NaN/Inf.  steps_taken and residual may be NULL. */
cdf_status cdf_lb_run_to_steady(cdf_lb *h, double tol, long long check_every, long long max_steps,
                                long long *steps_taken, double *residual);

/* Moments at the current time (Eqs. sum-phi, sum-u, sum-p) into a host FP64
 * stack [m+3][ny][nx]. */
cdf_status cdf_lb_moments(cdf_lb *h, double *host_out);

/* Same into a device FP32 stack [m+3][ny][nx], contiguous. */
cdf_status cdf_lb_moments_device(cdf_lb *h, float *dev_out);

/* Total of each scalar over the lattice, sum_x phi_a(x), accumulated in FP64 on
 * the device (mass check of Eq. CDE). sums has m entries (host). */
cdf_status cdf_lb_mass(cdf_lb *h, double *sums);

/* Heat and mass transfer through a wall of the double-diffusive cavity (Sec. 3.2,
 * the local Nusselt and Sherwood numbers and their averages over the wall), with
 * T = phi_0 and C = phi_1 of the current moments and lengths scaled by the lattice
 * width (dx = 1 / nx).  The wall derivative is the second-order one-sided (upwind)
 * difference through the wall value and the first two nodes, which sit half a
 * spacing and one and a half spacings from the half-way wall:
 * q'(wall) = (9 q_1 - q_2 - 8 q_wall) / (3 dx), taken along +x on either wall.
 * out[0] = mean_y Nu(y) = -mean_y (dT/dx + D_CT dC/dx), out[1] = mean_y Sh(y) =
 * -mean_y (S_TC dT/dx + dC/dx): the flux in +x (out of a hot west wall, into a
 * cold east wall; the paper prints the derivatives without the sign).  side: 0 west,
 * 1 east; T_wall, C_wall: that wall's values.  FP64 sums on the device; out has 2
 * host doubles.  Needs m >= 2 and nx >= 2. */
cdf_status cdf_lb_wall_transfer(cdf_lb *h, int side, double D_CT, double S_TC, double T_wall, double C_wall,
                                double *out);

/* Post-collision populations of the current time as FP64 on the host:
 * f [m][5][ny][nx] (D2Q5 order of Eq. D2Q5), hf [9][ny][nx] (Eq. D2Q9 order),
 * s_now [m][ny][nx] = S(phi) of the current time (zeros unless CONSUMPTION).
 * Any pointer may be NULL. */
cdf_status cdf_lb_populations(cdf_lb *h, double *f, double *hf, double *s_now);

/* Write / read the full state (populations, S(t-1), time, moments) to a file;
 * a restart continues bit-identically.  load checks that the file matches the
 * handle's grid, m, storage and reference state (CDF_EINVAL otherwise, CDF_EIO
 * on file errors). */
cdf_status cdf_lb_save(cdf_lb *h, const char *path);
cdf_status cdf_lb_load(cdf_lb *h, const char *path);

cdf_status cdf_lb_get_info(const cdf_lb *h, cdf_info *out);

/* The library's internal CUDA stream of the handle (cudaStream_t) on which the
 * step kernels run; for timing with events.  Borrowed, do not destroy. */
void *cdf_lb_stream(const cdf_lb *h);

/* ---- split lattice (slabs along y) ---------------------------------------------
 * The update of a node reads only the previous step's post-collision populations
 * of its nearest neighbours (Eqs. evolution12 and evolution3 with streaming,
 * Sec. 2), so a lattice cut into slabs of whole rows advances exactly like the
 * whole lattice when, before every step, each slab's halo row holds the
 * populations that cross the cut from its neighbour: per node of the cut, the
 * three D2Q9 and the m D2Q5 populations whose velocity points across it.  Every
 * node then computes the same bits as in the whole lattice.  One process per GPU
 * runs one slab (a cdf_lb created with options.halo_rows) and moves those rows
 * with its collective library; cdf_split runs all the slabs on one device.
 *
 * cdf_lb_halo_pack copies the crossing populations of the slab's boundary row on
 * `side` (0 = south, the first updated row; 1 = north, the last) into dev_buf,
 * a device FP32 array [3 + m][nx]: the rows of h_4, h_7, h_8, f_{a,4} (south) or
 * h_2, h_5, h_6, f_{a,2} (north).  cdf_lb_halo_unpack writes such an array, packed
 * by the neighbour on that side, into the slab's halo row.  Both act on the
 * current populations (after the last step), on the handle's stream order, and
 * return CDF_EINVAL when the slab has no halo row on `side`.
 *
 * cdf_lb_snapshot keeps a copy of the current moments; cdf_lb_change_sums then
 * gives the FP64 sums of the stop test over the slab's updated rows (3m + 5
 * values, laid out as in cdf_moment_sums_static): summed over the slabs, they
 * give the stop test of the whole lattice. */
cdf_status cdf_lb_halo_pack(cdf_lb *h, int side, float *dev_buf);
cdf_status cdf_lb_halo_unpack(cdf_lb *h, int side, const float *dev_buf);
cdf_status cdf_lb_snapshot(cdf_lb *h);
cdf_status cdf_lb_change_sums(cdf_lb *h, double *sums);

/* A lattice split into `nslabs` slabs of nearly equal row counts, all on the
 * current device, advanced with a halo exchange (pack, device copy, unpack)
 * after every step: the single-device form of the one-slab-per-GPU decomposition.
 * Arguments as cdf_lb_create (the whole lattice's grid, parameters and
 * boundaries); the options apply to every slab (FP32 storage; halo_rows,
 * origin_y and ny_global must be 0: the split sets them).  2 <= nslabs <= ny
 * (ny >= 2 nslabs on a periodic y axis).  The results equal the whole lattice's
 * bit for bit. */
typedef struct cdf_split cdf_split;
cdf_status cdf_split_create(const cdf_grid *grid, int m, const cdf_diffusion *diffusion, double nu,
                            const cdf_source *source, const cdf_force *force, const cdf_boundaries *boundaries,
                            const cdf_options *options, int nslabs, cdf_split **out);
/* Initial state of the whole lattice from host FP64 moments (as cdf_lb_init_moments). */
cdf_status cdf_split_init_moments(cdf_split *s, const double *phi, const double *u, const double *p);
/* n steps of every slab, with the halo exchange after each. */
cdf_status cdf_split_step(cdf_split *s, long long n);
/* Moments of the whole lattice, [m+3][ny][nx] host FP64. */
cdf_status cdf_split_moments(cdf_split *s, double *host_out);
/* Scalar totals: each slab's FP64 sums (cdf_lb_mass), added in slab order. */
cdf_status cdf_split_mass(cdf_split *s, double *sums);
/* The stop test of cdf_lb_run_to_steady on the whole lattice, from the slabs'
 * change sums added together. */
cdf_status cdf_split_run_to_steady(cdf_split *s, double tol, long long check_every, long long max_steps,
                                   long long *steps_taken, double *residual);
/* Slab k: its handle (borrowed), the first row of the whole lattice it updates
 * and the number of rows it updates. */
cdf_status cdf_split_slab(const cdf_split *s, int k, cdf_lb **slab, int *y0, int *rows);
void cdf_split_destroy(cdf_split *s);

/* ---- batched solver --------------------------------------------------------
 * Many independent lattices of uneven size (a parameter sweep) advanced together,
 * in one of two modes chosen by measurement: a persistent kernel that schedules
 * (instance, tile) units with a bounded grid barrier between the time steps of
 * a launch, or one CUDA graph of per-instance chains of step kernels fanned out
 * over a stream pool (the instances are independent, so the chains need no
 * barrier).  Each instance
 * is the model of cdf_lb_create (same equations, same boundary rules) with its
 * own grid, D, nu, S, F and boundaries; all share m, the source kind and FP32
 * population storage. */
typedef struct cdf_batch cdf_batch;
typedef struct {
    int storage;                 /* CDF_FP32 (the only mode of the batched solver) */
    double rho0;
    void *cuda_stream;           /* caller's stream, NULL = legacy default */
    int tile_x, tile_y;          /* tile shape (nodes); 0 = autotuned */
    int steps_per_launch;        /* time steps per persistent launch; 0 = 32 */
    double barrier_timeout_s;    /* bound of every grid-barrier wait; 0 = 1 s */
    int test_unreachable_barrier;/* test hook: the barrier expects one block more than runs,
                                    so every wait runs out and cdf_batch_step returns CDF_ETIMEOUT */
    int mode;                    /* with tile_x > 0: 0 = persistent kernel (tile = tile shape),
                                    1 = graph of per-instance kernel chains (tile = CTA shape),
                                    2 = the same chains of two-step launches (step2_kernel of
                                    cdf_options.temporal; tile = its CTA shape, tile_x 32 or 64);
                                    with tile_x = 0 the autotuner measures all three and picks */
    int chain_tile_y;            /* mode 2 with tile_x > 0: output tile height of the two-step
                                    kernel (0 = 14) */
    int chain_lanes;             /* mode 2 with tile_x > 0: nodes per thread of the two-step
                                    kernel (2: the paired-lane kernel of cdf_options.temporal_lanes,
                                    tile 32 x 8, chain_tile_y 14 or 30; 0 or 1: one) */
} cdf_batch_options;
typedef struct {
    int count, m;
    long long nodes, tiles;
    int tile_x, tile_y, grid_blocks, steps_per_launch;
    double bytes_per_lup;
    long long t;
    int mode;                    /* 0 persistent kernel, 1 graph of per-instance chains,
                                    2 chains of two-step launches */
    int chain_block_x, chain_block_y;
    int chain_tile_y;            /* mode 2: output tile height of the two-step kernel */
    int chain_lanes;             /* modes 1, 2: nodes per thread of the chains' kernel (1 or 2) */
} cdf_batch_info;

/* Create `count` lattices; every array argument has `count` entries (phi_ref:
 * count x m, p_ref_grad: count x 2, the references of cdf_options per instance).
 * Checks each instance like cdf_lb_create. */
cdf_status cdf_batch_create(int count, const cdf_grid *grids, int m, const cdf_diffusion *diffusion, const double *nu,
                            const cdf_source *source, const cdf_force *force, const cdf_boundaries *boundaries,
                            const double *phi_ref, const double *p_ref_grad, const cdf_batch_options *options,
                            cdf_batch **out);
/* Initial state of instance k from host FP64 moments (as cdf_lb_init_moments). */
cdf_status cdf_batch_init_moments(cdf_batch *b, int k, const double *phi, const double *u, const double *p);
/* Advance every instance by n steps (Eqs. evolution12, evolution3).  Returns
 * CDF_ETIMEOUT if a grid-barrier wait ran out (state then undefined). */
cdf_status cdf_batch_step(cdf_batch *b, long long n);
/* Moments of instance k at the current time into a host FP64 stack [m+3][ny][nx]. */
cdf_status cdf_batch_moments(cdf_batch *b, int k, double *host_out);
/* Device forms of the two calls above, without host staging or conversion:
 * instance k from / into a device FP32 stack [m+3][ny][nx] (phi_0..phi_{m-1}, u_x,
 * u_y, p; the layout of cdf_lb_init_moments_device), or, for k = -1, every
 * instance from / into one buffer of such stacks back to back in instance order
 * (instance k at float offset sum_{j<k} (m+3) nx_j ny_j).  Ordered on the batch's
 * stream and returning after the launches (the buffer may be reused once that
 * stream has reached this call); CDF_EINVAL for a NULL pointer or k outside
 * [-1, count). */
cdf_status cdf_batch_init_moments_device(cdf_batch *b, int k, const float *dev_fields);
cdf_status cdf_batch_moments_device(cdf_batch *b, int k, float *dev_out);
/* Keep a copy of every instance's current moments; cdf_batch_residuals then gives,
 * per instance, the stop-test residual R of cdf_lb_run_to_steady between that copy
 * and the current moments (FP64 sums; +Inf where a field is not finite).
 * residual has `count` entries (host). */
cdf_status cdf_batch_snapshot(cdf_batch *b);
cdf_status cdf_batch_residuals(cdf_batch *b, double *residual);
cdf_status cdf_batch_get_info(const cdf_batch *b, cdf_batch_info *out);
void *cdf_batch_stream(const cdf_batch *b);
void cdf_batch_destroy(cdf_batch *b);

/* Allocation-free FP64 sums over a device moment stack -- the reduction behind
 * cdf_lb_mass and the stop test of cdf_lb_run_to_steady, for callers that
 * cannot allocate device memory once running (real-time loops that forbid
 * allocation after start-up, plug-ins inside a host application that owns all
 * device memory through its own pool, processes under a fixed device-memory
 * quota).  The paper has no counterpart: it is a systems addition.
 *   dev_fields      device FP32 stack [m+3][ny][nx] (phi..., u_x, u_y, p), contiguous,
 *                   e.g. filled by cdf_lb_moments_device
 *   dev_fields_old  same layout, or NULL
 *   dev_out         device FP64 array of 3m + 5 entries, written on `stream`:
 *                   [0, m) sum phi_a; [m, 2m+2) sum |q - q_old| (0 without old);
 *                   [2m+2, 3m+4) sum |q| for q in {phi_0..phi_{m-1}, u_x, u_y};
 *                   [3m+4] number of non-finite values
 *   stream          cudaStream_t, NULL = legacy default stream
 * Allocates nothing: the block partials live in a file-scope device array of
 * 41,344 bytes (304 blocks x 17 sums) that every GPU loading the library holds
 * until exit.  Limits: 1 <= m <= 4, nx * ny < 2^31, current device index < 64
 * (CDF_EINVAL beyond).  The first call on each device -- and the first call after
 * that device's context was torn down and recreated (cudaDeviceReset) -- does a
 * set-up with that device current: it looks up the array's device address
 * (cudaGetSymbolAddress) and loads the reduction kernels' code, which under lazy
 * module loading may allocate.  Make that first call at start-up, before the
 * phase that must not allocate and before any stream capture.  All calls share
 * the array: calls that overlap on the GPU race.  Returns after launching;
 * dev_out is ready when `stream` is. */
cdf_status cdf_moment_sums_static(const float *dev_fields, const float *dev_fields_old, int nx, int ny, int m,
                                  double *dev_out, void *stream);

/* Release the handle and its device memory (NULL is a no-op). */
void cdf_lb_destroy(cdf_lb *h);

/* Message of the calling thread's last error ("" if none).  Valid until the
 * thread's next call into the library. */
const char *cdf_lb_last_error(void);

/* ---- checks build --------------------------------------------------------------
 * The library can be built a second time with -DCDF_CHECKS (libcdflb_checks.so)
 * for tests; it computes the same bits as the normal build.  Its step kernels
 * (2-D single lattice, one and two steps per launch, FP32 and 16-bit storage,
 * Case 1, the tile-resident and the batched persistent step) test every
 * population, moment and shared-memory offset against its buffer before the
 * access; an offset outside is recorded (first one wins) and replaced by an
 * in-range one, so the launch completes and never leaves its buffers.  Every
 * device buffer of a lattice and of a batch lies between two 64 KiB canary pads.
 * cdf_lb_step, cdf_lb_run_to_steady and cdf_batch_step wait for their stream and
 * return CDF_ECHECK (message: the access site and offset, or the damaged pad)
 * when either detector fired. */

/* 1 in a checks build, 0 in a normal one. */
int cdf_checks_enabled(void);

/* Self-test of a checks build's detectors (CDF_EINVAL in a normal build):
 *   which = 0: one kernel on a 64-float buffer asks for offsets 64..95 through the
 *              offset check (it reads and writes offset 0 instead);
 *   which = 1: the host writes one byte of the pad behind a 256-byte buffer.
 * Returns CDF_ECHECK when the detector caught it (the expected result), CDF_OK
 * when it did not; the detector's state is reset either way. */
cdf_status cdf_checks_selftest(int which);

#ifdef __cplusplus
}
#endif
#endif /* CDF_LB_H */
