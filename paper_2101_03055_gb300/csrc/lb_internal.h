// Internal declarations shared by the host runtime and the kernel translation
// units of libcdflb (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cdf_lb.h"

namespace cdflb {

constexpr int kMaxM = 4;

// Everything a step / init kernel needs besides its buffers; passed by value.
// All coefficients are in lattice units and already scaled for the kernels.
struct LbParams {
    int nx, ny, pitch;          // lattice size, elements per stored row
    long long plane;            // elements per plane (pitch * ny)
    int m;
    // Relaxation (Eq. omega-D).  For constant D: omega itself.  For the
    // chemotaxis closure: the inverse of the constant part B = D/cs^2 + I/2;
    // the node value follows by a rank-one update (Sherman-Morrison).
    float omega[kMaxM * kMaxM];
    float omega_f;              // fluid relaxation, 1 / (3 nu + 1/2)
    int chemotaxis;             // D_01 += -chi phi_0 r(phi_1)
    float chi3;                 // 3 chi (the 1/cs^2 of Eq. omega-D folded in)
    float c_star, eps2;         // cut-off and regularisation width squared
    int r_regularised;
    int skind;                  // 0 none, 1 const, 2 consumption (S_1 = -k phi_0 r)
    float S[kMaxM];
    float k;
    float g[2];                 // F = g (Fbase + sum_a beta_a phi_a)
    float beta[kMaxM];
    float Fbase;
    // Eq. force's second-order part (varphi != 0): varphi itself and the pressure
    // correction's coefficient varphi (1/omega_f - 1/2) W_0 / cs^2
    float varphi, varphi_p;
    float rho0;
    int periodic_x, periodic_y;
    int freeslip[4];            // per side (west, east, south, north)
    unsigned dirichlet[4];      // per side: bit a set -> scalar a is Dirichlet
    float abb[4][kMaxM];        // per side and scalar: 2 W_i (phi_w - phi_ref) = (phi_w - phi_ref) / 3
    // Reference state of the stored deviations: W_i phi_ref_a for scalar a;
    // h^eq(p_ref(x), 0) for the fluid with p_ref(x) = gref . (x - (xc, yc)).
    float phi_ref[kMaxM];
    float gref[2];
    float xc, yc;
    // Case 1 of Sec. 2.1 (no fluid populations): planes of the prescribed
    // velocity u_x, u_y (`vel`), and the m planes of phi_a(t - 1) a step reads
    // (`php_in`) and the m planes of phi_a(t) it writes (`php_out`), `plane`
    // floats each (device memory).  The two phi sets alternate with the
    // population buffers.
    int case1;
    float *vel;
    const float *php_in;
    float *php_out;
    // Rows the step updates, row_lo <= y < row_hi: all of them, except on a slab
    // of a split lattice, whose halo rows (y = 0 and/or y = ny - 1) hold the
    // neighbouring slab's post-collision populations and are written by the halo
    // exchange instead.
    int row_lo, row_hi;
    // Checks builds (-DCDF_CHECKS): the device word that records the first
    // out-of-range offset a step kernel met (see CDF_CHK in lb_device.cuh);
    // unused (nullptr) in a normal build.
    unsigned long long *check;
};

enum Storage { kFP32 = 0, kFP16 = 1, kBF16 = 2 };

// The population planes of a step, one pointer per plane, passed to the step
// kernels as a parameter: a plane's address is then an operand from the
// constant bank instead of a 64-bit multiply-add per access.
constexpr int kMaxPlanes = 9 + 5 * kMaxM;
template <typename T>
struct Planes {
    const T *in[kMaxPlanes];
    T *out[kMaxPlanes];
};
// The FP32 moment planes (phi_0 .. phi_{m-1}, u_x, u_y, p) that 16-bit storage
// keeps beside its populations, read (`in`) and written (`out`), one pointer each.
struct MomentPlanes {
    const float *in[kMaxM + 3];
    float *out[kMaxM + 3];
};

// Launchers (lb_kernels.cu), FP32 storage (16-bit storage has the _mr
// launchers below).  A step launch with block.y == 0 is flat: block.x
// threads per CTA over the nx * ny nodes in row order (FP32 storage path).  `in`/`out` point at the first of `planes`
// population planes; plane k starts at base + k * plane.  Planes are ordered
// h_0..h_8, then f_{a,0..4} for a = 0..m-1.
cudaError_t launch_step(const LbParams &p, int storage, const void *in, void *out, const float *sp_in,
                        float *sp_out, float *moments, dim3 block, cudaStream_t s);
// Two time steps in one launch (FP32 storage): block.x (32 or 64) x block.y
// threads per CTA, output tiles of (block.x - 2) x th nodes; sp_in and sp_out
// must be different planes.  step2_smem_bytes: its dynamic shared memory.
constexpr int kStep2MaxSmem = 227 * 1024;
// CTA size bound of step2_kernel: 64 registers a thread (1024 threads) hold the
// node update for m <= 2 without spills; m = 3, 4 need 128 (512 threads).
constexpr int step2_max_threads(int m) { return m <= 2 ? 1024 : 512; }
// The 16-bit form (step2_kernel_mr) also rebuilds the populations from stored
// deviations and moments: CTAs of at most 256 threads, three of them per SM for
// m <= 2 (80 registers a thread; measured 8 % faster at 4096^2 than two CTAs of
// 512 threads with 116 registers).
constexpr int step2_mr_max_threads(int) { return 256; }
size_t step2_smem_bytes(int m, dim3 block, int th);
cudaError_t launch_step2(const LbParams &p, const float *in, float *out, const float *sp_in, float *sp_out,
                         float *moments, dim3 block, int th, cudaStream_t s);
cudaError_t launch_init(const LbParams &p, int storage, const float *fields, int fields_pitch,
                        void *out, float *sprev, float *moments, cudaStream_t s);
cudaError_t launch_export(const LbParams &p, int storage, const void *in, float *dense,
                          cudaStream_t s);
// 16-bit storage (FP16/BF16): populations stored as deviations from each node's
// own equilibrium, with the node's moments (phi, u, p) in FP32 (m + 3 planes);
// moments are ping-ponged with the populations.
cudaError_t launch_step_mr(const LbParams &p, int storage, const void *in, const float *moments_in, void *out,
                           float *moments_out, const float *sp_in, float *sp_out, dim3 block, cudaStream_t s);
// Two steps per launch with 16-bit storage (tiling of launch_step2; the
// intermediate step stays in FP32 in shared memory).
cudaError_t launch_step2_mr(const LbParams &p, int storage, const void *in, const float *moments_in, void *out,
                            float *moments_out, const float *sp_in, float *sp_out, dim3 block, int th,
                            cudaStream_t s);
cudaError_t launch_init_mr(const LbParams &p, int storage, const float *fields, int fields_pitch, void *out,
                           float *moments_out, float *sprev, cudaStream_t s);
cudaError_t launch_export_mr(const LbParams &p, int storage, const void *in, const float *moments, float *dense,
                             cudaStream_t s);
cudaError_t launch_pack_moments(const LbParams &p, const float *moments, float *dense,
                                cudaStream_t s);

// Tile-resident persistent step (lb_resident.cu), FP32 storage.  The lattice
// is cut into tiles_x x tiles_y tiles of tw x th nodes (the last row and column
// of tiles may be smaller), one co-resident CTA of `threads` threads and
// `smem_bytes` of dynamic shared memory per tile.  stall_tile >= 0 is a test
// hook: that tile never publishes its step counter, so its neighbours' bounded
// waits run out.
struct ResidentGeom {
    int tiles_x, tiles_y, tw, th;
    int threads;
    size_t smem_bytes;
    int stall_tile;
};
// Finds a tiling of the nx x ny lattice with m scalars that fits one CTA per
// SM of the current device; false if the lattice is too large (or the device
// lacks the shared memory).
bool plan_resident(int nx, int ny, int m, ResidentGeom *out);
// nsteps steps from buffer parity0 (buf0 or buf1) in one cooperative launch;
// `counters` holds one step counter per tile (all equal between launches;
// zero them together), *err is set when a wait ran out.
cudaError_t launch_resident(const LbParams &p, const ResidentGeom &g, float *buf0, float *buf1, const float *sp_in,
                            float *sprev,
                            float *moments, int nsteps, int parity0, bool moments_last, unsigned *counters,
                            unsigned long long timeout_ns, int *err, cudaStream_t s);

// FP64 reductions (lb_reduce.cu).  Over `fields` stacks of (m+3) planes with the
// given pitch: out[0..m) = sum phi_a; out[m + q] = sum |q_new - q_old| and
// out[2m + 2 + q] = sum |q_new| for q in {phi_0..phi_{m-1}, u_x, u_y};
// out[3m + 4] = count of non-finite values in the first m + 3 planes.
constexpr int kReduceBlocks = 304;  // 2 x 152 SMs
int reduce_quantities(int m);
cudaError_t launch_reduce(const float *mom_new, const float *mom_old, int nx, int ny, int pitch,
                          long long plane, int m, double *partials, double *out, cudaStream_t s);
// Average Nusselt and Sherwood numbers on the west (east = 0) or east wall of a
// moment stack (T = plane 0, C = plane 1), FP64, into out[0..1] (device).
cudaError_t launch_wall_transfer(const float *mom, int nx, int ny, int pitch, long long plane, int east, double D_CT,
                                 double S_TC, double T_wall, double C_wall, double *out, cudaStream_t s);
// Loads the code of every reduction kernel on the current device now instead of
// at its first launch.
cudaError_t preload_reduce_kernels();

// Checks one lattice's parameter set and fills the kernel parameters.
cdf_status build_params(const cdf_grid *grid, int m, const cdf_diffusion *dif, double nu, const cdf_source *src,
                        const cdf_force *frc, const cdf_boundaries *bc, bool node_reference, double rho0,
                        const double *phi_ref, const double *p_ref_grad, int pitch, LbParams *out);

// Sets the calling thread's cdf_lb_last_error() message and returns `status`.
cdf_status report_error(cdf_status status, const char *msg);

// ---- checks builds (lb_checks.cu) ----------------------------------------------
// A library built with -DCDF_CHECKS tests the offsets of the step kernels'
// accesses before it makes them (CDF_CHK) and surrounds every device buffer of
// a lattice with canary pads.  dev_alloc / dev_free are cudaMalloc / cudaFree
// in a normal build; there check_word() is nullptr and checks_verify returns
// CDF_OK without touching the stream.  In a checks build checks_verify waits for
// the stream, then returns CDF_ECHECK (and resets what it found) when the word
// holds an offset or a pad of a live buffer lost its pattern.
unsigned long long *check_word();
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
#ifdef CDF_CHECKS
cdf_status checks_verify(cudaStream_t s);
#else
inline cdf_status checks_verify(cudaStream_t) { return CDF_OK; }
#endif

}  // namespace cdflb
