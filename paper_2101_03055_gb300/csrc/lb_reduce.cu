// FP64 reductions over moment fields: scalar totals (mass check) and the
// steady-state residual sums of the stop test (Sec. 3.1.1), accumulated in
// FP64 from FP32 fields.  Two passes with a fixed order (per-thread grid-stride
// sums, warp shuffles, a block tree, then one block over the block partials),
// so the result is bit-reproducible from run to run.
#include "lb_internal.h"

namespace cdflb {

int reduce_quantities(int m) { return 3 * m + 5; }

namespace {

constexpr int kThreads = 256;
constexpr int kMaxQ = 3 * kMaxM + 5;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-level sum of NQ per-thread values; thread 0 gets the totals in acc.
template <int NQ>
__device__ void block_sum(double (&acc)[NQ]) {
    __shared__ double red[kThreads / 32][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double v = warp_sum(acc[q]);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double v = lane < kThreads / 32 ? red[lane][q] : 0.0;
            acc[q] = warp_sum(v);
        }
    }
}

template <int M>
__global__ void __launch_bounds__(kThreads) partial_kernel(const float *__restrict__ nw,
                                                           const float *__restrict__ od, int nx, int ny,
                                                           int pitch, long long plane,
                                                           double *__restrict__ partials) {
    constexpr int NQ = 3 * M + 5;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    const long long n = (long long)nx * ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long y = idx / nx, x = idx - y * nx, o = y * pitch + x;
#pragma unroll
        for (int q = 0; q < M + 2; ++q) {
            const float v = nw[q * plane + o];
            if (q < M) acc[q] += (double)v;
            if (od) acc[M + q] += fabs((double)v - (double)od[q * plane + o]);
            acc[2 * M + 2 + q] += fabs((double)v);
            if (!isfinite(v)) acc[3 * M + 4] += 1.0;
        }
        if (!isfinite(nw[(M + 2) * plane + o])) acc[3 * M + 4] += 1.0;
    }
    block_sum<NQ>(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) partials[(long long)q * gridDim.x + blockIdx.x] = acc[q];
}

template <int M>
__global__ void __launch_bounds__(kThreads) final_kernel(const double *__restrict__ partials, int nblocks,
                                                         double *__restrict__ out) {
    constexpr int NQ = 3 * M + 5;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(long long)q * nblocks + b];
        acc[q] = v;
    }
    block_sum<NQ>(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] = acc[q];
}

template <int M>
cudaError_t run(const float *nw, const float *od, int nx, int ny, int pitch, long long plane,
                double *partials, double *out, cudaStream_t s) {
    partial_kernel<M><<<kReduceBlocks, kThreads, 0, s>>>(nw, od, nx, ny, pitch, plane, partials);
    final_kernel<M><<<1, kThreads, 0, s>>>(partials, kReduceBlocks, out);
    return cudaGetLastError();
}

}  // namespace

// Wall heat and mass transfer of the double-diffusive cavity (Sec. 3.2): per row y
// the x-derivative of T = phi_0 and C = phi_1 at the wall by the one-sided quadratic
// through the wall value and the first two nodes (half a spacing and one and a half
// spacings from the half-way wall), q'(wall) = (9 q_1 - q_2 - 8 q_w) / (3 dx) with dx
// = 1 / nx (lengths scaled by the cavity width), taken in +x on either wall; then
// Nu(y) = -(dT/dx + D_CT dC/dx), Sh(y) = -(S_TC dT/dx + dC/dx) (the flux in +x: out of
// the hot west wall, into the cold east wall) and their row means, in FP64 with a
// fixed summation order (one block, a strided run of rows per thread, a tree).
__global__ void __launch_bounds__(kThreads) wall_transfer_kernel(const float *__restrict__ mom, int nx, int ny,
                                                                 int pitch, long long plane, int east, double D_CT,
                                                                 double S_TC, double T_wall, double C_wall,
                                                                 double *__restrict__ out) {
    double acc[2] = {0.0, 0.0};
    const double dx = 1.0 / nx;
    for (int y = threadIdx.x; y < ny; y += blockDim.x) {
        const long long r = (long long)y * pitch;
        const int i1 = east ? nx - 1 : 0, i2 = east ? nx - 2 : 1;
        const double sgn = east ? -1.0 : 1.0;  // d/dx of the quadratic, pointing in +x
        const double T1 = mom[r + i1], T2 = mom[r + i2], C1 = mom[plane + r + i1], C2 = mom[plane + r + i2];
        const double dT = sgn * (9.0 * T1 - T2 - 8.0 * T_wall) / (3.0 * dx);
        const double dC = sgn * (9.0 * C1 - C2 - 8.0 * C_wall) / (3.0 * dx);
        acc[0] += -(dT + D_CT * dC);
        acc[1] += -(S_TC * dT + dC);
    }
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
        out[0] = acc[0] / ny;
        out[1] = acc[1] / ny;
    }
}

cudaError_t launch_wall_transfer(const float *mom, int nx, int ny, int pitch, long long plane, int east, double D_CT,
                                 double S_TC, double T_wall, double C_wall, double *out, cudaStream_t s) {
    wall_transfer_kernel<<<1, kThreads, 0, s>>>(mom, nx, ny, pitch, plane, east, D_CT, S_TC, T_wall, C_wall, out);
    return cudaGetLastError();
}

cudaError_t preload_reduce_kernels() {
    // cudaFuncGetAttributes makes the runtime load each kernel's code now (under
    // lazy module loading it would otherwise load, and may allocate, at the first
    // launch)
    cudaFuncAttributes a;
    const void *fns[] = {(const void *)partial_kernel<1>, (const void *)partial_kernel<2>,
                         (const void *)partial_kernel<3>, (const void *)partial_kernel<4>,
                         (const void *)final_kernel<1>,   (const void *)final_kernel<2>,
                         (const void *)final_kernel<3>,   (const void *)final_kernel<4>};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_reduce(const float *mom_new, const float *mom_old, int nx, int ny, int pitch,
                          long long plane, int m, double *partials, double *out, cudaStream_t s) {
    static_assert(kMaxQ == 17, "reduction slots");
    switch (m) {
        case 1: return run<1>(mom_new, mom_old, nx, ny, pitch, plane, partials, out, s);
        case 2: return run<2>(mom_new, mom_old, nx, ny, pitch, plane, partials, out, s);
        case 3: return run<3>(mom_new, mom_old, nx, ny, pitch, plane, partials, out, s);
        case 4: return run<4>(mom_new, mom_old, nx, ny, pitch, plane, partials, out, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cdflb
