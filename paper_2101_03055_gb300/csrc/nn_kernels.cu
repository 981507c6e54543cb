// BF16 kernels of the convolutional surrogate that warm-starts the steady
// solve: 3x3 convolutions as implicit GEMMs on the tensor cores (BF16 operands,
// FP32 accumulation), their two backward passes, and the small layers around
// them (bias + ReLU epilogue, 2x2 average pooling, nearest 2x upsampling,
// channel copies for skip connections, 1x1 output head, MSE loss, Adam).
// Activations are NHWC with the channel count a multiple of 16; 3x3 weights
// are [Cout][3][3][Cin].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <algorithm>
#include <cstdint>

#include "../../include/cdf_nn.h"

using namespace nvcuda;

namespace {

constexpr int kBM = 64;      // pixels per CTA tile (forward / backward-data)
constexpr int kThreads = 128;
constexpr int kLdA = 24;     // padded leading dimensions of the shared tiles (bf16 elements)

// ---------------------------------------------------------------------------
// 3x3 convolution as an implicit GEMM.
//   forward:       Y[p][co] = act(sum_{t, ci} X[p + d(t)][ci] W[co][t][ci] + b[co])
//   backward data: dX[p][ci] = sum_{t, co} dY[p + d(t)][co] W[co][8 - t][ci]
// with d(t) = (ky - 1, kx - 1) for tap t = 3 ky + kx and zero outside the image.
// GEMM: M = pixels (tile kBM), N = output channels (tile BN), K = 9 x input channels.
// ---------------------------------------------------------------------------
template <bool kBwdData, int BN>
__global__ void __launch_bounds__(kThreads) conv3x3_kernel(const __nv_bfloat16 *__restrict__ in,
                                                           const __nv_bfloat16 *__restrict__ w,
                                                           const float *__restrict__ bias,
                                                           __nv_bfloat16 *__restrict__ out, int N, int H, int Wd,
                                                           int Cin_g, int Cout_g, int relu) {
    // Cin_g / Cout_g: channels of the GEMM input / output (fwd: Cin / Cout; bwd: Cout / Cin).
    constexpr int kLdB = BN + 8;
    __shared__ __align__(32) __nv_bfloat16 As[kBM * kLdA];
    __shared__ __align__(32) __nv_bfloat16 Bs[16 * kLdB > BN * kLdA ? 16 * kLdB : BN * kLdA];
    __shared__ __align__(32) float Cs[kBM * (BN + 4)];
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long P = (long long)N * H * Wd;
    const long long p0 = (long long)blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    // The original weight tensor's channel counts: Cout_w x 9 x Cin_w.
    const int Cin_w = kBwdData ? Cout_g : Cin_g;

    // A-tile row handled by this thread: pixel p0 + tid / 2, 8 channels at (tid & 1) * 8.
    const int arow = tid >> 1, acol = (tid & 1) * 8;
    const long long pa = p0 + arow;
    int an = 0, ay = 0, ax = 0;
    if (pa < P) {
        an = (int)(pa / ((long long)H * Wd));
        const int rem = (int)(pa - (long long)an * H * Wd);
        ay = rem / Wd;
        ax = rem - ay * Wd;
    }

    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[BN / 16];
#pragma unroll
    for (int j = 0; j < BN / 16; ++j) wmma::fill_fragment(acc[j], 0.f);

    const int K = 9 * Cin_g;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int tap = k0 / Cin_g, c0 = k0 - tap * Cin_g;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        // A tile: 16 input channels of the shifted pixels (zero outside the image).
        {
            uint4 v = make_uint4(0, 0, 0, 0);
            const int sy = ay + dy, sx = ax + dx;
            if (pa < P && sy >= 0 && sy < H && sx >= 0 && sx < Wd)
                v = *reinterpret_cast<const uint4 *>(in + (((long long)an * H + sy) * Wd + sx) * Cin_g + c0 + acol);
            *reinterpret_cast<uint4 *>(As + arow * kLdA + acol) = v;
        }
        // B tile: 16 (k) x BN (n) weights.
        if (!kBwdData) {
            // B(k = ci, n = co) = W[co][tap][ci]: per output channel 16 contiguous ci (col-major).
            for (int e = tid; e < BN * 2; e += kThreads) {
                const int nn = e >> 1, half = (e & 1) * 8;
                const uint4 v = *reinterpret_cast<const uint4 *>(w + ((long long)(n0 + nn) * 9 + tap) * Cin_w + c0 + half);
                *reinterpret_cast<uint4 *>(Bs + nn * kLdA + half) = v;
            }
        } else {
            // B(k = co, n = ci) = W[co][8 - tap][ci]: per k a row of BN contiguous ci (row-major).
            for (int e = tid; e < 16 * (BN / 8); e += kThreads) {
                const int kk = e / (BN / 8), seg = (e % (BN / 8)) * 8;
                const uint4 v = *reinterpret_cast<const uint4 *>(
                    w + ((long long)(c0 + kk) * 9 + (8 - tap)) * Cin_w + n0 + seg);
                *reinterpret_cast<uint4 *>(Bs + kk * kLdB + seg) = v;
            }
        }
        __syncthreads();
        wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> a;
        wmma::load_matrix_sync(a, As + warp * 16 * kLdA, kLdA);
#pragma unroll
        for (int j = 0; j < BN / 16; ++j) {
            if (!kBwdData) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::col_major> b;
                wmma::load_matrix_sync(b, Bs + j * 16 * kLdA, kLdA);
                wmma::mma_sync(acc[j], a, b, acc[j]);
            } else {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
                wmma::load_matrix_sync(b, Bs + j * 16, kLdB);
                wmma::mma_sync(acc[j], a, b, acc[j]);
            }
        }
        __syncthreads();
    }
    // Epilogue: bias, ReLU, BF16, one 16-byte store per 8 channels.
#pragma unroll
    for (int j = 0; j < BN / 16; ++j)
        wmma::store_matrix_sync(Cs + warp * 16 * (BN + 4) + j * 16, acc[j], BN + 4, wmma::mem_row_major);
    __syncthreads();
    for (int e = tid; e < kBM * (BN / 8); e += kThreads) {
        const int r = e / (BN / 8), seg = (e % (BN / 8)) * 8;
        const long long p = p0 + r;
        if (p >= P) continue;
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float v = Cs[r * (BN + 4) + seg + q];
            if (bias) v += bias[n0 + seg + q];
            if (relu) v = fmaxf(v, 0.f);
            o[q] = __float2bfloat16_rn(v);
        }
        *reinterpret_cast<uint4 *>(out + p * Cout_g + n0 + seg) = *reinterpret_cast<const uint4 *>(o);
    }
}

// ---------------------------------------------------------------------------
// The same two convolutions on the 5th-generation tensor cores (tcgen05): one CTA
// of 128 threads owns 128 output pixels (one TMEM lane each) and BN output
// channels (BN TMEM columns of FP32 accumulators).  K = 9 x channels runs in
// stages of 64: all threads stage the im2col rows of A (128 x 64) and the
// weights B (BN x 64) in shared memory in the K-major core-matrix layout (8 rows
// x 16 bytes per 128-byte core matrix), one thread issues four
// tcgen05.mma.kind::f16 (M = 128, N = BN, K = 16) and commits them to an
// mbarrier; two stage buffers let the next stage load while the tensor core
// works.  The epilogue reads the accumulators with tcgen05.ld (warp w owns
// lanes 32w..32w+31), adds the bias, applies the ReLU and stores BF16.  Every
// mbarrier wait is bounded; on time-out the kernel sets g_tc_error and still
// frees its tensor memory.
// ---------------------------------------------------------------------------
constexpr int kTM = 128, kTK = 64, kTcThreads = 128;
__device__ int g_tc_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, K-major without swizzle: start address,
// leading byte offset (between the two core matrices along K of one MMA) and
// stride byte offset (between core matrices along M or N), all in 16-byte units;
// bit 46 is the descriptor version of this architecture.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator, BF16 A and B,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (r, k) of a rows x 64 stage tile in the core-matrix layout.
__device__ __forceinline__ uint32_t cm_offset(int r, int k, int rows) {
    return (uint32_t)((((k >> 3) * (rows >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < (1ll << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    atomicExch(&g_tc_error, 1);
    return false;
}

template <bool kBwdData, int BN>
__global__ void __launch_bounds__(kTcThreads) conv3x3_tc_kernel(const __nv_bfloat16 *__restrict__ in,
                                                                const __nv_bfloat16 *__restrict__ w,
                                                                const float *__restrict__ bias,
                                                                __nv_bfloat16 *__restrict__ out, int N, int H, int Wd,
                                                                int Cin_g, int Cout_g, int relu) {
    constexpr int kCols = BN < 32 ? 32 : BN;               // TMEM columns (power of two >= 32)
    constexpr uint32_t kABytes = kTM * kTK * 2, kBBytes = BN * kTK * 2;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char *A = tc_smem;                              // 2 x kABytes
    unsigned char *B = tc_smem + 2 * kABytes;                // 2 x kBBytes
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)N * H * Wd;
    const long long p0 = (long long)blockIdx.x * kTM;
    const int n0 = blockIdx.y * BN;
    const int Cin_w = kBwdData ? Cout_g : Cin_g;  // the weight tensor is Cout_w x 9 x Cin_w
    const int K = 9 * Cin_g, nst = (K + kTK - 1) / kTK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // the pixel of this thread's A row
    const long long pa = p0 + tid;
    int an = 0, ay = 0, ax = 0;
    if (pa < P) {
        an = (int)(pa / ((long long)H * Wd));
        const int rem = (int)(pa - (long long)an * H * Wd);
        ay = rem / Wd;
        ax = rem - ay * Wd;
    }
    constexpr uint32_t idesc = mma_idesc(kTM, BN);
    bool ok = true;
    int last = -1;  // last stage whose MMAs were committed
    for (int s = 0; s < nst && ok; ++s) {
        const int buf = s & 1;
        if (s >= 2) ok = mbar_wait(smem_u32(&mbar[buf]), (uint32_t)(((s - 2) >> 1) & 1));
        if (!ok) break;
        unsigned char *As = A + buf * kABytes, *Bs = B + buf * kBBytes;
        const int k0 = s * kTK;
        // A: row tid, eight 16-byte groups of 8 consecutive k (one tap, 8 channels each)
#pragma unroll
        for (int g = 0; g < kTK / 8; ++g) {
            const int k = k0 + 8 * g;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (pa < P && k < K) {
                const int tap = k / Cin_g, c = k - tap * Cin_g;
                const int sy = ay + tap / 3 - 1, sx = ax + tap % 3 - 1;
                if (sy >= 0 && sy < H && sx >= 0 && sx < Wd)
                    v = *reinterpret_cast<const uint4 *>(in + (((long long)an * H + sy) * Wd + sx) * Cin_g + c);
            }
            *reinterpret_cast<uint4 *>(As + cm_offset(tid, 8 * g, kTM)) = v;
        }
        // B: BN rows (output channels of the GEMM) x 64 k
        for (int e = tid; e < BN * (kTK / 8); e += kTcThreads) {
            const int nn = e / (kTK / 8), g = e % (kTK / 8);
            const int k = k0 + 8 * g;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (k < K) {
                const int tap = k / Cin_g, c = k - tap * Cin_g;
                if (!kBwdData) {
                    // B(k = (tap, ci), n = co) = W[co][tap][ci]: 8 contiguous ci
                    v = *reinterpret_cast<const uint4 *>(w + ((long long)(n0 + nn) * 9 + tap) * Cin_w + c);
                } else {
                    // B(k = (tap, co), n = ci) = W[co][8 - tap][ci]: 8 co with stride 9 Cin_w
                    __align__(16) __nv_bfloat16 t[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) t[q] = w[((long long)(c + q) * 9 + (8 - tap)) * Cin_w + n0 + nn];
                    v = *reinterpret_cast<const uint4 *>(t);
                }
            }
            *reinterpret_cast<uint4 *>(Bs + cm_offset(nn, 8 * g, BN)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int j = 0; j < kTK / 16; ++j) {
                // K slice j: core-matrix columns 2j and 2j + 1
                const uint64_t ad = smem_desc(a0 + 2 * j * (kTM / 8) * 128, (kTM / 8) * 128, 128);
                const uint64_t bd = smem_desc(b0 + 2 * j * (BN / 8) * 128, (BN / 8) * 128, 128);
                const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[buf]))
                         : "memory");
        }
        last = s;
    }
    // all MMAs done: the last commit tracks every earlier MMA of the issuing
    // thread (waited for also after a time-out, before the tensor memory is freed)
    if (last >= 0) ok = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1)) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const long long p = p0 + warp * 32 + lane;  // TMEM lane = tile row = pixel
#pragma unroll
        for (int c = 0; c < BN; c += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (p < P) {
                __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float v = __uint_as_float(r[q]);
                    if (bias) v += bias[n0 + c + q];
                    if (relu) v = fmaxf(v, 0.f);
                    o[q] = __float2bfloat16_rn(v);
                }
                *reinterpret_cast<uint4 *>(out + p * Cout_g + n0 + c) = *reinterpret_cast<const uint4 *>(o);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// ---------------------------------------------------------------------------
// The same convolution with its operand tiles copied by cp.async: three stage
// buffers, the copies of stage s + 2 in flight while the tensor core works on
// stage s.  Each thread copies its A row (8 x 16 bytes of the im2col row, zero
// fill outside the image: a copy of 0 source bytes writes zeros) and, for the
// forward pass, 16-byte runs of the weights straight into the K-major
// core-matrix layout; the backward-data weights are a gather of single elements
// and are staged with ordinary loads.  A buffer is refilled only after the MMAs
// that read it have completed (its mbarrier).  Same stage layout, descriptors,
// MMAs, bounded waits and epilogue as conv3x3_tc_kernel.
// ---------------------------------------------------------------------------
constexpr int kStages = 3;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <bool kBwdData, int BN>
__global__ void __launch_bounds__(kTcThreads) conv3x3_tc_pipe_kernel(const __nv_bfloat16 *__restrict__ in,
                                                                     const __nv_bfloat16 *__restrict__ w,
                                                                     const float *__restrict__ bias,
                                                                     __nv_bfloat16 *__restrict__ out, int N, int H,
                                                                     int Wd, int Cin_g, int Cout_g, int relu) {
    constexpr int kCols = BN < 32 ? 32 : BN;
    constexpr uint32_t kABytes = kTM * kTK * 2, kBBytes = BN * kTK * 2;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char *A = tc_smem;                    // kStages x kABytes
    unsigned char *B = tc_smem + kStages * kABytes;  // kStages x kBBytes
    __shared__ __align__(8) uint64_t mbar[kStages];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)N * H * Wd;
    const long long p0 = (long long)blockIdx.x * kTM;
    const int n0 = blockIdx.y * BN;
    const int Cin_w = kBwdData ? Cout_g : Cin_g;
    const int K = 9 * Cin_g, nst = (K + kTK - 1) / kTK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < kStages; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    const long long pa = p0 + tid;
    int an = 0, ay = 0, ax = 0;
    if (pa < P) {
        an = (int)(pa / ((long long)H * Wd));
        const int rem = (int)(pa - (long long)an * H * Wd);
        ay = rem / Wd;
        ax = rem - ay * Wd;
    }
    // copies of stage s into its buffer
    auto load_stage = [&](int s) {
        unsigned char *As = A + (s % kStages) * kABytes, *Bs = B + (s % kStages) * kBBytes;
        const int k0 = s * kTK;
#pragma unroll
        for (int g = 0; g < kTK / 8; ++g) {
            const int k = k0 + 8 * g;
            const __nv_bfloat16 *src = in;
            int bytes = 0;
            if (pa < P && k < K) {
                const int tap = k / Cin_g, c = k - tap * Cin_g;
                const int sy = ay + tap / 3 - 1, sx = ax + tap % 3 - 1;
                if (sy >= 0 && sy < H && sx >= 0 && sx < Wd) {
                    src = in + (((long long)an * H + sy) * Wd + sx) * Cin_g + c;
                    bytes = 16;
                }
            }
            cp_async16(As + cm_offset(tid, 8 * g, kTM), src, bytes);
        }
        for (int e = tid; e < BN * (kTK / 8); e += kTcThreads) {
            const int nn = e / (kTK / 8), g = e % (kTK / 8);
            const int k = k0 + 8 * g;
            if (!kBwdData) {
                const __nv_bfloat16 *src = w;
                int bytes = 0;
                if (k < K) {
                    const int tap = k / Cin_g, c = k - tap * Cin_g;
                    src = w + ((long long)(n0 + nn) * 9 + tap) * Cin_w + c;
                    bytes = 16;
                }
                cp_async16(Bs + cm_offset(nn, 8 * g, BN), src, bytes);
            } else {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (k < K) {
                    const int tap = k / Cin_g, c = k - tap * Cin_g;
                    __align__(16) __nv_bfloat16 t[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) t[q] = w[((long long)(c + q) * 9 + (8 - tap)) * Cin_w + n0 + nn];
                    v = *reinterpret_cast<const uint4 *>(t);
                }
                *reinterpret_cast<uint4 *>(Bs + cm_offset(nn, 8 * g, BN)) = v;
            }
        }
    };
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nst) load_stage(s);
        cp_async_commit();
    }
    constexpr uint32_t idesc = mma_idesc(kTM, BN);
    bool ok = true;
    int last = -1;
    for (int s = 0; s < nst && ok; ++s) {
        cp_async_wait<kStages - 2>();  // this thread's copies of stage s have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const int buf = s % kStages;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(A + buf * kABytes), b0 = smem_u32(B + buf * kBBytes);
#pragma unroll
            for (int j = 0; j < kTK / 16; ++j) {
                const uint64_t ad = smem_desc(a0 + 2 * j * (kTM / 8) * 128, (kTM / 8) * 128, 128);
                const uint64_t bd = smem_desc(b0 + 2 * j * (BN / 8) * 128, (BN / 8) * 128, 128);
                const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[buf]))
                         : "memory");
        }
        last = s;
        // refill the buffer of stage s - 1 (its MMAs must be done) with stage s + kStages - 1
        const int nxt = s + kStages - 1;
        if (nxt < nst) {
            if (s >= 1) ok = mbar_wait(smem_u32(&mbar[(s - 1) % kStages]), (uint32_t)(((s - 1) / kStages) & 1));
            if (ok) load_stage(nxt);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (last >= 0) ok = mbar_wait(smem_u32(&mbar[last % kStages]), (uint32_t)((last / kStages) & 1)) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const long long p = p0 + warp * 32 + lane;
#pragma unroll
        for (int c = 0; c < BN; c += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (p < P) {
                __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float v = __uint_as_float(r[q]);
                    if (bias) v += bias[n0 + c + q];
                    if (relu) v = fmaxf(v, 0.f);
                    o[q] = __float2bfloat16_rn(v);
                }
                *reinterpret_cast<uint4 *>(out + p * Cout_g + n0 + c) = *reinterpret_cast<const uint4 *>(o);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// ---------------------------------------------------------------------------
// Forward 3x3 convolution, persistent and warp-specialised.  One CTA per SM
// walks the (pixel tile, output-channel tile) items of the layer; its warps have
// fixed roles:
//   warps 0-3  producers: cp.async copies of the A rows (im2col, zero fill) and of
//              the weight tile into a ring of kWsStages stage buffers; each copy's
//              completion arrives on the stage's `full` mbarrier (count 128);
//   warp 8     one thread issues the tcgen05.mma of a stage once it is full and
//              commits them to the stage's `empty` mbarrier (the buffer may be
//              refilled when the MMAs reading it are done); after an item's last
//              stage it commits to `acc_full` of the item's accumulator;
//   warps 4-7  epilogue: wait for `acc_full`, read the accumulator from tensor
//              memory (warp 4 + q owns lanes 32q..32q+31 = pixels), bias, ReLU,
//              BF16 stores, then arrive on `acc_empty` (count 128).
// Two accumulators (2 x BN TMEM columns) alternate between items, so the epilogue
// of one item runs while the next one accumulates, and the producers run ahead
// by up to kWsStages stages across item boundaries.  Tile layout, descriptors and
// MMAs are those of conv3x3_tc_kernel.  Every wait is bounded; a thread whose
// wait runs out sets g_tc_error and a shared abort flag that ends the others' waits.
// ---------------------------------------------------------------------------
constexpr int kWsThreads = 288;  // 9 warps

__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity, volatile int *abort) {
    for (long long it = 0; it < (1ll << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    atomicExch(&g_tc_error, 1);
    *abort = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int BN, int kWsStages>
__global__ void __launch_bounds__(kWsThreads, 1) conv3x3_ws_kernel(const __nv_bfloat16 *__restrict__ in,
                                                                   const __nv_bfloat16 *__restrict__ w,
                                                                   const float *__restrict__ bias,
                                                                   __nv_bfloat16 *__restrict__ out, int N, int H,
                                                                   int Wd, int Cin, int Cout, int relu) {
    constexpr uint32_t kABytes = kTM * kTK * 2, kBBytes = BN * kTK * 2;
    constexpr int kCols = 2 * BN;  // two accumulators
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char *A = tc_smem;
    unsigned char *B = tc_smem + kWsStages * kABytes;
    __shared__ __align__(8) uint64_t full[kWsStages], empty[kWsStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)N * H * Wd;
    const long long ptiles = (P + kTM - 1) / kTM;
    const int ntiles = Cout / BN;
    const long long items = ptiles * ntiles;
    const int K = 9 * Cin, nst = (K + kTK - 1) / kTK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_flag = 0;
        for (int b = 0; b < kWsStages; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(128) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_empty[b])), "r"(128) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp < 4) {
        // ---- producers: thread tid copies A row tid and a share of the B tile
        long long g = 0;  // stage counter over all items of this CTA
        bool ok = true;
        for (long long item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const long long p0 = (item / ntiles) * kTM;
            const int n0 = (int)(item % ntiles) * BN;
            const long long pa = p0 + tid;
            int an = 0, ay = 0, ax = 0;
            if (pa < P) {
                an = (int)(pa / ((long long)H * Wd));
                const int rem = (int)(pa - (long long)an * H * Wd);
                ay = rem / Wd;
                ax = rem - ay * Wd;
            }
            for (int s = 0; s < nst && ok; ++s, ++g) {
                const int buf = (int)(g % kWsStages);
                ok = ws_wait(smem_u32(&empty[buf]), (uint32_t)(((g / kWsStages) & 1) ^ 1), &abort_flag);
                if (!ok) break;
                unsigned char *As = A + buf * kABytes, *Bs = B + buf * kBBytes;
                const int k0 = s * kTK;
#pragma unroll
                for (int gg = 0; gg < kTK / 8; ++gg) {
                    const int k = k0 + 8 * gg;
                    const __nv_bfloat16 *src = in;
                    int bytes = 0;
                    if (pa < P && k < K) {
                        const int tap = k / Cin, c = k - tap * Cin;
                        const int sy = ay + tap / 3 - 1, sx = ax + tap % 3 - 1;
                        if (sy >= 0 && sy < H && sx >= 0 && sx < Wd) {
                            src = in + (((long long)an * H + sy) * Wd + sx) * Cin + c;
                            bytes = 16;
                        }
                    }
                    cp_async16(As + cm_offset(tid, 8 * gg, kTM), src, bytes);
                }
                for (int e = tid; e < BN * (kTK / 8); e += 128) {
                    const int nn = e / (kTK / 8), gg = e % (kTK / 8);
                    const int k = k0 + 8 * gg;
                    const __nv_bfloat16 *src = w;
                    int bytes = 0;
                    if (k < K) {
                        const int tap = k / Cin, c = k - tap * Cin;
                        src = w + ((long long)(n0 + nn) * 9 + tap) * Cin + c;
                        bytes = 16;
                    }
                    cp_async16(Bs + cm_offset(nn, 8 * gg, BN), src, bytes);
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[buf]))
                             : "memory");
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 8) {
        // ---- one thread issues the MMAs
        if (lane == 0) {
            constexpr uint32_t idesc = mma_idesc(kTM, BN);
            long long g = 0, j = 0;
            bool ok = true, issued = false;
            for (long long item = blockIdx.x; item < items && ok; item += gridDim.x, ++j) {
                const int ab = (int)(j & 1);
                ok = ws_wait(smem_u32(&acc_empty[ab]), (uint32_t)(((j >> 1) & 1) ^ 1), &abort_flag);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dcol = tmem + (uint32_t)(ab * BN);
                for (int s = 0; s < nst && ok; ++s, ++g) {
                    const int buf = (int)(g % kWsStages);
                    ok = ws_wait(smem_u32(&full[buf]), (uint32_t)((g / kWsStages) & 1), &abort_flag);
                    if (!ok) break;
                    // the producers' cp.async writes are generic-proxy writes; order them
                    // before the tensor core's reads
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(A + buf * kABytes), b0 = smem_u32(B + buf * kBBytes);
#pragma unroll
                    for (int jj = 0; jj < kTK / 16; ++jj) {
                        const uint64_t ad = smem_desc(a0 + 2 * jj * (kTM / 8) * 128, (kTM / 8) * 128, 128);
                        const uint64_t bd = smem_desc(b0 + 2 * jj * (BN / 8) * 128, (BN / 8) * 128, 128);
                        const uint32_t acc = (s > 0 || jj > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dcol),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty[buf]))
                                 : "memory");
                    issued = true;
                }
                if (ok)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&acc_full[ab]))
                                 : "memory");
            }
            // before the tensor memory is released: the last MMAs must be done
            // (a commit tracks all earlier MMAs of this thread)
            if (issued) {
                uint64_t *fin = &empty[(int)((g - 1) % kWsStages)];
                ws_wait(smem_u32(fin), (uint32_t)(((g - 1) / kWsStages) & 1), &abort_flag);
            }
        }
    } else {
        // ---- epilogue: warp 4 + q reads TMEM lanes 32q..32q+31
        const int q = warp - 4, row = q * 32 + lane;
        long long j = 0;
        bool ok = true;
        for (long long item = blockIdx.x; item < items && ok; item += gridDim.x, ++j) {
            const int ab = (int)(j & 1);
            ok = ws_wait(smem_u32(&acc_full[ab]), (uint32_t)((j >> 1) & 1), &abort_flag);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const long long p = (item / ntiles) * kTM + row;
            const int n0 = (int)(item % ntiles) * BN;
#pragma unroll
            for (int c = 0; c < BN; c += 8) {
                uint32_t r[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN + c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (p < P) {
                    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        float v = __uint_as_float(r[t]);
                        if (bias) v += bias[n0 + c + t];
                        if (relu) v = fmaxf(v, 0.f);
                        o[t] = __float2bfloat16_rn(v);
                    }
                    *reinterpret_cast<uint4 *>(out + p * Cout + n0 + c) = *reinterpret_cast<const uint4 *>(o);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(smem_u32(&acc_empty[ab]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

template <int BN, int S>
cudaError_t launch_conv_ws(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias, __nv_bfloat16 *out,
                           int N, int H, int W, int Cin, int Cout, int relu, cudaStream_t s) {
    const size_t smem = S * (size_t)(kTM * kTK * 2) + S * (size_t)(BN * kTK * 2);
    cudaError_t e = cudaFuncSetAttribute(conv3x3_ws_kernel<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long P = (long long)N * H * W;
    const long long items = ((P + kTM - 1) / kTM) * (Cout / BN);
    const int grid = (int)std::min<long long>(items, sms);
    conv3x3_ws_kernel<BN, S><<<grid, kWsThreads, smem, s>>>(in, w, bias, out, N, H, W, Cin, Cout, relu);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Forward 3x3 convolution without an im2col copy, for images whose rows are a
// whole number of 128-pixel tiles and Cin = 8 G (16, 32 or 64 channels).  An
// output tile is 128 consecutive pixels of one image row.  For each tile the CTA
// stages the three input rows that the tile reads, 130 pixels each (one pixel of
// zero padding on either side), once in shared memory, laid out
// [ky][channel group g][pixel][8 channels]: 8 consecutive pixels of one group form
// one 128-byte core matrix.  The A operand of tap (ky, kx) and channels 16j..16j+15
// is that slab seen from pixel kx: a K-major descriptor whose start address moves
// 16 bytes per pixel, with 128 bytes between 8-pixel groups and 130 x 16 bytes
// between the two channel groups of one MMA.  So every input element is staged
// once per tile, where the im2col staging copies it nine times.  The weights of
// all nine taps for the CTA's BN output channels are staged once per CTA,
// [tap][g][co][8 channels].  The CTA is persistent over tiles: the slab of the
// next tile is copied (cp.async, zero fill outside the image) while the tensor
// core works on the current one, and two accumulators in tensor memory let the
// epilogue of one tile run while the next accumulates.  Every wait is bounded;
// on a time-out the kernel sets g_tc_error, waits (bounded) for its own MMAs and
// copies, frees its tensor memory and returns.
// ---------------------------------------------------------------------------
constexpr int kSlabW = kTM + 2;  // staged pixels per input row

__host__ __device__ constexpr uint32_t slab_bytes(int G) {
    return (uint32_t)((3 * G * kSlabW * 16 + 127) / 128 * 128);
}

template <int BN, int G>
__global__ void __launch_bounds__(kTcThreads) conv3x3_slab_kernel(const __nv_bfloat16 *__restrict__ in,
                                                                  const __nv_bfloat16 *__restrict__ w,
                                                                  const float *__restrict__ bias,
                                                                  __nv_bfloat16 *__restrict__ out, int N, int H,
                                                                  int Wd, int Cout, int relu) {
    constexpr int Cin = 8 * G;
    constexpr int kAcc = BN < 32 ? 32 : BN;  // TMEM columns of one accumulator
    constexpr int kCols = 2 * kAcc;
    constexpr uint32_t kSlab = slab_bytes(G);
    extern __shared__ __align__(128) unsigned char sl_smem[];
    unsigned char *const Wsm = sl_smem + 2 * kSlab;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * BN;
    const int tiles_x = Wd / kTM;
    const long long ntiles = (long long)N * H * tiles_x;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // weights: W[n0 + co][t][8g .. 8g + 7] -> Wsm[(t G + g) BN + co]
    for (int e = tid; e < 9 * G * BN; e += kTcThreads) {
        const int g = e % G, co = (e / G) % BN, t = e / (G * BN);
        cp_async16(Wsm + ((t * G + g) * BN + co) * 16, w + ((long long)(n0 + co) * 9 + t) * Cin + 8 * g, 16);
    }
    // the three input rows of a tile, channel group fastest (coalesced reads)
    const auto stage = [&](long long tile, unsigned char *dst) {
        const int tx = (int)(tile % tiles_x);
        const long long ry = tile / tiles_x;
        const int y = (int)(ry % H), n = (int)(ry / H), x0 = tx * kTM;
        for (int e = tid; e < 3 * G * kSlabW; e += kTcThreads) {
            const int g = e % G, px = (e / G) % kSlabW, ky = e / (G * kSlabW);
            const int sy = y + ky - 1, sx = x0 + px - 1;
            const bool inside = sy >= 0 && sy < H && sx >= 0 && sx < Wd;
            const __nv_bfloat16 *src = inside ? in + (((long long)n * H + sy) * Wd + sx) * Cin + 8 * g : in;
            cp_async16(dst + ((ky * G + g) * kSlabW + px) * 16, src, inside ? 16 : 0);
        }
    };
    const auto epilogue = [&](long long tile, int acc) {
        const int tx = (int)(tile % tiles_x);
        const long long row = tile / tiles_x;  // n H + y
        const long long p = row * Wd + tx * kTM + warp * 32 + lane;
#pragma unroll
        for (int c = 0; c < BN; c += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * kAcc + c)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            __align__(16) __nv_bfloat16 o[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float v = __uint_as_float(r[q]);
                if (bias) v += bias[n0 + c + q];
                if (relu) v = fmaxf(v, 0.f);
                o[q] = __float2bfloat16_rn(v);
            }
            *reinterpret_cast<uint4 *>(out + p * Cout + n0 + c) = *reinterpret_cast<const uint4 *>(o);
        }
    };

    constexpr uint32_t idesc = mma_idesc(kTM, BN);
    long long tile = blockIdx.x;
    if (tile < ntiles) stage(tile, sl_smem);
    cp_async_commit();  // the weights and the first slab
    bool ok = true;
    int i = 0;
    long long prev = -1;
    for (; tile < ntiles; tile += gridDim.x, ++i) {
        const int b = i & 1;
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sl_smem + b * kSlab), w0 = smem_u32(Wsm);
            int k = 0;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t % 3;
#pragma unroll
                for (int j = 0; j < G / 2; ++j, ++k) {
                    const uint64_t ad = smem_desc(a0 + (uint32_t)(((ky * G + 2 * j) * kSlabW + kx) * 16), kSlabW * 16, 128);
                    const uint64_t bd = smem_desc(w0 + (uint32_t)((t * G + 2 * j) * BN * 16), BN * 16, 128);
                    const uint32_t accum = k > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)(b * kAcc)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[b]))
                         : "memory");
        }
        // the previous tile's MMAs: done -> its slab buffer and accumulator are free
        if (i > 0) {
            const bool mine = ok && mbar_wait(smem_u32(&mbar[b ^ 1]), (uint32_t)(((i - 1) >> 1) & 1));
            ok = __syncthreads_and(mine) != 0;  // one decision for the whole CTA
        }
        const long long next = tile + gridDim.x;
        if (ok && next < ntiles) stage(next, sl_smem + (b ^ 1) * kSlab);
        cp_async_commit();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok && i > 0) epilogue(prev, b ^ 1);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        prev = tile;
        if (!ok) {
            ++i;
            break;
        }
    }
    // the last tile (its commit tracks every earlier MMA of the issuing thread;
    // waited for also after a time-out, before the tensor memory is freed)
    if (i > 0) {
        const bool done = mbar_wait(smem_u32(&mbar[(i - 1) & 1]), (uint32_t)(((i - 1) >> 1) & 1));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok && done) epilogue(prev, (i - 1) & 1);
    }
    cp_async_wait<0>();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

template <int BN, int G>
cudaError_t launch_conv_slab(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias, __nv_bfloat16 *out,
                             int N, int H, int W, int Cout, int relu, cudaStream_t s) {
    const size_t smem = 2 * (size_t)slab_bytes(G) + 9 * (size_t)G * BN * 16;
    cudaError_t e = cudaFuncSetAttribute(conv3x3_slab_kernel<BN, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    // the whole unified L1 / shared memory as shared memory, so that several CTAs fit on an SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(conv3x3_slab_kernel<BN, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, smem_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    // CTAs per SM (the persistent grid): as many as the shared memory (1 KB reserved a
    // CTA) and the tensor memory (512 columns per SM, two accumulators a CTA) hold; 48
    // registers a thread never limit it.  (The occupancy query answered one CTA per SM
    // here, which left two thirds of the SMs' slots empty: 142 against 93 us.)
    const int per_sm = std::max(1, std::min((int)(smem_sm / (smem + 1024)), 512 / (2 * (BN < 32 ? 32 : BN))));
    const long long tiles = (long long)N * H * (W / kTM);
    const int gx = (int)std::max<long long>(1, std::min<long long>(tiles, (long long)sms * per_sm / (Cout / BN)));
    dim3 grid(gx, Cout / BN);
    conv3x3_slab_kernel<BN, G><<<grid, kTcThreads, smem, s>>>(in, w, bias, out, N, H, W, Cout, relu);
    return cudaGetLastError();
}

// The slab kernel's shapes: forward, rows of whole 128-pixel tiles, Cin 16, 32 or 64.
bool slab_shape(int W, int Cin_g, int Cout_g) {
    return W % kTM == 0 && (Cin_g == 16 || Cin_g == 32 || Cin_g == 64) && Cout_g % 16 == 0;
}

cudaError_t conv_dispatch_slab(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias, __nv_bfloat16 *out,
                               int N, int H, int W, int Cin_g, int Cout_g, int relu, cudaStream_t s) {
    // (for 64 input channels at most 64 output channels a CTA: the staged weights of
    // 128 would not fit beside the two slabs)
    int BN = Cout_g % 128 == 0 ? 128 : (Cout_g % 64 == 0 ? 64 : (Cout_g % 32 == 0 ? 32 : 16));
    if (Cin_g == 64 && BN > 64) BN = 64;
#define CDF_SLAB(G, WIDE)                                                                               \
    switch (BN) {                                                                                       \
        case 128: return launch_conv_slab<WIDE, G>(in, w, bias, out, N, H, W, Cout_g, relu, s);         \
        case 64: return launch_conv_slab<64, G>(in, w, bias, out, N, H, W, Cout_g, relu, s);            \
        case 32: return launch_conv_slab<32, G>(in, w, bias, out, N, H, W, Cout_g, relu, s);            \
        default: return launch_conv_slab<16, G>(in, w, bias, out, N, H, W, Cout_g, relu, s);            \
    }
    if (Cin_g == 16) CDF_SLAB(2, 128)
    if (Cin_g == 32) CDF_SLAB(4, 128)
    CDF_SLAB(8, 64)  // BN is at most 64 here
#undef CDF_SLAB
}

template <bool kBwdData, int BN>
cudaError_t launch_conv_tc_pipe(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias,
                                __nv_bfloat16 *out, int N, int H, int W, int Cin_g, int Cout_g, int relu,
                                cudaStream_t s) {
    const size_t smem = kStages * (size_t)(kTM * kTK * 2) + kStages * (size_t)(BN * kTK * 2);
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_pipe_kernel<kBwdData, BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long P = (long long)N * H * W;
    dim3 grid((unsigned)((P + kTM - 1) / kTM), Cout_g / BN);
    conv3x3_tc_pipe_kernel<kBwdData, BN><<<grid, kTcThreads, smem, s>>>(in, w, bias, out, N, H, W, Cin_g, Cout_g,
                                                                        relu);
    return cudaGetLastError();
}

template <bool kBwdData, int BN>
cudaError_t launch_conv_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias, __nv_bfloat16 *out,
                           int N, int H, int W, int Cin_g, int Cout_g, int relu, cudaStream_t s) {
    const size_t smem = 2 * (size_t)(kTM * kTK * 2) + 2 * (size_t)(BN * kTK * 2);
    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<kBwdData, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long P = (long long)N * H * W;
    dim3 grid((unsigned)((P + kTM - 1) / kTM), Cout_g / BN);
    conv3x3_tc_kernel<kBwdData, BN><<<grid, kTcThreads, smem, s>>>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu);
    return cudaGetLastError();
}

// Convolution path: 1 = tcgen05, the faster staging per shape (default), 2 = tcgen05
// with synchronous staging, 3 = tcgen05 persistent warp-specialised forward,
// 4 = the forward without im2col copy (conv3x3_slab_kernel) where the shape allows it,
// else as 1, 0 = the warp-level MMA kernels.
int g_path = 1;
bool g_use_tc = true;

template <bool kBwdData>
cudaError_t conv_dispatch_path2(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias, __nv_bfloat16 *out,
                                int N, int H, int W, int Cin_g, int Cout_g, int relu, cudaStream_t s, int BN) {
    switch (BN) {
        case 128: return launch_conv_tc<kBwdData, 128>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
        case 64: return launch_conv_tc<kBwdData, 64>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
        case 32: return launch_conv_tc<kBwdData, 32>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
        default: return launch_conv_tc<kBwdData, 16>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
    }
}

template <bool kBwdData>
cudaError_t conv_dispatch(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias, __nv_bfloat16 *out,
                          int N, int H, int W, int Cin_g, int Cout_g, int relu, cudaStream_t s) {
    const int BN = Cout_g % 128 == 0 ? 128 : (Cout_g % 64 == 0 ? 64 : (Cout_g % 32 == 0 ? 32 : 16));
    if ((g_path == 1 || g_path == 4) && !kBwdData && slab_shape(W, Cin_g, Cout_g))
        return conv_dispatch_slab(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
    if (g_path == 3 && !kBwdData) {  // forward: the persistent warp-specialised kernel
        switch (BN) {
            case 128: return launch_conv_ws<128, 4>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
            case 64: return launch_conv_ws<64, 5>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
            default: return launch_conv_ws<32, 6>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
        }
    }
    // the default picks by the measured faster form: the cp.async pipeline for long K
    // (Cin >= 128, e.g. 159 against 101 TFLOP/s at 32^2 x 256 -> 256), two-buffer
    // synchronous staging for short K, where more CTAs per SM hide more latency
    // (80 against 72 TFLOP/s at 256^2 x 32 -> 32)
    if ((g_path == 1 || g_path == 4) && Cin_g < 128)
        return conv_dispatch_path2<kBwdData>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s, BN);
    if (g_path == 1 || g_path == 3 || g_path == 4) {
        switch (BN) {
            case 128: return launch_conv_tc_pipe<kBwdData, 128>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
            case 64: return launch_conv_tc_pipe<kBwdData, 64>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
            case 32: return launch_conv_tc_pipe<kBwdData, 32>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
            default: return launch_conv_tc_pipe<kBwdData, 16>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s);
        }
    }
    if (g_path == 2) return conv_dispatch_path2<kBwdData>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu, s, BN);
    const long long P = (long long)N * H * W;
    const int bn = BN >= 64 ? 64 : BN;
    dim3 grid((unsigned)((P + kBM - 1) / kBM), Cout_g / bn);
    if (bn == 64) conv3x3_kernel<kBwdData, 64><<<grid, kThreads, 0, s>>>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu);
    else if (bn == 32) conv3x3_kernel<kBwdData, 32><<<grid, kThreads, 0, s>>>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu);
    else conv3x3_kernel<kBwdData, 16><<<grid, kThreads, 0, s>>>(in, w, bias, out, N, H, W, Cin_g, Cout_g, relu);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 3x3 convolution, weight gradient: dW[co][t][ci] += sum_p dY[p][co] X[p + d(t)][ci]
// GEMM per tap: M = Cout (tile 64), N = Cin (tile 16), K = pixels (chunk of 64 per
// stage, split over the grid's z dimension); FP32 partial sums are added atomically.
// ---------------------------------------------------------------------------
constexpr int kWBM = 64, kWBK = 64;
__global__ void __launch_bounds__(kThreads) conv3x3_wgrad_kernel(const __nv_bfloat16 *__restrict__ x,
                                                                 const __nv_bfloat16 *__restrict__ dy,
                                                                 float *__restrict__ dw, int N, int H, int Wd,
                                                                 int Cin, int Cout, long long pix_per_split) {
    __shared__ __align__(32) __nv_bfloat16 As[kWBK * (kWBM + 8)];  // [k = pixel][m = co]
    __shared__ __align__(32) __nv_bfloat16 Bs[kWBK * kLdA];       // [k = pixel][n = ci]
    __shared__ __align__(32) float Cs[kWBM * 20];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int co0 = blockIdx.x * kWBM;
    const int tap = blockIdx.y / (Cin / 16), ci0 = (blockIdx.y % (Cin / 16)) * 16;
    const int dyy = tap / 3 - 1, dxx = tap % 3 - 1;
    const long long P = (long long)N * H * Wd;
    const long long pbeg = (long long)blockIdx.z * pix_per_split;
    const long long pend = pbeg + pix_per_split < P ? pbeg + pix_per_split : P;
    const int mrows = Cout - co0 < kWBM ? Cout - co0 : kWBM;  // 32 or 64 output channels

    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
    wmma::fill_fragment(acc, 0.f);
    for (long long pk = pbeg; pk < pend; pk += kWBK) {
        // A: dY rows (pixel k, output channels co0..co0+63), 8 channels per 16-byte load.
        for (int e = tid; e < kWBK * (kWBM / 8); e += kThreads) {
            const int kk = e / (kWBM / 8), seg = (e % (kWBM / 8)) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            const long long p = pk + kk;
            if (p < pend && seg < mrows) v = *reinterpret_cast<const uint4 *>(dy + p * Cout + co0 + seg);
            *reinterpret_cast<uint4 *>(As + kk * (kWBM + 8) + seg) = v;
        }
        // B: X at the shifted pixel, 16 input channels.
        {
            const int kk = tid >> 1, half = (tid & 1) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            const long long p = pk + kk;
            if (p < pend) {
                const int n = (int)(p / ((long long)H * Wd));
                const int rem = (int)(p - (long long)n * H * Wd);
                const int yy = rem / Wd + dyy, xx = rem % Wd + dxx;
                if (yy >= 0 && yy < H && xx >= 0 && xx < Wd)
                    v = *reinterpret_cast<const uint4 *>(x + (((long long)n * H + yy) * Wd + xx) * Cin + ci0 + half);
            }
            *reinterpret_cast<uint4 *>(Bs + kk * kLdA + half) = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kWBK; ks += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::col_major> a;
            wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
            wmma::load_matrix_sync(a, As + ks * (kWBM + 8) + warp * 16, kWBM + 8);
            wmma::load_matrix_sync(b, Bs + ks * kLdA, kLdA);
            wmma::mma_sync(acc, a, b, acc);
        }
        __syncthreads();
    }
    wmma::store_matrix_sync(Cs + warp * 16 * 20, acc, 20, wmma::mem_row_major);
    __syncthreads();
    for (int e = tid; e < kWBM * 16; e += kThreads) {
        const int r = e >> 4, c = e & 15;
        if (r < mrows) atomicAdd(dw + ((long long)(co0 + r) * 9 + tap) * Cin + ci0 + c, Cs[r * 20 + c]);
    }
}

// ---------------------------------------------------------------------------
// 3x3 convolution, weight gradient, on the tcgen05 tensor cores with a
// deterministic split over the pixels:
//   dW[co][t][ci] = sum_p dY[p][co] X[p + d(t)][ci].
// GEMM: M = 9 Cin rows m = t Cin + ci (tile 128), N = Cout (one tile, <= 256),
// K = pixels in stages of 64, split over blockIdx.y into `splits` contiguous
// pixel ranges.  Both operands are channel-contiguous in memory (NHWC) while the
// MMA reads K-major tiles, so each thread stages an 8 x 8 block -- 8 rows (8
// consecutive channels) x 8 pixels -- with eight 16-byte loads, transposes it in
// registers and writes eight 16-byte K-major rows.  Each split writes its FP32
// partial tile to the workspace; wgrad_reduce_kernel then adds the splits in a
// fixed order (no atomics: the result is the same bits on every run).
// ---------------------------------------------------------------------------
// 8 x 8 BF16 transpose: in[k] holds channels 0..7 of pixel k; out[c] holds
// pixels 0..7 of channel c.
__device__ __forceinline__ void transpose8x8(const uint4 (&in)[8], uint4 (&out)[8]) {
    const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(in);
    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out);
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k) o[c * 8 + k] = e[k * 8 + c];
}

template <int BN, int MT>
__global__ void __launch_bounds__(kTcThreads) conv3x3_wgrad_tc_kernel(const __nv_bfloat16 *__restrict__ x,
                                                                      const __nv_bfloat16 *__restrict__ dy,
                                                                      float *__restrict__ part, int N, int H, int Wd,
                                                                      int Cin, int Cout, long long pix_per_split) {
    // MT accumulators of 128 x BN in tensor memory, columns mt * BN (a power of two >= 32 allocated)
    constexpr int kNeed = MT * BN;
    constexpr int kCols = kNeed <= 32 ? 32 : (kNeed <= 64 ? 64 : (kNeed <= 128 ? 128 : (kNeed <= 256 ? 256 : 512)));
    constexpr uint32_t kABytes = kTM * kTK * 2, kBBytes = BN * kTK * 2;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char *A = tc_smem;                     // [2 stages][MT tiles][kABytes]
    unsigned char *B = tc_smem + 2 * MT * kABytes;  // [2 stages][kBBytes]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)N * H * Wd;
    const int M = 9 * Cin, mtiles = (M + kTM - 1) / kTM;
    const int t0 = blockIdx.x * MT, n0 = blockIdx.z * BN;
    const int nt = mtiles - t0 < MT ? mtiles - t0 : MT;  // M tiles of this CTA (>= 1)
    const long long pbeg = (long long)blockIdx.y * pix_per_split;
    const long long pend = pbeg + pix_per_split < P ? pbeg + pix_per_split : P;
    const int nst = (int)((pend - pbeg + kTK - 1) / kTK);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // this thread's A block in each M tile: rows (t0 + mt) * 128 + mg * 8 .. + 7 (one tap, eight
    // consecutive channels), pixels kg * 8 .. + 7 of the stage
    const int mg = tid >> 3, kg = tid & 7;
    int ddy[MT], ddx[MT], cib[MT];
    bool rok[MT];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
        const int ma = (t0 + mt) * kTM + mg * 8;
        rok[mt] = mt < nt && ma < M;  // M is a multiple of 8 (Cin % 16 == 0)
        const int tap = rok[mt] ? ma / Cin : 0;
        cib[mt] = rok[mt] ? ma - tap * Cin : 0;
        ddy[mt] = tap / 3 - 1;
        ddx[mt] = tap % 3 - 1;
    }
    const long long hw = (long long)H * Wd;
    constexpr uint32_t idesc = mma_idesc(kTM, BN);
    bool ok = true;
    int last = -1;
    for (int s = 0; s < nst && ok; ++s) {
        const int buf = s & 1;
        if (s >= 2) ok = mbar_wait(smem_u32(&mbar[buf]), (uint32_t)(((s - 2) >> 1) & 1));
        if (!ok) break;
        unsigned char *Bs = B + buf * kBBytes;
        const long long pk = pbeg + (long long)s * kTK + kg * 8;
        // image coordinates of this thread's eight pixels (one division per stage, then a walk)
        int pn[8], py[8], px[8];
        {
            int n = (int)(pk / hw);
            const int rem = (int)(pk - (long long)n * hw);
            int yy = rem / Wd, xx = rem - (rem / Wd) * Wd;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                pn[k] = n;
                py[k] = yy;
                px[k] = xx;
                if (++xx == Wd) {
                    xx = 0;
                    if (++yy == H) {
                        yy = 0;
                        ++n;
                    }
                }
            }
        }
        // A: X at the tap-shifted pixels, 8 channels each (zero outside the image, the range or M)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            if (mt >= nt) break;
            uint4 v[8], t[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                v[k] = make_uint4(0, 0, 0, 0);
                const int yy = py[k] + ddy[mt], xx = px[k] + ddx[mt];
                if (rok[mt] && pk + k < pend && yy >= 0 && yy < H && xx >= 0 && xx < Wd)
                    v[k] = *reinterpret_cast<const uint4 *>(x + (((long long)pn[k] * H + yy) * Wd + xx) * Cin + cib[mt]);
            }
            transpose8x8(v, t);
            unsigned char *As = A + (buf * MT + mt) * kABytes;
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4 *>(As + cm_offset(mg * 8 + c, kg * 8, kTM)) = t[c];
        }
        // B: dY rows of the same pixels, 8 output channels per block, spread from the last thread
        // down (the first threads carry the most A work when the last M tile is partial)
        for (int e = kTcThreads - 1 - tid; e < (BN / 8) * 8; e += kTcThreads) {
            const int ng = e >> 3, kb = e & 7;
            const long long pb = pbeg + (long long)s * kTK + kb * 8;
            uint4 v[8], t[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                v[k] = make_uint4(0, 0, 0, 0);
                if (pb + k < pend) v[k] = *reinterpret_cast<const uint4 *>(dy + (pb + k) * Cout + n0 + ng * 8);
            }
            transpose8x8(v, t);
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4 *>(Bs + cm_offset(ng * 8 + c, kb * 8, BN)) = t[c];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t b0 = smem_u32(Bs);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                if (mt >= nt) break;
                const uint32_t a0 = smem_u32(A + (buf * MT + mt) * kABytes);
#pragma unroll
                for (int j = 0; j < kTK / 16; ++j) {
                    const uint64_t ad = smem_desc(a0 + 2 * j * (kTM / 8) * 128, (kTM / 8) * 128, 128);
                    const uint64_t bd = smem_desc(b0 + 2 * j * (BN / 8) * 128, (BN / 8) * 128, 128);
                    const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)(mt * BN)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[buf]))
                         : "memory");
        }
        last = s;
    }
    if (last >= 0) ok = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1)) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // TMEM lane = tile row; each tile's partial sums into part[split][m][co]
        // (a split without pixels writes zeros)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            if (mt >= nt) break;
            const int m = (t0 + mt) * kTM + warp * 32 + lane;
            float *row = part + ((long long)blockIdx.y * M + m) * Cout + n0;
#pragma unroll
            for (int c = 0; c < BN; c += 8) {
                uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (nst > 0) {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                                   "=r"(r[6]), "=r"(r[7])
                                 : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * BN + c)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                }
                if (m < M) {
                    float4 *d = reinterpret_cast<float4 *>(row + c);
                    d[0] = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]),
                                       __uint_as_float(r[3]));
                    d[1] = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]),
                                       __uint_as_float(r[7]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// dW[co][m] += sum_{split = 0..splits-1} part[split][m][co], in that order.
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, float *__restrict__ dw, int M, int Cout,
                                    int splits) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // i = co * M + m
    if (i >= (long long)M * Cout) return;
    const int co = (int)(i / M), m = (int)(i - (long long)co * M);
    float acc = 0.f;
    for (int z = 0; z < splits; ++z) acc += part[((long long)z * M + m) * Cout + co];
    dw[i] += acc;
}

// Bias gradient with a fixed summation order, db[c] += sum_p dY[p][c], in two
// passes: bias_partial_kernel gives each block of 256 threads 8 channels and one
// run of `per` pixels (each thread a strided part of the run, then a tree in
// shared memory) and writes its sums to part[split][c]; bias_sum_kernel adds the
// splits in order.
__global__ void bias_partial_kernel(const __nv_bfloat16 *__restrict__ dy, float *__restrict__ part, long long P,
                                    int C, long long per) {
    const int c0 = blockIdx.x * 8;
    const long long p0 = (long long)blockIdx.y * per, p1 = min(P, p0 + per);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const uint4 v = *reinterpret_cast<const uint4 *>(dy + p * C + c0);
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int q = 0; q < 8; ++q) s[q] += __bfloat162float(e[q]);
    }
    __shared__ float red[8][256];
#pragma unroll
    for (int q = 0; q < 8; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
#pragma unroll
            for (int q = 0; q < 8; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 8) part[(long long)blockIdx.y * C + c0 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void bias_sum_kernel(const float *__restrict__ part, float *__restrict__ db, int C, int splits) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float acc = 0.f;
    for (int z = 0; z < splits; ++z) acc += part[(long long)z * C + c];
    db[c] += acc;
}

// Pixel splits of the bias gradient: about two blocks per SM over the C / 8
// channel groups, at least 2048 pixels a split.
long long bias_splits(long long P, int C) {
    const long long groups = C / 8;
    long long s = (304 + groups - 1) / groups;
    const long long cap = (P + 2047) / 2048;
    if (s > cap) s = cap;
    return s < 1 ? 1 : s;
}

// The weight gradient's tiling: output-channel tile BN (the largest of 256, 128,
// 64, 32 that divides Cout); MT of the 128-row M tiles per CTA, which share each
// staged tile of dY (at most 256 tensor-memory columns, MT * BN, and three tiles),
// spread evenly over gx CTAs; pixel splits for about two CTAs per SM in all with at
// least 16 stages of 64 pixels each, and the pixels per split (a multiple of 64;
// no split is empty).
struct WgradPlan {
    int bn, mt, gx, splits;
    long long per;
};
WgradPlan wgrad_plan(long long P, int Cin, int Cout) {
    WgradPlan w;
    w.bn = Cout % 256 == 0 ? 256 : (Cout % 128 == 0 ? 128 : (Cout % 64 == 0 ? 64 : 32));
    const int mtiles = (9 * Cin + kTM - 1) / kTM;
    const int mtmax = w.bn >= 256 ? 1 : (w.bn >= 128 ? 2 : 3);
    w.gx = (mtiles + mtmax - 1) / mtmax;
    w.mt = (mtiles + w.gx - 1) / w.gx;
    const long long tiles = (long long)w.gx * (Cout / w.bn);
    long long s = (304 + tiles - 1) / tiles;
    const long long cap = (P + 16 * kTK - 1) / (16 * kTK);
    if (s > cap) s = cap;
    if (s < 1) s = 1;
    w.per = ((P + s - 1) / s + kTK - 1) / kTK * kTK;
    w.splits = (int)((P + w.per - 1) / w.per);
    return w;
}

template <int BN, int MT>
cudaError_t launch_wgrad_tc(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, float *part, int N, int H, int W,
                            int Cin, int Cout, const WgradPlan &w, cudaStream_t s) {
    const size_t smem = 2 * MT * (size_t)(kTM * kTK * 2) + 2 * (size_t)(BN * kTK * 2);
    cudaError_t e = cudaFuncSetAttribute(conv3x3_wgrad_tc_kernel<BN, MT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)w.gx, (unsigned)w.splits, (unsigned)(Cout / BN));
    conv3x3_wgrad_tc_kernel<BN, MT><<<grid, kTcThreads, smem, s>>>(x, dy, part, N, H, W, Cin, Cout, w.per);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small layers (one thread per element unless stated).
// ---------------------------------------------------------------------------
__global__ void bias_grad_kernel(const __nv_bfloat16 *__restrict__ dy, float *__restrict__ db, long long P, int C) {
    // block: 256 threads over pixels for one channel group of 8; grid.x = C / 8, grid.y = splits
    const int c0 = blockIdx.x * 8;
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long p = (long long)blockIdx.y * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.y * blockDim.x) {
        const uint4 v = *reinterpret_cast<const uint4 *>(dy + p * C + c0);
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int q = 0; q < 8; ++q) s[q] += __bfloat162float(e[q]);
    }
    __shared__ float red[8][256];
#pragma unroll
    for (int q = 0; q < 8; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
#pragma unroll
            for (int q = 0; q < 8; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 8) atomicAdd(db + c0 + threadIdx.x, red[threadIdx.x][0]);
}

__global__ void relu_bwd_kernel(__nv_bfloat16 *__restrict__ d, const __nv_bfloat16 *__restrict__ y, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(__bfloat162float(y[i]) > 0.f)) d[i] = __float2bfloat16_rn(0.f);
}

__global__ void avgpool2_fwd_kernel(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y, int N, int H,
                                    int W, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    const long long n_out = (long long)N * Ho * Wo * C;
    if (i >= n_out) return;
    const int c = (int)(i % C);
    long long q = i / C;
    const int xo = (int)(q % Wo);
    q /= Wo;
    const int yo = (int)(q % Ho);
    const int n = (int)(q / Ho);
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            s += __bfloat162float(x[(((long long)n * H + 2 * yo + a) * W + 2 * xo + b) * C + c]);
    y[i] = __float2bfloat16_rn(0.25f * s);
}

__global__ void avgpool2_bwd_kernel(const __nv_bfloat16 *__restrict__ dy, __nv_bfloat16 *__restrict__ dx, int N, int H,
                                    int W, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over dx
    const long long n_in = (long long)N * H * W * C;
    if (i >= n_in) return;
    const int c = (int)(i % C);
    long long q = i / C;
    const int xx = (int)(q % W);
    q /= W;
    const int yy = (int)(q % H);
    const int n = (int)(q / H);
    const float g = __bfloat162float(dy[(((long long)n * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c]);
    dx[i] = __float2bfloat16_rn(0.25f * g);
}

// Nearest 2x upsampling of x [N, H, W, C] into channels [coff, coff + C) of y [N, 2H, 2W, Cy].
__global__ void upsample2_fwd_kernel(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y, int N, int H,
                                     int W, int C, int Cy, int coff) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over y's selected channels
    const long long n_out = (long long)N * 2 * H * 2 * W * C;
    if (i >= n_out) return;
    const int c = (int)(i % C);
    long long q = i / C;
    const int xo = (int)(q % (2 * W));
    q /= 2 * W;
    const int yo = (int)(q % (2 * H));
    const int n = (int)(q / (2 * H));
    y[(((long long)n * 2 * H + yo) * 2 * W + xo) * Cy + coff + c] = x[(((long long)n * H + yo / 2) * W + xo / 2) * C + c];
}

// Backward of the above: dx[n][y][x][c] = sum of the 4 covering dy values (channels coff..coff+C of dy).
__global__ void upsample2_bwd_kernel(const __nv_bfloat16 *__restrict__ dy, __nv_bfloat16 *__restrict__ dx, int N, int H,
                                     int W, int C, int Cy, int coff) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n_in = (long long)N * H * W * C;
    if (i >= n_in) return;
    const int c = (int)(i % C);
    long long q = i / C;
    const int xx = (int)(q % W);
    q /= W;
    const int yy = (int)(q % H);
    const int n = (int)(q / H);
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            s += __bfloat162float(dy[(((long long)n * 2 * H + 2 * yy + a) * 2 * W + 2 * xx + b) * Cy + coff + c]);
    dx[i] = __float2bfloat16_rn(s);
}

// y[:, :, :, dst_off + c] = x[:, :, :, src_off + c] for c < count (skip concat / split).
__global__ void copy_channels_kernel(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y, long long P,
                                     int Cx, int Cy, int src_off, int dst_off, int count, int accumulate) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * count) return;
    const long long p = i / count;
    const int c = (int)(i - p * count);
    const float v = __bfloat162float(x[p * Cx + src_off + c]);
    __nv_bfloat16 *d = y + p * Cy + dst_off + c;
    *d = __float2bfloat16_rn(accumulate ? v + __bfloat162float(*d) : v);
}

// 1x1 output head in FP32 arithmetic: out[p][o] = sum_c x[p][c] w[o][c] + b[o].
__global__ void head_fwd_kernel(const __nv_bfloat16 *__restrict__ x, const float *__restrict__ w,
                                const float *__restrict__ b, float *__restrict__ out, long long P, int C, int O) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * O) return;
    const long long p = i / O;
    const int o = (int)(i - p * O);
    float s = b[o];
    for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(x[p * C + c]), w[o * C + c], s);
    out[i] = s;
}

// dx[p][c] = sum_o dout[p][o] w[o][c]
__global__ void head_bwd_data_kernel(const float *__restrict__ dout, const float *__restrict__ w,
                                     __nv_bfloat16 *__restrict__ dx, long long P, int C, int O) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * C) return;
    const long long p = i / C;
    const int c = (int)(i - p * C);
    float s = 0.f;
    for (int o = 0; o < O; ++o) s = fmaf(dout[p * O + o], w[o * C + c], s);
    dx[i] = __float2bfloat16_rn(s);
}

// dw[o][c] += sum_p dout[p][o] x[p][c]; db[o] += sum_p dout[p][o]  (one block per (o, c-chunk) pair, grid-stride)
__global__ void head_bwd_weight_kernel(const __nv_bfloat16 *__restrict__ x, const float *__restrict__ dout,
                                       float *__restrict__ dw, float *__restrict__ db, long long P, int C, int O) {
    const int o = blockIdx.x / (C + 1), c = blockIdx.x % (C + 1);  // c == C: bias
    float s = 0.f;
    for (long long p = (long long)blockIdx.y * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.y * blockDim.x)
        s += dout[p * O + o] * (c < C ? __bfloat162float(x[p * C + c]) : 1.f);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(c < C ? dw + o * C + c : db + o, red[0]);
}

// Mean squared error over n values; loss (FP32 sum, atomically added) and its gradient 2 (pred - target) / n.
__global__ void mse_kernel(const float *__restrict__ pred, const float *__restrict__ target, float *__restrict__ grad,
                           float *__restrict__ loss, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (i < n) {
        const float d = pred[i] - target[i];
        grad[i] = 2.f * d / (float)n;
        e = d * d / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, e);
}

// Adam on FP32 master weights; refreshes the BF16 copy when one is given.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
}

inline unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

thread_local char g_nn_err[256] = "";
cdf_nn_status nn_fail(const char *m) {
    int i = 0;
    for (; m[i] && i < 255; ++i) g_nn_err[i] = m[i];
    g_nn_err[i] = 0;
    return CDF_NN_EINVAL;
}
cdf_nn_status launched() {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return CDF_NN_OK;
    int i = 0;
    const char *m = cudaGetErrorString(e);
    for (; m[i] && i < 255; ++i) g_nn_err[i] = m[i];
    g_nn_err[i] = 0;
    return CDF_NN_ECUDA;
}

}  // namespace

extern "C" {

const char *cdf_nn_last_error(void) { return g_nn_err; }

cdf_nn_status cdf_nn_set_tensor_path(int tcgen05) {
    if (tcgen05 < 0 || tcgen05 > 4) return nn_fail("set_tensor_path: 0, 1, 2, 3 or 4");
    g_path = tcgen05;
    g_use_tc = tcgen05 != 0;
    return CDF_NN_OK;
}

cdf_nn_status cdf_nn_error_flag(int *out) {
    if (!out) return nn_fail("error_flag: NULL argument");
    const cudaError_t e = cudaMemcpyFromSymbol(out, g_tc_error, sizeof(int));
    if (e != cudaSuccess) return nn_fail(cudaGetErrorString(e));
    return CDF_NN_OK;
}

cdf_nn_status cdf_nn_conv3x3_fwd(const void *x, const void *w, const float *bias, void *y, int N, int H, int W,
                                 int Cin, int Cout, int relu, void *stream) {
    if (!x || !w || !y || N < 1 || H < 1 || W < 1 || Cin % 16 || Cout % 32 || Cin < 16)
        return nn_fail("conv3x3_fwd: bad arguments (Cin % 16, Cout % 32)");
    cudaError_t e = conv_dispatch<false>(static_cast<const __nv_bfloat16 *>(x), static_cast<const __nv_bfloat16 *>(w),
                                         bias, static_cast<__nv_bfloat16 *>(y), N, H, W, Cin, Cout, relu,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) { cudaGetLastError(); return nn_fail(cudaGetErrorString(e)); }
    return launched();
}

cdf_nn_status cdf_nn_conv3x3_bwd_data(const void *dy, const void *w, void *dx, int N, int H, int W, int Cin, int Cout,
                                      void *stream) {
    if (!dy || !w || !dx || N < 1 || H < 1 || W < 1 || Cin % 16 || Cout % 32)
        return nn_fail("conv3x3_bwd_data: bad arguments (Cin % 16, Cout % 32)");
    cudaError_t e = conv_dispatch<true>(static_cast<const __nv_bfloat16 *>(dy), static_cast<const __nv_bfloat16 *>(w),
                                        nullptr, static_cast<__nv_bfloat16 *>(dx), N, H, W, Cout, Cin, 0,
                                        static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) { cudaGetLastError(); return nn_fail(cudaGetErrorString(e)); }
    return launched();
}

long long cdf_nn_conv3x3_bwd_weight_workspace(int N, int H, int W, int Cin, int Cout) {
    if (N < 1 || H < 1 || W < 1 || Cin < 16 || Cin % 16 || Cout < 32 || Cout % 32) return -1;
    const long long P = (long long)N * H * W;
    const WgradPlan w = wgrad_plan(P, Cin, Cout);
    return ((long long)w.splits * 9 * Cin * Cout + bias_splits(P, Cout) * Cout) * (long long)sizeof(float);
}

cdf_nn_status cdf_nn_conv3x3_bwd_weight(const void *x, const void *dy, float *dw, float *db, int N, int H, int W,
                                        int Cin, int Cout, void *workspace, long long workspace_bytes, void *stream) {
    if (!x || !dy || !dw || N < 1 || H < 1 || W < 1 || Cin % 16 || Cout % 32)
        return nn_fail("conv3x3_bwd_weight: bad arguments (Cin % 16, Cout % 32)");
    const long long P = (long long)N * H * W;
    auto s = static_cast<cudaStream_t>(stream);
    const auto *xb = static_cast<const __nv_bfloat16 *>(x);
    const auto *dyb = static_cast<const __nv_bfloat16 *>(dy);
    if (g_use_tc) {
        const long long need = cdf_nn_conv3x3_bwd_weight_workspace(N, H, W, Cin, Cout);
        if (!workspace || workspace_bytes < need)
            return nn_fail("conv3x3_bwd_weight: the workspace is missing or smaller than "
                           "cdf_nn_conv3x3_bwd_weight_workspace()");
        const WgradPlan w = wgrad_plan(P, Cin, Cout);
        float *part = static_cast<float *>(workspace);
        cudaError_t e;
        // M = 9 Cin >= 144 spans at least two tiles, so MT = 1 occurs only with BN = 256
        switch (w.bn * 4 + w.mt) {
            case 256 * 4 + 1: e = launch_wgrad_tc<256, 1>(xb, dyb, part, N, H, W, Cin, Cout, w, s); break;
            case 128 * 4 + 2: e = launch_wgrad_tc<128, 2>(xb, dyb, part, N, H, W, Cin, Cout, w, s); break;
            case 64 * 4 + 2: e = launch_wgrad_tc<64, 2>(xb, dyb, part, N, H, W, Cin, Cout, w, s); break;
            case 64 * 4 + 3: e = launch_wgrad_tc<64, 3>(xb, dyb, part, N, H, W, Cin, Cout, w, s); break;
            case 32 * 4 + 2: e = launch_wgrad_tc<32, 2>(xb, dyb, part, N, H, W, Cin, Cout, w, s); break;
            case 32 * 4 + 3: e = launch_wgrad_tc<32, 3>(xb, dyb, part, N, H, W, Cin, Cout, w, s); break;
            default: return nn_fail("conv3x3_bwd_weight: no kernel for this tiling");
        }
        if (e != cudaSuccess) { cudaGetLastError(); return nn_fail(cudaGetErrorString(e)); }
        const long long n = 9LL * Cin * Cout;
        wgrad_reduce_kernel<<<blocks_for(n), 256, 0, s>>>(part, dw, 9 * Cin, Cout, w.splits);
        if (db) {
            float *bpart = part + (long long)w.splits * 9 * Cin * Cout;  // after the weight partials
            const long long bs = bias_splits(P, Cout), per = (P + bs - 1) / bs;
            bias_partial_kernel<<<dim3(Cout / 8, (unsigned)bs), 256, 0, s>>>(dyb, bpart, P, Cout, per);
            bias_sum_kernel<<<(Cout + 127) / 128, 128, 0, s>>>(bpart, db, Cout, (int)bs);
        }
    } else {
        // the warp-level MMA path: split-K partial sums added atomically (order-dependent)
        const long long per = 4096;
        dim3 grid((unsigned)((Cout + kWBM - 1) / kWBM), 9 * (Cin / 16), (unsigned)((P + per - 1) / per));
        conv3x3_wgrad_kernel<<<grid, kThreads, 0, s>>>(xb, dyb, dw, N, H, W, Cin, Cout, per);
        if (db) {
            dim3 g2(Cout / 8, (unsigned)((P + 256 * 64 - 1) / (256 * 64)));
            bias_grad_kernel<<<g2, 256, 0, s>>>(dyb, db, P, Cout);
        }
    }
    return launched();
}

cdf_nn_status cdf_nn_relu_bwd(void *d, const void *y, long long n, void *stream) {
    if (!d || !y || n < 0) return nn_fail("relu_bwd: bad arguments");
    if (n) relu_bwd_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<__nv_bfloat16 *>(d), static_cast<const __nv_bfloat16 *>(y), n);
    return launched();
}

cdf_nn_status cdf_nn_avgpool2_fwd(const void *x, void *y, int N, int H, int W, int C, void *stream) {
    if (!x || !y || H % 2 || W % 2) return nn_fail("avgpool2: H and W must be even");
    const long long n = (long long)N * (H / 2) * (W / 2) * C;
    avgpool2_fwd_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16 *>(x), static_cast<__nv_bfloat16 *>(y), N, H, W, C);
    return launched();
}

cdf_nn_status cdf_nn_avgpool2_bwd(const void *dy, void *dx, int N, int H, int W, int C, void *stream) {
    if (!dy || !dx || H % 2 || W % 2) return nn_fail("avgpool2: H and W must be even");
    const long long n = (long long)N * H * W * C;
    avgpool2_bwd_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16 *>(dy), static_cast<__nv_bfloat16 *>(dx), N, H, W, C);
    return launched();
}

cdf_nn_status cdf_nn_upsample2_fwd(const void *x, void *y, int N, int H, int W, int C, int Cy, int coff, void *stream) {
    if (!x || !y || coff < 0 || coff + C > Cy) return nn_fail("upsample2: bad channel slice");
    const long long n = (long long)N * 4 * H * W * C;
    upsample2_fwd_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16 *>(x), static_cast<__nv_bfloat16 *>(y), N, H, W, C, Cy, coff);
    return launched();
}

cdf_nn_status cdf_nn_upsample2_bwd(const void *dy, void *dx, int N, int H, int W, int C, int Cy, int coff, void *stream) {
    if (!dy || !dx || coff < 0 || coff + C > Cy) return nn_fail("upsample2: bad channel slice");
    const long long n = (long long)N * H * W * C;
    upsample2_bwd_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16 *>(dy), static_cast<__nv_bfloat16 *>(dx), N, H, W, C, Cy, coff);
    return launched();
}

cdf_nn_status cdf_nn_copy_channels(const void *x, void *y, long long P, int Cx, int Cy, int src_off, int dst_off,
                                   int count, int accumulate, void *stream) {
    if (!x || !y || src_off + count > Cx || dst_off + count > Cy || count < 0) return nn_fail("copy_channels: bad slice");
    const long long n = P * count;
    if (n) copy_channels_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16 *>(x), static_cast<__nv_bfloat16 *>(y), P, Cx, Cy, src_off, dst_off, count,
        accumulate);
    return launched();
}

cdf_nn_status cdf_nn_head_fwd(const void *x, const float *w, const float *b, float *out, long long P, int C, int O,
                              void *stream) {
    if (!x || !w || !b || !out) return nn_fail("head_fwd: NULL argument");
    head_fwd_kernel<<<blocks_for(P * O), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16 *>(x), w, b, out, P, C, O);
    return launched();
}

cdf_nn_status cdf_nn_head_bwd(const void *x, const float *w, const float *dout, void *dx, float *dw, float *db,
                              long long P, int C, int O, void *stream) {
    if (!x || !w || !dout || !dx || !dw || !db) return nn_fail("head_bwd: NULL argument");
    auto s = static_cast<cudaStream_t>(stream);
    head_bwd_data_kernel<<<blocks_for(P * C), 256, 0, s>>>(dout, w, static_cast<__nv_bfloat16 *>(dx), P, C, O);
    dim3 g((unsigned)(O * (C + 1)), (unsigned)((P + 256 * 32 - 1) / (256 * 32)));
    head_bwd_weight_kernel<<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(x), dout, dw, db, P, C, O);
    return launched();
}

cdf_nn_status cdf_nn_mse(const float *pred, const float *target, float *grad, float *loss, long long n, void *stream) {
    if (!pred || !target || !grad || !loss) return nn_fail("mse: NULL argument");
    mse_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(pred, target, grad, loss, n);
    return launched();
}

cdf_nn_status cdf_nn_adam(float *w, const float *g, float *m, float *v, void *w_bf16, long long n, float lr, float b1,
                          float b2, float eps, long long step, void *stream) {
    if (!w || !g || !m || !v || step < 1) return nn_fail("adam: bad arguments");
    float c1 = 1.f, c2 = 1.f, p1 = 1.f, p2 = 1.f;
    for (long long i = 0; i < step && i < 100000; ++i) { p1 *= b1; p2 *= b2; }
    c1 -= p1;
    c2 -= p2;
    adam_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        w, g, m, v, static_cast<__nv_bfloat16 *>(w_bf16), n, lr, b1, b2, eps, c1, c2);
    return launched();
}

}  // extern "C"
