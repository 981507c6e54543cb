// Tile-resident persistent step for lattices that fit in the GPU's shared
// memory (about 150 k nodes for m = 2 on 152 SMs).
//
// A lattice of that size lives in L2 between steps, so the one-launch-per-step
// kernel is bound by latency: each launch pays the graph-node gap, the L2
// round trip of every pull and a single short wave.  Here one cooperative launch
// advances many steps.  Each CTA owns a rectangular tile whose post-collision
// populations stay in shared memory (two buffers, pull from one, write the
// other), and one thread owns one node for the whole launch (its S_1(t-1)
// stays in a register).  Only the tile's outer ring of nodes talks to other
// CTAs: ring nodes also write their populations to the global ping-pong
// buffers, and before a step the ring threads wait for the neighbouring tiles'
// counters to say that their ring values of that step are published.  Interior
// nodes pull from shared memory only, so their collision overlaps the
// exchange.  The update of each node is the same pull table and collision as
// the global-memory kernel, so the results are bitwise the same.
//
// Every wait is bounded (GPU global timer and an iteration cap); on time-out
// the CTA sets the error word, the others see it at their next wait, and the
// host reports CDF_ETIMEOUT.
#include "lb_device.cuh"

#include <algorithm>

namespace cdflb {
namespace {
using namespace dev;

constexpr int kResidentThreads = 1024;

// Thread t of a w x hgt tile: the R ring nodes first (bottom row, top row,
// left column, right column), then the interior in row order.
__device__ __forceinline__ void tile_node(int t, int w, int hgt, int R, int &lx, int &ly) {
    if (t < R) {
        if (t < w) { lx = t; ly = 0; return; }
        t -= w;
        if (hgt > 1) {
            if (t < w) { lx = t; ly = hgt - 1; return; }
            t -= w;
        }
        const int side = hgt - 2;  // rows 1 .. hgt - 2 of the side columns
        if (t < side) { lx = 0; ly = 1 + t; return; }
        t -= side;
        lx = w - 1;
        ly = 1 + t;
        return;
    }
    const int i = t - R, iw = w - 2;
    lx = 1 + i % iw;
    ly = 1 + i / iw;
}

// Wait until the counter at `flag` reaches `target` (wrapping compare).
__device__ bool wait_counter(const unsigned *flag, unsigned target, unsigned long long timeout_ns, int *err) {
    volatile const unsigned *vf = flag;
    volatile int *verr = err;
    if ((int)(*vf - target) < 0) {
        const unsigned long long t0 = global_ns();
        const unsigned long long cap = timeout_ns / 32ull + (1ull << 20);
        unsigned long long it = 0;
        while ((int)(*vf - target) < 0) {
            if (*verr) return false;
            if (++it > cap || ((it & 63ull) == 0 && global_ns() - t0 > timeout_ns)) {
                atomicExch(err, 1);
                return false;
            }
        }
    }
    __threadfence();
    return true;
}

// One node of the resident step.  A: current populations of the tile (shared
// memory, plane stride TS, row stride tw); B: the next ones.  Ring nodes read
// sources outside the tile from the global buffer `in` (through L2: other CTAs
// wrote them during this launch) and write their result to `out` as well.
template <int M, bool kInterior>
__device__ __forceinline__ void resident_node(const LbParams &p, int x, int y, int X0, int Y0, int w, int hgt,
                                              int tw, int TS, const float *A, float *B, const float *in,
                                              float *out, bool to_global, float &sp1, float *sprev, bool last,
                                              float *moments) {
    const long long P = p.plane;
    const int pitch = p.pitch;
    float f[M][5], h[9];
    if (kInterior) {
        const auto mk = [tw, X0, Y0](int sx, int sy) { return (sy - Y0) * tw + (sx - X0); };
        const auto ld = [A, TS, &p](int plane, int off) { return A[plane * TS + CDF_CHK(p, off, TS, 8)]; };
        pull_node<M, true>(p, x, y, mk, ld, f, h);
    } else {
        const auto mk = [](int sx, int sy) { return make_int2(sx, sy); };
        const auto ld = [=](int plane, int2 c) {
            const int lx = c.x - X0, ly = c.y - Y0;
            return ((unsigned)lx < (unsigned)w && (unsigned)ly < (unsigned)hgt)
                       ? A[plane * TS + CDF_CHK(p, ly * tw + lx, TS, 8)]
                       : __ldcg(in + plane * P + CDF_CHK(p, (long long)c.y * pitch + c.x, P, 7));
        };
        pull_node<M, false>(p, x, y, mk, ld, f, h);
    }
    NodeOut<M> o;
    collide<M>(p, f, h, pref_at(p, x, y), sp1, false, o);
    const int l0 = CDF_CHK(p, (y - Y0) * tw + (x - X0), TS, 8);
#pragma unroll
    for (int i = 0; i < 9; ++i) B[i * TS + l0] = h[i];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) B[(9 + 5 * a + i) * TS + l0] = f[a][i];
    const int o0 = CDF_CHK(p, y * pitch + x, P, 2);
    if (to_global) store_node<M, float>(out, P, o0, f, h);
    if (M >= 2 && p.skind == 2) {
        sp1 = o.s1;
        if (last) sprev[o0] = o.s1;
    }
    if (moments) write_moments<M>(moments, P, o0, o);
}

__device__ __forceinline__ void ring_barrier(int threads) {
    asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}

template <int M>
__global__ void __launch_bounds__(kResidentThreads, 1)
    resident_kernel(const LbParams p, const ResidentGeom g, float *buf0, float *buf1, const float *sp_in,
                    float *sprev, float *moments,
                    int nsteps, int parity0, int moments_last, unsigned *counters, unsigned long long timeout_ns,
                    int *err) {
    constexpr int NP = 9 + 5 * M;
    extern __shared__ float sm[];
    __shared__ int s_abort;
    __shared__ unsigned s_base;
    const int tid = threadIdx.x, b = blockIdx.x;
    const int bx = b % g.tiles_x, by = b / g.tiles_x;
    const int X0 = bx * g.tw, Y0 = by * g.th;
    const int w = min(g.tw, p.nx - X0), hgt = min(g.th, p.ny - Y0);
    const int nodes = w * hgt;
    const int R = nodes - max(w - 2, 0) * max(hgt - 2, 0);
    const int ring_threads = min((R + 31) & ~31, (int)blockDim.x);
    const int TS = g.tw * g.th;
    const long long P = p.plane;
    const bool has_node = tid < nodes, ring = tid < R;
    int lx = 0, ly = 0;
    if (has_node) tile_node(tid, w, hgt, R, lx, ly);
    const int x = X0 + lx, y = Y0 + ly;

    // Threads 0..7 each watch one neighbouring tile (wrapping on periodic axes).
    int nb = -1;
    if (tid < 8) {
        const int d = tid < 4 ? tid : tid + 1;  // the 3 x 3 block without its centre
        int nx_ = bx + d % 3 - 1, ny_ = by + d / 3 - 1;
        bool ok = true;
        if (nx_ < 0 || nx_ >= g.tiles_x) {
            ok = ok && p.periodic_x;
            nx_ = (nx_ + g.tiles_x) % g.tiles_x;
        }
        if (ny_ < 0 || ny_ >= g.tiles_y) {
            ok = ok && p.periodic_y;
            ny_ = (ny_ + g.tiles_y) % g.tiles_y;
        }
        const int k = ny_ * g.tiles_x + nx_;
        if (ok && k != b) nb = k;
    }
    if (tid == 0) {
        s_abort = *(volatile int *)err;
        // Every counter ends a launch at the same value, so this tile's own
        // counter is the common base of the step numbering of this launch.
        s_base = *(volatile unsigned *)(counters + b);
    }
    const bool consume = M >= 2 && p.skind == 2;
    float sp1 = 0.f;
    {
        const float *in = parity0 ? buf1 : buf0;
        if (has_node) {
            const int o0 = CDF_CHK(p, y * p.pitch + x, P, 2), l0 = CDF_CHK(p, ly * g.tw + lx, TS, 8);
#pragma unroll
            for (int k = 0; k < NP; ++k) sm[k * TS + l0] = in[k * P + o0];
            if (consume) sp1 = sp_in[o0];
        }
    }
    __syncthreads();
    if (s_abort) return;
    const unsigned base = s_base;

    for (int s = 0; s < nsteps; ++s) {
        const float *A = sm + (s & 1) * NP * TS;
        float *B = sm + ((s + 1) & 1) * NP * TS;
        const float *in = ((parity0 + s) & 1) ? buf1 : buf0;
        float *out = ((parity0 + s) & 1) ? buf0 : buf1;
        const bool last = s == nsteps - 1;
        float *mom = (moments_last && last) ? moments : nullptr;
        int abort_now = 0;
        if (tid < ring_threads) {
            if (s > 0) {
                if (nb >= 0 && !wait_counter(counters + nb, base + s, timeout_ns, err)) s_abort = 1;
                ring_barrier(ring_threads);
            }
            // s_abort is written only before the first ring barrier of a step
            // and read after it (the next writes follow the step's __syncthreads).
            abort_now = s_abort;
            if (!abort_now && has_node) {
                if (ring)
                    resident_node<M, false>(p, x, y, X0, Y0, w, hgt, g.tw, TS, A, B, in, out, true, sp1, sprev,
                                            last, mom);
                else
                    resident_node<M, true>(p, x, y, X0, Y0, w, hgt, g.tw, TS, A, B, in, out, last, sp1, sprev,
                                           last, mom);
            }
            ring_barrier(ring_threads);
            if (tid == 0 && !abort_now && b != g.stall_tile) {
                __threadfence();  // the ring's global stores before the counter
                atomicExch(counters + b, base + s + 1);
            }
        } else if (has_node) {
            resident_node<M, true>(p, x, y, X0, Y0, w, hgt, g.tw, TS, A, B, in, out, last, sp1, sprev, last, mom);
        }
        if (__syncthreads_or(abort_now)) return;
    }
}

template <int M>
const void *kernel_of() {
    return reinterpret_cast<const void *>(resident_kernel<M>);
}

const void *resident_kernel_for(int m) {
    switch (m) {
        case 1: return kernel_of<1>();
        case 2: return kernel_of<2>();
        case 3: return kernel_of<3>();
        case 4: return kernel_of<4>();
        default: return nullptr;
    }
}

}  // namespace

bool plan_resident(int nx, int ny, int m, ResidentGeom *out) {
    const void *kern = resident_kernel_for(m);
    if (!kern || nx < 1 || ny < 1) return false;
    int dev = 0, sms = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return false;
    const int np = 9 + 5 * m;
    const int max_threads = std::min(kResidentThreads, fa.maxThreadsPerBlock);
    const long long smem_cap = (long long)smem_optin - (long long)fa.sharedSizeBytes;
    const int max_nodes = (int)std::min<long long>(max_threads, smem_cap / (2LL * np * 4));
    if (max_nodes < 1) return false;
    bool found = false;
    ResidentGeom best{};
    long long best_nodes = 0, best_ring = 0;
    // One CTA per SM: choose the tiling with the smallest largest tile (the
    // critical path of a step), then the shortest ring (least exchange).
    for (int tx = 1; tx <= std::min(nx, sms); ++tx) {
        const int tw = (nx + tx - 1) / tx;
        const int tiles_x = (nx + tw - 1) / tw;
        if (tiles_x != tx) continue;
        const int max_ty = sms / tiles_x;
        if (max_ty < 1) break;
        const int ty0 = std::min(ny, max_ty);
        const int th = (ny + ty0 - 1) / ty0;
        const int tiles_y = (ny + th - 1) / th;
        const long long nodes = (long long)tw * th;
        if (nodes > max_nodes) continue;
        const long long ring = 2LL * (tw + th);
        if (!found || nodes < best_nodes || (nodes == best_nodes && ring < best_ring)) {
            found = true;
            best_nodes = nodes;
            best_ring = ring;
            best.tiles_x = tiles_x;
            best.tiles_y = tiles_y;
            best.tw = tw;
            best.th = th;
        }
    }
    if (!found) return false;
    best.threads = (int)((best_nodes + 31) / 32 * 32);
    best.smem_bytes = (size_t)2 * np * best_nodes * sizeof(float);
    best.stall_tile = -1;
    // The attribute is per kernel, shared by every handle: allow the largest tile.
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap) != cudaSuccess)
        return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, best.threads, best.smem_bytes) != cudaSuccess ||
        (long long)per_sm * sms < (long long)best.tiles_x * best.tiles_y)
        return false;
    *out = best;
    return true;
}

cudaError_t launch_resident(const LbParams &p, const ResidentGeom &g, float *buf0, float *buf1, const float *sp_in,
                            float *sprev,
                            float *moments, int nsteps, int parity0, bool moments_last, unsigned *counters,
                            unsigned long long timeout_ns, int *err, cudaStream_t s) {
    const void *kern = resident_kernel_for(p.m);
    if (!kern) return cudaErrorInvalidValue;
    LbParams pp = p;
    ResidentGeom gg = g;
    int ml = moments_last ? 1 : 0;
    void *args[] = {&pp, &gg, &buf0, &buf1, &sp_in, &sprev, &moments, &nsteps, &parity0, &ml, &counters, &timeout_ns, &err};
    return cudaLaunchCooperativeKernel(kern, dim3(g.tiles_x * g.tiles_y), dim3(g.threads), args, g.smem_bytes, s);
}

}  // namespace cdflb
