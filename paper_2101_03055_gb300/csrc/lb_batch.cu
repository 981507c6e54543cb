// Batched solver: many lattices of uneven size advanced by one persistent
// kernel.  Work is scheduled as (instance, tile) units; a bounded grid barrier
// separates time steps inside a launch, so one launch advances every instance
// by `steps_per_launch` steps.  Each node runs the same step_node() as the
// single-lattice kernel, with its instance's parameters staged in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "lb_device.cuh"

namespace cdflb {
namespace {

struct BatchInst {
    LbParams p;
    long long pop_off;  // element offset of the instance's planes in a population buffer
    long long sp_off;   // offset in the S(t-1) buffer
    long long mom_off;  // offset in the moment buffer
    int tile_base;      // first tile of the instance
    int tiles_x;
};

// Grid-wide barrier for a co-resident (cooperative) grid.  bar[0] counts
// arrivals, bar[1] is the generation.  Every wait is bounded: after timeout_ns
// (or an iteration cap) the block sets err[0] and the whole grid gives up; the
// first block to give up records the step, the arrivals it saw and the time it
// waited (err[1..3], microseconds) for the host's message.  Returns false when
// the barrier failed.
__device__ bool grid_barrier(unsigned *bar, unsigned expected, unsigned long long timeout_ns, int *err, int step) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        ok = 1;
        volatile unsigned *vgen = bar + 1;
        volatile int *verr = err;
        const unsigned gen = *vgen;
        __threadfence();  // this block's stores of the step before the arrival
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = dev::global_ns();
            const unsigned long long cap = timeout_ns / 32ull + (1ull << 20);
            unsigned long long it = 0;
            while (*vgen == gen) {
                if (*verr) { ok = 0; break; }
                if (++it > cap || ((it & 63ull) == 0 && dev::global_ns() - t0 > timeout_ns)) {
                    if (atomicCAS(err, 0, 1) == 0) {
                        err[1] = step;
                        err[2] = (int)*(volatile unsigned *)bar;
                        err[3] = (int)min((dev::global_ns() - t0) / 1000ull, 2000000000ull);
                    }
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            __threadfence();
        }
    }
    __syncthreads();
    return ok != 0;
}

template <int M>
__global__ void __launch_bounds__(256, 4) batch_kernel(const BatchInst *__restrict__ inst, const int *__restrict__ tile_inst,
                                                    int total_tiles, float *buf0, float *buf1, float *sprev,
                                                    float *moments, int nsteps, int parity0, int moments_last,
                                                    unsigned *bar, unsigned expected, unsigned long long timeout_ns,
                                                    int *err) {
    __shared__ LbParams sp;
    __shared__ long long s_off[3];
    __shared__ int s_tile[2];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    for (int s = 0; s < nsteps; ++s) {
        const float *in = ((parity0 + s) & 1) ? buf1 : buf0;
        float *out = ((parity0 + s) & 1) ? buf0 : buf1;
        float *mom = (moments_last && s == nsteps - 1) ? moments : nullptr;
        int cur_inst = -1;
        // Each block takes a contiguous range of tiles: long runs of one instance
        // (parameters staged once) and neighbouring tiles whose halos are still in L1.
        const int t_begin = (int)((long long)total_tiles * blockIdx.x / gridDim.x);
        const int t_end = (int)((long long)total_tiles * (blockIdx.x + 1) / gridDim.x);
        for (int t = t_begin; t < t_end; ++t) {
            const int k = tile_inst[t];
            if (k != cur_inst) {  // stage the instance's parameters in shared memory
                __syncthreads();
                const int *src = reinterpret_cast<const int *>(&inst[k].p);
                int *dst = reinterpret_cast<int *>(&sp);
                for (int w = tid; w < (int)(sizeof(LbParams) / sizeof(int)); w += nthreads) dst[w] = src[w];
                if (tid == 0) {
                    s_off[0] = inst[k].pop_off;
                    s_off[1] = inst[k].sp_off;
                    s_off[2] = inst[k].mom_off;
                    s_tile[0] = inst[k].tile_base;
                    s_tile[1] = inst[k].tiles_x;
                }
                __syncthreads();
                cur_inst = k;
            }
            const int lt = t - s_tile[0];
            const int ty = lt / s_tile[1], tx = lt - ty * s_tile[1];
            const int x = tx * blockDim.x + threadIdx.x, y = ty * blockDim.y + threadIdx.y;
            if (x < sp.nx && y < sp.ny)
                dev::step_node<M, float, true>(sp, x, y, in + s_off[0], out + s_off[0], sprev + s_off[1],
                                               sprev + s_off[1], mom ? mom + s_off[2] : nullptr);
        }
        if (s + 1 < nsteps && !grid_barrier(bar, expected, timeout_ns, err, s)) return;
    }
}

thread_local char g_berr[512] = "";
cdf_status bfail(cdf_status st, const char *msg) {
    std::snprintf(g_berr, sizeof g_berr, "%s", msg);
    return report_error(st, msg);
}

#define BCK(call)                                                                     \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            char m_[400];                                                             \
            std::snprintf(m_, sizeof m_, "%s failed: %s", #call, cudaGetErrorString(e_)); \
            return bfail(CDF_ECUDA, m_);                                              \
        }                                                                             \
    } while (0)

using TuneKey = std::tuple<long long, long long, int, int>;
std::mutex g_btune_mu;
std::map<TuneKey, dim3> g_btune;

}  // namespace
}  // namespace cdflb

using namespace cdflb;

struct cdf_batch {
    int device = 0;
    int count = 0, m = 0;
    std::vector<LbParams> params;
    std::vector<long long> pop_off, sp_off, mom_off;
    long long pop_total = 0, sp_total = 0, mom_total = 0, nodes = 0;
    int sprev_planes = 0;
    float *buf[2] = {nullptr, nullptr};
    // S_1(t - 1): the persistent kernel updates `sprev` in place; the kernel
    // chains alternate `sprev` and `sprev2` with the population buffers (a
    // two-step launch reads halo nodes that other CTAs rewrite).
    float *sprev = nullptr, *sprev2 = nullptr, *mom = nullptr, *dense = nullptr, *host_stage = nullptr;
    float *mom_prev = nullptr;                        // snapshot for per-instance residuals
    double *partials = nullptr, *red = nullptr, *red_host = nullptr;  // per-instance reductions
    size_t stage_floats = 0;
    BatchInst *d_inst = nullptr;
    int *d_tile_inst = nullptr;
    unsigned *d_bar = nullptr;
    int *d_err = nullptr, *h_err = nullptr;
    int total_tiles = 0, grid_blocks = 0;
    dim3 tile{64, 4, 1};
    int steps_per_launch = 32;
    unsigned long long timeout_ns = 1000000000ull;
    int extra_arrivals = 0;
    cudaStream_t s = nullptr, user = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int cur = 0;
    long long t = 0;
    // Second execution mode: one chain of single-lattice step kernels per
    // instance (each launch reads its parameters as kernel operands), fanned out
    // over a pool of streams and captured as one CUDA graph; instances are
    // independent, so the chains need no barrier between them.
    int mode = 0;  // 0: persistent kernel, 1: graph of per-instance chains, 2: chains of two-step launches
    dim3 chain_block{128, 1, 1};
    int chain_th = 14;  // mode 2: output tile height of step2_kernel (chain_block is its CTA)
    std::vector<cudaStream_t> pool;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    cudaGraphExec_t chain_graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [parity][moments]
};

namespace {

void brelease(cdf_batch *b) {
    if (!b) return;
    for (auto &row : b->chain_graph)
        for (auto &g : row)
            if (g) cudaGraphExecDestroy(g);
    for (cudaStream_t ps : b->pool) cudaStreamDestroy(ps);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    dev_free(b->buf[0]);
    dev_free(b->buf[1]);
    dev_free(b->sprev);
    dev_free(b->sprev2);
    dev_free(b->mom);
    dev_free(b->mom_prev);
    cudaFree(b->partials);
    cudaFree(b->red);
    if (b->red_host) cudaFreeHost(b->red_host);
    dev_free(b->dense);
    cudaFree(b->d_inst);
    cudaFree(b->d_tile_inst);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->host_stage) cudaFreeHost(b->host_stage);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->s) cudaStreamDestroy(b->s);
    delete b;
}

// Tile table and instance descriptors for a tile shape; sets the grid size.
cdf_status setup_tiles(cdf_batch *b, dim3 tile) {
    std::vector<BatchInst> inst(b->count);
    std::vector<int> tiles;
    for (int k = 0; k < b->count; ++k) {
        const LbParams &p = b->params[k];
        const int tx = (p.nx + tile.x - 1) / tile.x, ty = (p.ny + tile.y - 1) / tile.y;
        inst[k].p = p;
        inst[k].pop_off = b->pop_off[k];
        inst[k].sp_off = b->sp_off[k];
        inst[k].mom_off = b->mom_off[k];
        inst[k].tile_base = (int)tiles.size();
        inst[k].tiles_x = tx;
        for (int i = 0; i < tx * ty; ++i) tiles.push_back(k);
    }
    cudaFree(b->d_tile_inst);
    b->d_tile_inst = nullptr;
    BCK(cudaMalloc(&b->d_tile_inst, tiles.size() * sizeof(int)));
    BCK(cudaMemcpy(b->d_inst, inst.data(), inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_tile_inst, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice));
    b->total_tiles = (int)tiles.size();
    b->tile = tile;
    int per_sm = 0, sms = 0;
    void (*kern)(const BatchInst *, const int *, int, float *, float *, float *, float *, int, int, int, unsigned *,
                 unsigned, unsigned long long, int *) = nullptr;
    switch (b->m) {
        case 1: kern = batch_kernel<1>; break;
        case 2: kern = batch_kernel<2>; break;
        case 3: kern = batch_kernel<3>; break;
        default: kern = batch_kernel<4>; break;
    }
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tile.x * tile.y, 0));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid_blocks = std::max(1, std::min(per_sm * sms, b->total_tiles));
    return CDF_OK;
}

cdf_status launch_batch(cdf_batch *b, int nsteps, bool moments_last) {
    BCK(cudaMemsetAsync(b->d_err, 0, 4 * sizeof(int), b->s));
    BCK(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->s));
    unsigned expected = (unsigned)b->grid_blocks + (unsigned)b->extra_arrivals;
    int parity = b->cur, ml = moments_last ? 1 : 0;
    void *args[] = {&b->d_inst, &b->d_tile_inst, &b->total_tiles, &b->buf[0], &b->buf[1], &b->sprev, &b->mom,
                    &nsteps, &parity, &ml, &b->d_bar, &expected, &b->timeout_ns, &b->d_err};
    const void *kern = nullptr;
    switch (b->m) {
        case 1: kern = (const void *)batch_kernel<1>; break;
        case 2: kern = (const void *)batch_kernel<2>; break;
        case 3: kern = (const void *)batch_kernel<3>; break;
        default: kern = (const void *)batch_kernel<4>; break;
    }
    BCK(cudaLaunchCooperativeKernel(kern, dim3(b->grid_blocks), b->tile, args, 0, b->s));
    BCK(cudaMemcpyAsync(b->h_err, b->d_err, 4 * sizeof(int), cudaMemcpyDeviceToHost, b->s));
    if (nsteps & 1) b->cur ^= 1;
    b->t += nsteps;
    return CDF_OK;
}

constexpr int kPoolStreams = 32;
constexpr int kChainGraphSteps = 32;  // even: the buffer parity returns

// S_1(t - 1) plane set that belongs to population buffer `par`.
float *sprev_of(cdf_batch *b, int par) { return (b->mode == 0 || par == 0) ? b->sprev : b->sprev2; }

// Kernel launches of the chains for n steps: one per step, or in mode 2 one per
// two steps plus one single step for an odd n.  Each launch flips the parity.
int chain_launches(const cdf_batch *b, int nsteps) { return b->mode == 2 ? nsteps / 2 + nsteps % 2 : nsteps; }

// Enqueue n steps of every instance as chains of single-lattice step kernels on
// the stream pool (fork from and join back to the batch stream).
cdf_status enqueue_chains(cdf_batch *b, int nsteps, bool moments_last, int parity0) {
    BCK(cudaEventRecord(b->ev_fork, b->s));
    for (cudaStream_t ps : b->pool) BCK(cudaStreamWaitEvent(ps, b->ev_fork, 0));
    const int launches = chain_launches(b, nsteps);
    for (int j = 0; j < launches; ++j) {
        const int par = (parity0 + j) & 1;
        const bool two = b->mode == 2 && 2 * (j + 1) <= nsteps;
        for (int k = 0; k < b->count; ++k) {
            float *mom = (moments_last && j == launches - 1) ? b->mom + b->mom_off[k] : nullptr;
            float *in = b->buf[par] + b->pop_off[k], *out = b->buf[par ^ 1] + b->pop_off[k];
            float *sin = sprev_of(b, par) + b->sp_off[k], *sout = sprev_of(b, par ^ 1) + b->sp_off[k];
            cudaStream_t ps = b->pool[k % b->pool.size()];
            if (two)
                BCK(launch_step2(b->params[k], in, out, sin, sout, mom, b->chain_block, b->chain_th, ps));
            else
                BCK(launch_step(b->params[k], kFP32, in, out, sin, sout, mom,
                                b->mode == 2 ? dim3(128, 1) : b->chain_block, ps));
        }
    }
    for (size_t j = 0; j < b->pool.size(); ++j) {
        BCK(cudaEventRecord(b->ev_join[j], b->pool[j]));
        BCK(cudaStreamWaitEvent(b->s, b->ev_join[j], 0));
    }
    return CDF_OK;
}

// Changing the CTA shape of the chains invalidates their captured graphs.
void set_chain_block(cdf_batch *b, dim3 blk) {
    for (auto &row : b->chain_graph)
        for (auto &g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    b->chain_block = blk;
}

cdf_status run_chains(cdf_batch *b, int nsteps, bool moments_last) {
    if (nsteps == kChainGraphSteps) {
        cudaGraphExec_t &ge = b->chain_graph[b->cur][moments_last ? 1 : 0];
        if (!ge) {
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
            cdf_status st = enqueue_chains(b, nsteps, moments_last, b->cur);
            cudaError_t e = cudaStreamEndCapture(b->s, &g);
            if (st != CDF_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            BCK(e);
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            BCK(e);
        }
        BCK(cudaGraphLaunch(ge, b->s));
    } else {
        cdf_status st = enqueue_chains(b, nsteps, moments_last, b->cur);
        if (st != CDF_OK) return st;
    }
    if (chain_launches(b, nsteps) & 1) b->cur ^= 1;
    b->t += nsteps;
    return CDF_OK;
}

// Can step2_kernel with CTA blk and tile height th run every instance?  blk.z
// == 2: the paired-lane kernel (m <= 2, CTAs of 32 x 8, tile heights 14 and 30).
bool chain_pair_fits(const cdf_batch *b, dim3 blk, int th) {
    if (blk.z == 2 && (b->m > 2 || blk.x != 32 || blk.y != 8 || (th != 14 && th != 30))) return false;
    if (blk.x % 32 != 0 || (int)(blk.x * blk.y) > step2_max_threads(b->m) || th < 1) return false;
    if (step2_smem_bytes(b->m, blk, th) > (size_t)kStep2MaxSmem) return false;
    for (const LbParams &p : b->params)
        if ((p.periodic_x && p.nx < (int)blk.x) || (p.periodic_y && p.ny < th + 2)) return false;
    return true;
}

cdf_status check_err(cdf_batch *b) {
    if (*b->h_err) {
        char m[256];
        std::snprintf(m, sizeof m,
                      "grid barrier wait timed out after step %d of a launch (%d of %d blocks had arrived, waited %d "
                      "us); the batch state is undefined",
                      b->h_err[1], b->h_err[2], b->grid_blocks + b->extra_arrivals, b->h_err[3]);
        return bfail(CDF_ETIMEOUT, m);
    }
    return CDF_OK;
}

// (mode, tile or chain block, tile height of mode 2); a chain block with z == 2
// names the paired-lane two-step kernel
struct ModeChoice {
    int mode;
    dim3 shape;
    int th;
};
std::map<TuneKey, ModeChoice> g_bmode;

cdf_status bautotune(cdf_batch *b) {
    TuneKey key{b->nodes, (long long)b->count, b->m, b->params[0].chemotaxis};
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        auto it = g_bmode.find(key);
        if (it != g_bmode.end() && (it->second.mode != 2 || chain_pair_fits(b, it->second.shape, it->second.th))) {
            b->mode = it->second.mode;
            if (b->mode >= 1) {
                set_chain_block(b, it->second.shape);
                b->chain_th = it->second.th;
                return setup_tiles(b, dim3(64, 4));
            }
            return setup_tiles(b, it->second.shape);
        }
    }
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    float best = 1e30f;
    ModeChoice choice{0, dim3(64, 4), 0};
    const int steps = b->nodes > (1 << 22) ? 4 : 16;
    auto time_it = [&](auto &&run, int nsteps) -> float {
        if (run(nsteps) != CDF_OK) return -1.f;  // warm-up (and graph capture)
        if (cudaEventRecord(e0, b->s) != cudaSuccess) return -1.f;
        if (run(nsteps) != CDF_OK) return -1.f;
        if (cudaEventRecord(e1, b->s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        if (check_err(b) != CDF_OK) return -1.f;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const dim3 tiles[] = {dim3(32, 4), dim3(32, 8), dim3(64, 2), dim3(64, 4), dim3(128, 1), dim3(128, 2),
                          dim3(256, 1)};
    for (const dim3 &c : tiles) {
        cdf_status st = setup_tiles(b, c);
        if (st != CDF_OK) return st;
        float ms = time_it([&](int n) { return launch_batch(b, n, false); }, steps);
        if (ms < 0) return bfail(CDF_ECUDA, "autotuning the persistent kernel failed");
        ms *= (float)kChainGraphSteps / steps;  // per 32 steps, comparable with the chains
        if (ms < best) { best = ms; choice = {0, c, 0}; }
    }
    const dim3 blocks[] = {dim3(128, 1), dim3(128, 2), dim3(256, 1), dim3(64, 4), dim3(32, 8), dim3(128, 0),
                           dim3(256, 0)};  // y == 0: flat launch
    b->mode = 1;
    for (const dim3 &c : blocks) {
        set_chain_block(b, c);
        float ms = time_it([&](int n) { return run_chains(b, n, false); }, kChainGraphSteps);
        if (ms < 0) return bfail(CDF_ECUDA, "autotuning the kernel chains failed");
        if (ms < best) { best = ms; choice = {1, c, 0}; }
    }
    // chains of two-step launches: CTA shape and tile height (the paired-lane
    // kernel, chain_lanes = 2, measured slower on GB300 and is not timed here)
    const std::pair<dim3, int> pairs[] = {{dim3(32, 8), 14}, {dim3(32, 8), 6}, {dim3(32, 16), 14},
                                          {dim3(64, 8), 14}, {dim3(32, 16), 30}};
    b->mode = 2;
    for (const auto &c : pairs) {
        if (!chain_pair_fits(b, c.first, c.second)) continue;
        set_chain_block(b, c.first);
        b->chain_th = c.second;
        float ms = time_it([&](int n) { return run_chains(b, n, false); }, kChainGraphSteps);
        if (ms < 0) return bfail(CDF_ECUDA, "autotuning the two-step kernel chains failed");
        if (ms < best) { best = ms; choice = {2, c.first, c.second}; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->t = 0;
    b->cur = 0;
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        g_bmode[key] = choice;
    }
    b->mode = choice.mode;
    if (b->mode >= 1) {
        set_chain_block(b, choice.shape);
        b->chain_th = choice.th;
        return setup_tiles(b, dim3(64, 4));
    }
    return setup_tiles(b, choice.shape);
}

}  // namespace

extern "C" {

cdf_status cdf_batch_create(int count, const cdf_grid *grids, int m, const cdf_diffusion *diffusion, const double *nu,
                            const cdf_source *source, const cdf_force *force, const cdf_boundaries *boundaries,
                            const double *phi_ref, const double *p_ref_grad, const cdf_batch_options *opt,
                            cdf_batch **out) {
    if (!out) return bfail(CDF_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !grids || !diffusion || !nu || !source || !force || !boundaries || !phi_ref || !p_ref_grad || !opt)
        return bfail(CDF_EINVAL, "NULL argument or count < 1");
    if (opt->storage != CDF_FP32) return bfail(CDF_EINVAL, "the batched solver stores FP32 populations only");
    if (!(opt->rho0 > 0.0)) return bfail(CDF_EINVAL, "rho0 must be positive");
    if (opt->mode < 0 || opt->mode > 2) return bfail(CDF_EINVAL, "mode must be 0, 1 or 2");
    if ((opt->tile_x != 0 || opt->tile_y != 0) && opt->mode != 2) {
        if (opt->tile_x <= 0 || opt->tile_y <= 0 || opt->tile_x * opt->tile_y > 256 || opt->tile_x % 32 != 0)
            return bfail(CDF_EINVAL, "tile must be a multiple of 32 wide and at most 256 nodes");
    }
    if (opt->steps_per_launch < 0 || opt->barrier_timeout_s < 0) return bfail(CDF_EINVAL, "bad launch options");
    cdf_batch *b = new (std::nothrow) cdf_batch;
    if (!b) return bfail(CDF_ENOMEM, "host allocation failed");
    b->count = count;
    b->m = m;
    b->params.resize(count);
    int sprev_planes = -1;
    for (int k = 0; k < count; ++k) {
        const int pitch = grids[k].nx >= 1 ? (grids[k].nx + 31) / 32 * 32 : 0;
        cdf_status st = build_params(&grids[k], m, &diffusion[k], nu[k], &source[k], &force[k], &boundaries[k], false,
                                     opt->rho0, phi_ref + (size_t)k * m, p_ref_grad + 2 * (size_t)k, pitch,
                                     &b->params[k]);
        if (st != CDF_OK) {
            delete b;
            return st;
        }
        const int spp = source[k].kind == CDF_S_CONSUMPTION ? 1 : 0;
        if (sprev_planes >= 0 && spp != sprev_planes) {
            delete b;
            return bfail(CDF_EINVAL, "all instances must use the same source kind");
        }
        sprev_planes = spp;
        b->pop_off.push_back(b->pop_total);
        b->sp_off.push_back(b->sp_total);
        b->mom_off.push_back(b->mom_total);
        const long long plane = b->params[k].plane;
        b->pop_total += (long long)(9 + 5 * m) * plane;
        b->sp_total += plane;
        b->mom_total += (long long)(m + 3) * plane;
        b->nodes += (long long)grids[k].nx * grids[k].ny;
        b->stage_floats = std::max(b->stage_floats, (size_t)(m + 3) * grids[k].nx * grids[k].ny);
    }
    b->sprev_planes = sprev_planes;
    b->steps_per_launch = opt->steps_per_launch > 0 ? opt->steps_per_launch : 32;
    b->timeout_ns = opt->barrier_timeout_s > 0 ? (unsigned long long)(opt->barrier_timeout_s * 1e9) : 1000000000ull;
    b->extra_arrivals = opt->test_unreachable_barrier ? 1 : 0;
    b->user = static_cast<cudaStream_t>(opt->cuda_stream);
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return bfail(CDF_ECUDA, "no CUDA device"); }
    bool ok = dev_alloc((void **)&b->buf[0], b->pop_total * 4) == cudaSuccess &&
              dev_alloc((void **)&b->buf[1], b->pop_total * 4) == cudaSuccess &&
              dev_alloc((void **)&b->sprev, b->sp_total * 4) == cudaSuccess &&
              dev_alloc((void **)&b->sprev2, b->sp_total * 4) == cudaSuccess &&
              dev_alloc((void **)&b->mom, b->mom_total * 4) == cudaSuccess &&
              dev_alloc((void **)&b->mom_prev, b->mom_total * 4) == cudaSuccess &&
              cudaMalloc(&b->partials, (size_t)reduce_quantities(m) * kReduceBlocks * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&b->red, (size_t)count * reduce_quantities(m) * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&b->red_host, (size_t)count * reduce_quantities(m) * sizeof(double)) == cudaSuccess &&
              dev_alloc((void **)&b->dense, b->stage_floats * 4) == cudaSuccess &&
              cudaMalloc(&b->d_inst, count * sizeof(BatchInst)) == cudaSuccess &&
              cudaMalloc(&b->d_bar, 2 * sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&b->d_err, 4 * sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&b->h_err, 4 * sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&b->host_stage, b->stage_floats * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        brelease(b);
        return bfail(CDF_ENOMEM, "device allocation failed");
    }
    std::memset(b->h_err, 0, 4 * sizeof(int));  // read after every step call, also in the chain modes
    if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaMemset(b->buf[0], 0, b->pop_total * 4) != cudaSuccess || cudaMemset(b->buf[1], 0, b->pop_total * 4) != cudaSuccess ||
        cudaMemset(b->sprev, 0, b->sp_total * 4) != cudaSuccess || cudaMemset(b->sprev2, 0, b->sp_total * 4) != cudaSuccess ||
        cudaMemset(b->mom, 0, b->mom_total * 4) != cudaSuccess ||
        cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned)) != cudaSuccess) {
        brelease(b);
        return bfail(CDF_ECUDA, "stream / memory set-up failed");
    }
    b->pool.resize(std::min(count, kPoolStreams));
    b->ev_join.resize(b->pool.size());
    bool pok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (size_t j = 0; j < b->pool.size() && pok; ++j)
        pok = cudaStreamCreateWithFlags(&b->pool[j], cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_join[j], cudaEventDisableTiming) == cudaSuccess;
    if (!pok) {
        brelease(b);
        return bfail(CDF_ECUDA, "stream pool set-up failed");
    }
    b->mode = opt->mode;
    if (opt->chain_lanes < 0 || opt->chain_lanes > 2 || (opt->chain_lanes == 2 && !(opt->mode == 2 && opt->tile_x > 0))) {
        brelease(b);
        return bfail(CDF_EINVAL, "chain_lanes: 0, 1, or 2 with mode 2 and a given tile");
    }
    if (opt->mode >= 1 && opt->tile_x > 0)
        set_chain_block(b, dim3(opt->tile_x, opt->tile_y, opt->mode == 2 && opt->chain_lanes == 2 ? 2 : 1));
    if (opt->mode == 2 && opt->tile_x > 0) {
        b->chain_th = opt->chain_tile_y > 0 ? opt->chain_tile_y : 14;
        if (!chain_pair_fits(b, b->chain_block, b->chain_th)) {
            brelease(b);
            return bfail(CDF_EINVAL, "the two-step kernel shape cannot run every instance");
        }
    }
    cdf_status st;
    if (opt->mode >= 1 && opt->tile_x > 0) st = setup_tiles(b, dim3(64, 4));
    else if (opt->tile_x > 0) st = setup_tiles(b, dim3(opt->tile_x, opt->tile_y));
    else if (b->extra_arrivals) st = setup_tiles(b, dim3(64, 4));
    else st = bautotune(b);
    if (st == CDF_OK && cudaStreamSynchronize(b->s) != cudaSuccess) st = bfail(CDF_ECUDA, "set-up failed");
    if (st != CDF_OK) {
        brelease(b);
        return st;
    }
    *out = b;
    return CDF_OK;
}

void cdf_batch_destroy(cdf_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->s);
    brelease(b);
}

cdf_status cdf_batch_init_moments(cdf_batch *b, int k, const double *phi, const double *u, const double *p) {
    if (!b || !phi || !u || k < 0 || k >= b->count) return bfail(CDF_EINVAL, "bad argument");
    const LbParams &P = b->params[k];
    const size_t n = (size_t)P.nx * P.ny;
    BCK(cudaStreamSynchronize(b->s));  // the staging buffer may still feed a copy
    float *h = b->host_stage;
    for (int a = 0; a < b->m; ++a)
        for (size_t i = 0; i < n; ++i) h[a * n + i] = (float)phi[a * n + i];
    for (size_t i = 0; i < 2 * n; ++i) h[b->m * n + i] = (float)u[i];
    for (size_t i = 0; i < n; ++i) h[(b->m + 2) * n + i] = p ? (float)p[i] : 0.f;
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    BCK(cudaMemcpyAsync(b->dense, h, (size_t)(b->m + 3) * n * 4, cudaMemcpyHostToDevice, b->s));
    BCK(launch_init(P, kFP32, b->dense, P.nx, b->buf[b->cur] + b->pop_off[k], sprev_of(b, b->cur) + b->sp_off[k],
                    b->mom + b->mom_off[k], b->s));
    BCK(cudaEventRecord(b->ev_out, b->s));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CDF_OK;
}

cdf_status cdf_batch_step(cdf_batch *b, long long n) {
    if (!b || n < 0) return bfail(CDF_EINVAL, "bad argument");
    if (n == 0) return CDF_OK;
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    while (n > 0) {
        const int k = (int)std::min<long long>(n, b->mode >= 1 ? kChainGraphSteps : b->steps_per_launch);
        cdf_status st = b->mode >= 1 ? run_chains(b, k, n == k) : launch_batch(b, k, n == k);
        if (st != CDF_OK) return st;
        n -= k;
    }
    BCK(cudaStreamSynchronize(b->s));  // the barrier's error flag is read on the host
    cdf_status st = check_err(b);
    if (st != CDF_OK) return st;
    if ((st = checks_verify(b->s)) != CDF_OK) return st;  // no-op unless built with -DCDF_CHECKS
    BCK(cudaEventRecord(b->ev_out, b->s));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CDF_OK;
}

// Instances [k0, k1) of a device call: one instance, or all of them for k = -1.
static bool batch_range(const cdf_batch *b, int k, int *k0, int *k1) {
    if (k == -1) {
        *k0 = 0;
        *k1 = b->count;
        return true;
    }
    if (k < 0 || k >= b->count) return false;
    *k0 = k;
    *k1 = k + 1;
    return true;
}

cdf_status cdf_batch_init_moments_device(cdf_batch *b, int k, const float *dev_fields) {
    int k0, k1;
    if (!b || !dev_fields || !batch_range(b, k, &k0, &k1)) return bfail(CDF_EINVAL, "bad argument");
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    const float *src = dev_fields;
    for (int j = k0; j < k1; ++j) {
        const LbParams &P = b->params[j];
        BCK(launch_init(P, kFP32, src, P.nx, b->buf[b->cur] + b->pop_off[j], sprev_of(b, b->cur) + b->sp_off[j],
                        b->mom + b->mom_off[j], b->s));
        src += (size_t)(b->m + 3) * P.nx * P.ny;
    }
    BCK(cudaEventRecord(b->ev_out, b->s));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CDF_OK;
}

cdf_status cdf_batch_moments_device(cdf_batch *b, int k, float *dev_out) {
    int k0, k1;
    if (!b || !dev_out || !batch_range(b, k, &k0, &k1)) return bfail(CDF_EINVAL, "bad argument");
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    float *dst = dev_out;
    for (int j = k0; j < k1; ++j) {
        const LbParams &P = b->params[j];
        BCK(launch_pack_moments(P, b->mom + b->mom_off[j], dst, b->s));
        dst += (size_t)(b->m + 3) * P.nx * P.ny;
    }
    BCK(cudaEventRecord(b->ev_out, b->s));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CDF_OK;
}

cdf_status cdf_batch_moments(cdf_batch *b, int k, double *host_out) {
    if (!b || !host_out || k < 0 || k >= b->count) return bfail(CDF_EINVAL, "bad argument");
    const LbParams &P = b->params[k];
    const size_t n = (size_t)P.nx * P.ny * (b->m + 3);
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    BCK(launch_pack_moments(P, b->mom + b->mom_off[k], b->dense, b->s));
    BCK(cudaMemcpyAsync(b->host_stage, b->dense, n * 4, cudaMemcpyDeviceToHost, b->s));
    BCK(cudaStreamSynchronize(b->s));
    for (size_t i = 0; i < n; ++i) host_out[i] = b->host_stage[i];
    return CDF_OK;
}

cdf_status cdf_batch_get_info(const cdf_batch *b, cdf_batch_info *out) {
    if (!b || !out) return bfail(CDF_EINVAL, "NULL argument");
    out->count = b->count;
    out->m = b->m;
    out->nodes = b->nodes;
    out->tiles = b->total_tiles;
    out->tile_x = (int)b->tile.x;
    out->tile_y = (int)b->tile.y;
    out->grid_blocks = b->grid_blocks;
    out->steps_per_launch = b->steps_per_launch;
    out->bytes_per_lup = 2.0 * (9 + 5 * b->m) * 4.0 + 8.0 * b->sprev_planes;
    out->mode = b->mode;
    out->chain_block_x = (int)b->chain_block.x;
    out->chain_block_y = (int)b->chain_block.y;
    out->chain_tile_y = b->mode == 2 ? b->chain_th : 0;
    out->chain_lanes = b->mode >= 1 ? (int)b->chain_block.z : 1;
    out->t = b->t;
    return CDF_OK;
}

cdf_status cdf_batch_snapshot(cdf_batch *b) {
    if (!b) return bfail(CDF_EINVAL, "NULL handle");
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    BCK(cudaMemcpyAsync(b->mom_prev, b->mom, b->mom_total * 4, cudaMemcpyDeviceToDevice, b->s));
    BCK(cudaEventRecord(b->ev_out, b->s));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return CDF_OK;
}

cdf_status cdf_batch_residuals(cdf_batch *b, double *residual) {
    if (!b || !residual) return bfail(CDF_EINVAL, "NULL argument");
    const int nq = reduce_quantities(b->m), m = b->m;
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    for (int k = 0; k < b->count; ++k) {
        const LbParams &P = b->params[k];
        BCK(launch_reduce(b->mom + b->mom_off[k], b->mom_prev + b->mom_off[k], P.nx, P.ny, P.pitch, P.plane, m,
                          b->partials, b->red + (size_t)k * nq, b->s));
    }
    BCK(cudaMemcpyAsync(b->red_host, b->red, (size_t)b->count * nq * sizeof(double), cudaMemcpyDeviceToHost, b->s));
    BCK(cudaStreamSynchronize(b->s));
    for (int k = 0; k < b->count; ++k) {
        const double *q = b->red_host + (size_t)k * nq;
        double R = 0.0;
        for (int f = 0; f < m + 2; ++f) R = std::max(R, q[m + f] / std::max(q[2 * m + 2 + f], 1e-300));
        residual[k] = q[3 * m + 4] > 0 ? INFINITY : R;
    }
    return CDF_OK;
}

void *cdf_batch_stream(const cdf_batch *b) { return b ? static_cast<void *>(b->s) : nullptr; }

}  // extern "C"
