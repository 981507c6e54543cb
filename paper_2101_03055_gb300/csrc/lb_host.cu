// Host runtime behind the C ABI of include/cdf_lb.h: parameter checks and
// scaling, device buffers, stream ordering, CUDA-graph batches of fused steps,
// the steady-state driver with FP64 device reductions, checkpoints and the
// CTA-shape autotuner.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/cdf_lb.h"
#include "lb_internal.h"

using namespace cdflb;

namespace {

thread_local char g_err[512] = "";

cdf_status fail(cdf_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(CDF_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

// Keeps the caller's current device and restores it on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Gauss-Jordan inverse with partial pivoting (double).  false if singular.
bool invert(int n, const double *a_in, double *inv) {
    double a[kMaxM * kMaxM];
    for (int i = 0; i < n * n; ++i) a[i] = a_in[i];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = r == c ? 1.0 : 0.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
        if (!(std::fabs(a[piv * n + col]) > 1e-300)) return false;
        for (int c = 0; c < n; ++c) {
            std::swap(a[col * n + c], a[piv * n + c]);
            std::swap(inv[col * n + c], inv[piv * n + c]);
        }
        const double d = a[col * n + col];
        for (int c = 0; c < n; ++c) { a[col * n + c] /= d; inv[col * n + c] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = a[r * n + col];
            for (int c = 0; c < n; ++c) { a[r * n + c] -= f * a[col * n + c]; inv[r * n + c] -= f * inv[col * n + c]; }
        }
    }
    return true;
}

// Cholesky test of a symmetric matrix.
bool positive_definite(int n, const double *s) {
    double L[kMaxM * kMaxM] = {0};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = s[i * n + j];
            for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(v > 0.0)) return false;
                L[i * n + i] = std::sqrt(v);
            } else {
                L[i * n + j] = v / L[j * n + j];
            }
        }
    return true;
}

size_t elem_size(int storage) { return storage == CDF_FP32 ? 4 : 2; }

using TuneKey = std::tuple<int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, dim3> g_tune_cache;

// Steps per captured graph: a long graph for long calls (fewer gaps between
// graphs, 1.7 % on the 512 x 256 plume) and a short one for the rest of a call.
// Both even, so a graph returns the buffer parity it started with.
constexpr int kGraphSteps = 32;
constexpr int kGraphStepsLong = 256;

}  // namespace

struct cdf_lb {
    int device = 0;
    int nx = 0, ny = 0, m = 0, pitch = 0;
    long long plane = 0;
    int storage = 0;
    int planes = 0, sprev_planes = 0;
    LbParams P{};
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;  // buffer that holds the current post-collision populations
    // S_1(t - 1) of the consumption closure: two planes that alternate with the
    // population buffers (sprev_pp[cur] belongs to buf[cur]); a launch that
    // advances two steps reads halo nodes that other CTAs rewrite, so the
    // planes cannot be updated in place.
    float *sprev_pp[2] = {nullptr, nullptr};
    float *vel = nullptr;  // Case 1: prescribed velocity (2 planes) and two sets of m phi planes
    float *mom = nullptr, *mom_prev = nullptr;
    bool mr = false;                       // 16-bit storage: node-equilibrium deviations
    float *mom_pp[2] = {nullptr, nullptr};  // 16-bit storage: moments beside buf[0], buf[1]
    float *dense = nullptr;       // dense FP32 staging (export, host init)
    float *host_stage = nullptr;  // pinned host staging of one moment stack
    double *partials = nullptr, *red = nullptr, *red_host = nullptr;
    cudaStream_t s = nullptr;
    cudaStream_t user = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2][2][2] = {};  // [long][parity][moments]
    dim3 block{64, 4, 1};
    // Two time steps per launch (step2_kernel), FP32 storage: CTA shape and tile height.
    bool pair = false;
    dim3 pair_block{32, 16, 1};
    int pair_th = 30;
    // Tile-resident persistent step (FP32 lattices that fit in shared memory).
    bool resident = false;
    ResidentGeom rg{};
    unsigned *counters = nullptr;  // one step counter per tile
    int *d_err = nullptr, *h_err = nullptr;  // wait time-out flag (device, pinned copy)
    unsigned long long wait_ns = 1000000000ull;
    long long t = 0;
    bool initialised = false;
    int halo = 0;  // slab of a split lattice: bit 0 south halo row (y = 0), bit 1 north (y = ny - 1)
};

namespace {

void release(cdf_lb *h) {
    if (!h) return;
    DeviceGuard g(h->device);
    for (auto &size : h->graph)
        for (auto &row : size)
            for (auto &ge : row)
                if (ge) cudaGraphExecDestroy(ge);
    dev_free(h->buf[0]);
    dev_free(h->buf[1]);
    dev_free(h->sprev_pp[0]);
    dev_free(h->sprev_pp[1]);
    dev_free(h->vel);
    dev_free(h->mom);
    dev_free(h->mom_prev);
    dev_free(h->mom_pp[0]);
    dev_free(h->mom_pp[1]);
    dev_free(h->dense);
    cudaFree(h->counters);
    cudaFree(h->d_err);
    if (h->h_err) cudaFreeHost(h->h_err);
    dev_free(h->partials);
    dev_free(h->red);
    if (h->red_host) cudaFreeHost(h->red_host);
    if (h->host_stage) cudaFreeHost(h->host_stage);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->s) cudaStreamDestroy(h->s);
    delete h;
}

// Order the library stream after the caller's stream, and back.
cdf_status enter(cdf_lb *h) {
    CK(cudaEventRecord(h->ev_in, h->user));
    CK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
    return CDF_OK;
}
cdf_status leave(cdf_lb *h) {
    CK(cudaEventRecord(h->ev_out, h->s));
    CK(cudaStreamWaitEvent(h->user, h->ev_out, 0));
    return CDF_OK;
}

// Moments of the current time: FP32 storage writes them to `mom` on the last
// step of a call; 16-bit storage keeps them beside the current populations.
float *current_moments(cdf_lb *h) { return h->mr ? h->mom_pp[h->cur] : h->mom; }

// Case 1: the phi set that belongs to population buffer `par`.
float *phi_set(cdf_lb *h, int par) { return h->vel + (2 + (long long)par * h->m) * h->plane; }

// The step parameters for a launch reading buffer `src` (Case 1: its phi sets).
LbParams params_for(cdf_lb *h, int src) {
    LbParams p = h->P;
    if (p.case1) {
        p.php_in = phi_set(h, src);
        p.php_out = phi_set(h, src ^ 1);
    }
    return p;
}

cudaError_t launch_any(cdf_lb *h, int src, bool with_moments) {
    if (h->mr)
        return launch_step_mr(h->P, h->storage, h->buf[src], h->mom_pp[src], h->buf[src ^ 1], h->mom_pp[src ^ 1],
                              h->sprev_pp[src], h->sprev_pp[src ^ 1], h->block, h->s);
    return launch_step(params_for(h, src), h->storage, h->buf[src], h->buf[src ^ 1], h->sprev_pp[src],
                       h->sprev_pp[src ^ 1], with_moments ? h->mom : nullptr, h->block, h->s);
}

// Two steps from buf[src] to buf[src ^ 1] in one launch (16-bit storage keeps
// its moments beside the populations, so they are written every launch).
cudaError_t launch_two(cdf_lb *h, int src, bool with_moments) {
    if (h->mr)
        return launch_step2_mr(h->P, h->storage, h->buf[src], h->mom_pp[src], h->buf[src ^ 1], h->mom_pp[src ^ 1],
                               h->sprev_pp[src], h->sprev_pp[src ^ 1], h->pair_block, h->pair_th, h->s);
    return launch_step2(params_for(h, src), static_cast<const float *>(h->buf[src]),
                        static_cast<float *>(h->buf[src ^ 1]),
                        h->sprev_pp[src], h->sprev_pp[src ^ 1], with_moments ? h->mom : nullptr, h->pair_block,
                        h->pair_th, h->s);
}

cdf_status launch_one(cdf_lb *h, int src, bool with_moments) {
    CK(launch_any(h, src, with_moments));
    return CDF_OK;
}

cdf_status get_graph(cdf_lb *h, int lng, int parity, int with_moments, cudaGraphExec_t *out) {
    cudaGraphExec_t &slot = h->graph[lng][parity][with_moments];
    if (!slot) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
        int src = parity;
        const int steps = lng ? kGraphStepsLong : kGraphSteps;
        const int launches = h->pair ? steps / 2 : steps;  // even: the graph keeps the parity
        for (int k = 0; k < launches; ++k) {
            const bool wm = with_moments && k == launches - 1;
            cudaError_t e = h->pair ? launch_two(h, src, wm) : launch_any(h, src, wm);
            if (e != cudaSuccess) {
                cudaStreamEndCapture(h->s, &graph);
                if (graph) cudaGraphDestroy(graph);
                return fail(CDF_ECUDA, "step launch during capture: %s", cudaGetErrorString(e));
            }
            src ^= 1;
        }
        CK(cudaStreamEndCapture(h->s, &graph));
        cudaError_t e = cudaGraphInstantiate(&slot, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
    }
    *out = slot;
    return CDF_OK;
}

constexpr long long kResidentMaxSteps = 4096;  // steps per resident launch

// Zero the resident step counters and the time-out flag (after a new state).
cdf_status reset_resident(cdf_lb *h) {
    if (!h->resident) return CDF_OK;
    CK(cudaMemsetAsync(h->counters, 0, sizeof(unsigned) * h->rg.tiles_x * h->rg.tiles_y, h->s));
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    CK(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    return CDF_OK;
}

// After a stream synchronisation: did a wait of the resident step run out?
// The state is then undefined; the handle needs a new initial state.
cdf_status check_wait(cdf_lb *h) {
    if (!h->resident || !*h->h_err) return CDF_OK;
    *h->h_err = 0;
    h->initialised = false;
    reset_resident(h);
    cudaStreamSynchronize(h->s);
    return fail(CDF_ETIMEOUT, "a wait of the resident step timed out; the state is undefined (initialise again)");
}

cdf_status sync(cdf_lb *h) {
    CK(cudaStreamSynchronize(h->s));
    return check_wait(h);
}

// n steps on the library stream; the last one writes the moments.
cdf_status run_steps(cdf_lb *h, long long n) {
    while (h->resident && n > 0) {
        const int k = (int)std::min(n, kResidentMaxSteps);
        CK(launch_resident(h->P, h->rg, static_cast<float *>(h->buf[0]), static_cast<float *>(h->buf[1]),
                           h->sprev_pp[h->cur], h->sprev_pp[h->cur ^ (k & 1)], h->mom, k, h->cur, k == n,
                           h->counters, h->wait_ns, h->d_err, h->s));
        CK(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
        if (k & 1) h->cur ^= 1;
        h->t += k;
        n -= k;
    }
    while (n > 0) {
        if (n >= kGraphSteps) {
            const int lng = n >= kGraphStepsLong ? 1 : 0;
            const long long k = lng ? kGraphStepsLong : kGraphSteps;
            cudaGraphExec_t ge;
            cdf_status st = get_graph(h, lng, h->cur, n == k, &ge);
            if (st != CDF_OK) return st;
            CK(cudaGraphLaunch(ge, h->s));
            n -= k;
            h->t += k;
        } else {
            long long j = 0;
            for (; h->pair && j + 2 <= n; j += 2) {
                CK(launch_two(h, h->cur, j + 2 == n));
                h->cur ^= 1;
            }
            for (; j < n; ++j) {
                cdf_status st = launch_one(h, h->cur, j == n - 1);
                if (st != CDF_OK) return st;
                h->cur ^= 1;
            }
            h->t += n;
            n = 0;
        }
    }
    return CDF_OK;
}

// FP64 sums over the rows the step updates (a slab's halo rows belong to its
// neighbour and are left out).
cdf_status reduce(cdf_lb *h, const float *nw, const float *od, double *host_out) {
    const long long off = (long long)h->P.row_lo * h->pitch;
    CK(launch_reduce(nw + off, od ? od + off : nullptr, h->nx, h->P.row_hi - h->P.row_lo, h->pitch, h->plane,
                     h->m, h->partials, h->red, h->s));
    const int nq = reduce_quantities(h->m);
    CK(cudaMemcpyAsync(h->red_host, h->red, nq * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    cdf_status st = sync(h);
    if (st != CDF_OK) return st;
    std::memcpy(host_out, h->red_host, nq * sizeof(double));
    return CDF_OK;
}

std::map<TuneKey, bool> g_resident_cache;

// Time `steps` steps of the current mode on the library stream (ms).
cdf_status time_steps(cdf_lb *h, long long steps, float *ms) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    cdf_status st = run_steps(h, steps);  // warm-up (captures graphs)
    if (st == CDF_OK) {
        cudaEventRecord(a, h->s);
        st = run_steps(h, steps);
        cudaEventRecord(b, h->s);
    }
    cudaError_t e = cudaEventSynchronize(b);
    if (st == CDF_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != CDF_OK) return st;
    if (e != cudaSuccess) return fail(CDF_ECUDA, "timing failed: %s", cudaGetErrorString(e));
    return check_wait(h);
}

// Drop the captured step graphs (after a change of launch mode or shape).
void drop_graphs(cdf_lb *h) {
    for (auto &size : h->graph)
        for (auto &row : size)
            for (auto &ge : row)
                if (ge) {
                    cudaGraphExecDestroy(ge);
                    ge = nullptr;
                }
}

// Time the step kernel for a few CTA shapes on the (zeroed) buffers and keep the
// fastest; results are cached per (nx, ny, m, storage).  The shapes are timed
// through the path the steps run in (CUDA graphs of 32 launches): a short step
// launched one by one from the host would time the host's launch rate.
cdf_status autotune(cdf_lb *h) {
    TuneKey key{h->nx, h->ny, h->m, h->storage * 2 + h->P.case1, h->P.chemotaxis};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { h->block = it->second; return CDF_OK; }
    }
    // block.y == 0 marks a flat launch (one thread per node in row order)
    std::vector<dim3> cands = {dim3(32, 4), dim3(32, 8), dim3(64, 2), dim3(64, 4),
                               dim3(128, 1), dim3(128, 2), dim3(256, 1)};
    if (!h->mr && !h->P.case1) {
        // flat launches of several widths: a lattice that fills about one wave
        // is fastest when its nodes split evenly over the 152 SMs (e.g. 131,072
        // nodes in 1366 CTAs of 96 threads: nine CTAs on every SM)
        for (unsigned w : {64u, 96u, 128u, 160u, 192u, 224u, 256u}) cands.push_back(dim3(w, 0));
    }
    const long long nodes = (long long)h->nx * h->ny;
    const long long steps = nodes >= (1 << 22) ? 4 : 2 * kGraphSteps;
    float best = 1e30f;
    dim3 best_b = h->block;
    for (const dim3 &c : cands) {
        if ((int)c.x > 2 * h->nx && c.x > 32) continue;
        h->block = c;
        drop_graphs(h);
        float ms = 0.f;
        cdf_status st = time_steps(h, steps, &ms);
        if (st != CDF_OK) return st;
        if (ms < best) { best = ms; best_b = c; }
    }
    drop_graphs(h);
    h->block = best_b;
    h->cur = 0;
    h->t = 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_b;
    return CDF_OK;
}

// Can step2_kernel run this lattice with CTA shape b and tile height th?
// b.z == 2: the paired-lane kernel (step2_kernel_x2: FP32, m <= 2, full model,
// CTAs of 32 x 8, tile heights 14 and 30).
bool pair_fits(const cdf_lb *h, dim3 b, int th) {
    if (b.z == 2 && (h->mr || h->P.case1 || h->m > 2 || b.x != 32 || b.y != 8 || (th != 14 && th != 30)))
        return false;
    const int max_threads = h->mr ? step2_mr_max_threads(h->m) : step2_max_threads(h->m);
    if (b.x % 32 != 0 || b.x < 32 || (int)(b.x * b.y) > max_threads || th < 1) return false;
    if (step2_smem_bytes(h->m, b, th) > (size_t)kStep2MaxSmem) return false;
    if (h->P.periodic_x && h->nx < (int)b.x) return false;
    if (h->P.periodic_y && h->ny < th + 2) return false;
    return true;
}

// Decide whether two steps per launch (step2_kernel) run this lattice: always
// when asked for (with the best measured tile), never when refused, otherwise
// when a pair of steps measures faster than two launches of the step kernel.
// Results are cached per (nx, ny, m, storage, closure).
struct PairChoice {
    bool use;
    dim3 block;
    int th;
};
using PairKey = std::tuple<int, int, int, int, int, int>;  // + periodic axes
std::map<PairKey, PairChoice> g_pair_cache;

cdf_status setup_pair(cdf_lb *h, const cdf_options *opt) {
    // a fixed CTA shape of the step kernel fixes the one-step launch unless two
    // steps per launch are asked for explicitly
    if (opt->temporal == -1 || opt->resident == 1 || (opt->block_x > 0 && opt->temporal == 0)) return CDF_OK;
    if (opt->temporal_block_x > 0) {  // a given shape
        const dim3 b(opt->temporal_block_x, opt->temporal_block_y, opt->temporal_lanes == 2 ? 2 : 1);
        if (!pair_fits(h, b, opt->temporal_tile_y))
            return fail(CDF_EINVAL, "the two-step kernel shape %d x %d, tile height %d, cannot run this lattice",
                        opt->temporal_block_x, opt->temporal_block_y, opt->temporal_tile_y);
        h->pair = true;
        h->pair_block = b;
        h->pair_th = opt->temporal_tile_y;
        return CDF_OK;
    }
    PairKey key{h->nx, h->ny, (h->m * 4 + h->storage) * 2 + h->P.case1, h->P.chemotaxis, h->P.periodic_x,
                h->P.periodic_y};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_pair_cache.find(key);
        if (it != g_pair_cache.end()) {
            h->pair = opt->temporal == 1 || it->second.use;
            h->pair_block = it->second.block;
            h->pair_th = it->second.th;
            return CDF_OK;
        }
    }
    // candidates: R1 rows of 32 or 64 nodes, tile heights that give one or two
    // passes of the CTA's thread rows
    std::vector<std::pair<dim3, int>> cands;
    const long long nodes = (long long)h->nx * h->ny;
    if (nodes >= (1ll << 24)) {
        // a large lattice: a launch takes milliseconds, so time only the shapes that
        // measured best on large boxes (many small CTAs, or 512-thread CTAs)
        for (auto c : {std::make_pair(dim3(32, 8, 1), 14), std::make_pair(dim3(32, 16, 1), 30),
                       std::make_pair(dim3(64, 8, 1), 14)})
            if (pair_fits(h, c.first, c.second)) cands.push_back(c);
    } else {
        for (unsigned w : {32u, 64u})
            for (int th : {6, 14, 30, 32, 46, 62})
                for (unsigned by : {(unsigned)(th + 2), (unsigned)((th + 3) / 2), 8u, 16u}) {
                    const dim3 b(w, by, 1);
                    if (!pair_fits(h, b, th)) continue;
                    bool dup = false;
                    for (auto &c : cands)
                        dup = dup || (c.first.x == b.x && c.first.y == b.y && c.first.z == b.z && c.second == th);
                    if (!dup) cands.push_back({b, th});
                }
    }
    if (cands.empty()) {
        if (opt->temporal == 1) return fail(CDF_EINVAL, "the lattice is too small for two steps per launch");
        return CDF_OK;
    }
    // timed through the path the steps run in (CUDA graphs; see autotune)
    const long long steps = nodes >= (1 << 22) ? 4 : 2 * kGraphSteps;
    h->pair = false;
    drop_graphs(h);
    float t_single = 0.f;
    cdf_status st = time_steps(h, steps, &t_single);
    float best = 1e30f;
    PairChoice choice{false, h->pair_block, h->pair_th};
    for (size_t k = 0; st == CDF_OK && k < cands.size(); ++k) {
        h->pair = true;
        h->pair_block = cands[k].first;
        h->pair_th = cands[k].second;
        drop_graphs(h);
        float ms = 0.f;
        st = time_steps(h, steps, &ms);
        if (st == CDF_OK && ms < best) {
            best = ms;
            choice.block = cands[k].first;
            choice.th = cands[k].second;
        }
    }
    h->cur = 0;
    h->t = 0;
    if (st != CDF_OK) return st;
    const bool prefer = best < t_single;
    choice.use = opt->temporal == 1 || prefer;
    h->pair = choice.use;
    h->pair_block = choice.block;
    h->pair_th = choice.th;
    drop_graphs(h);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_pair_cache[key] = PairChoice{prefer, choice.block, choice.th};
    }
    // the timing ran on the zeroed buffers; the init calls set the state
    CK(cudaMemsetAsync(h->sprev_pp[0], 0, (size_t)h->plane * 4, h->s));
    CK(cudaMemsetAsync(h->sprev_pp[1], 0, (size_t)h->plane * 4, h->s));
    return CDF_OK;
}

// Decide whether the tile-resident step runs this lattice: always when asked
// for, never when refused or when the lattice does not fit, otherwise when it
// measures faster than the graph-launched kernel with the autotuned block.
cdf_status setup_resident(cdf_lb *h, const cdf_options *opt) {
    // two steps per launch asked for explicitly excludes the resident step
    if (h->storage != CDF_FP32 || opt->resident == -1 || h->P.case1 || (opt->temporal == 1 && opt->resident == 0))
        return CDF_OK;
    if (!plan_resident(h->nx, h->ny, h->m, &h->rg)) {
        cudaGetLastError();
        if (opt->resident == 1) return fail(CDF_EINVAL, "the lattice does not fit the resident step");
        return CDF_OK;
    }
    h->rg.stall_tile = opt->test_stall_tile - 1;
    h->wait_ns = opt->wait_timeout_s > 0 ? (unsigned long long)(opt->wait_timeout_s * 1e9) : 1000000000ull;
    const size_t tiles = (size_t)h->rg.tiles_x * h->rg.tiles_y;
    if (cudaMalloc((void **)&h->counters, tiles * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void **)&h->d_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(CDF_ENOMEM, "allocation of the resident step's counters failed");
    }
    *h->h_err = 0;
    h->resident = true;
    cdf_status st = reset_resident(h);
    if (st != CDF_OK || opt->resident == 1) return st;
    // opt->resident == 0: keep the faster mode (the tuner runs on the zeroed
    // buffers; the state is set by the init calls afterwards)
    TuneKey key{h->nx, h->ny, h->m, h->storage * 2 + h->P.case1, h->P.chemotaxis};
    bool use = false;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_resident_cache.find(key);
        if (it != g_resident_cache.end()) { use = it->second; cached = true; }
    }
    if (!cached) {
        float t_res = 0.f, t_graph = 0.f;
        const long long steps = 128;
        if ((st = time_steps(h, steps, &t_res)) != CDF_OK) return st;
        h->resident = false;
        if ((st = time_steps(h, steps, &t_graph)) != CDF_OK) return st;
        use = t_res < t_graph;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_resident_cache[key] = use;
    }
    h->resident = use;
    h->cur = 0;
    h->t = 0;
    return reset_resident(h);
}

cdf_status check_side_pair(const cdf_side &a, const cdf_side &b, const char *axis) {
    for (const cdf_side *s : {&a, &b})
        if (s->kind != CDF_BC_PERIODIC && s->kind != CDF_BC_WALL)
            return fail(CDF_EINVAL, "boundary kind must be CDF_BC_PERIODIC or CDF_BC_WALL");
    if (a.kind != b.kind)
        return fail(CDF_EINVAL, "opposite %s sides must both be periodic or both walls", axis);
    return CDF_OK;
}

}  // namespace

cdf_status cdflb::report_error(cdf_status status, const char *msg) {
    std::snprintf(g_err, sizeof g_err, "%s", msg);
    return status;
}

// Checks one lattice's parameter set and scales it for the kernels (shared by
// the single-lattice and the batched solver).  node_reference: 16-bit storage,
// whose deviations are taken from each node's own equilibrium.
cdf_status cdflb::build_params(const cdf_grid *grid, int m, const cdf_diffusion *dif, double nu,
                               const cdf_source *src, const cdf_force *frc, const cdf_boundaries *bc,
                               bool node_reference, double rho0, const double *phi_ref, const double *p_ref_grad,
                               int pitch, LbParams *out) {
    if (!grid || !dif || !src || !frc || !bc || !phi_ref || !p_ref_grad || !out) return fail(CDF_EINVAL, "NULL argument");
    if (grid->nx < 1 || grid->ny < 1) return fail(CDF_EINVAL, "grid must be at least 1 x 1");
    if ((long long)(grid->nx + 63) * grid->ny >= (1LL << 31) - 1)
        return fail(CDF_EINVAL, "grid too large: one padded plane must hold fewer than 2^31 elements");
    if (m < 1 || m > CDF_MAX_M) return fail(CDF_EINVAL, "m must be in [1, %d]", CDF_MAX_M);
    if (!(nu > 0.0) || !std::isfinite(nu)) return fail(CDF_EINVAL, "nu must be positive");
    if (dif->kind != CDF_D_CONST && dif->kind != CDF_D_CHEMOTAXIS) return fail(CDF_EINVAL, "bad diffusion kind");
    if (src->kind != CDF_S_NONE && src->kind != CDF_S_CONST && src->kind != CDF_S_CONSUMPTION)
        return fail(CDF_EINVAL, "bad source kind");
    if ((dif->kind == CDF_D_CHEMOTAXIS || src->kind == CDF_S_CONSUMPTION) && m < 2)
        return fail(CDF_EINVAL, "chemotaxis / consumption closures need m >= 2");
    for (int a = 0; a < m; ++a)
        if (!std::isfinite(phi_ref[a])) return fail(CDF_EINVAL, "phi_ref must be finite");
    if (!std::isfinite(p_ref_grad[0]) || !std::isfinite(p_ref_grad[1]))
        return fail(CDF_EINVAL, "p_ref_grad must be finite");
    cdf_status st;
    if ((st = check_side_pair(bc->west, bc->east, "x")) != CDF_OK) return st;
    if ((st = check_side_pair(bc->south, bc->north, "y")) != CDF_OK) return st;

    // Eq. omega-D with lambda = I, dt = 1: omega^-1 = D / cs^2 + I / 2 = 3 D + I / 2.
    double B[kMaxM * kMaxM], Binv[kMaxM * kMaxM], Bs[kMaxM * kMaxM];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            B[a * m + b] = 3.0 * dif->D[a * m + b] + (a == b ? 0.5 : 0.0);
            if (!std::isfinite(B[a * m + b])) return fail(CDF_EINVAL, "D has a non-finite entry");
        }
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) Bs[a * m + b] = 0.5 * (B[a * m + b] + B[b * m + a]);
    if (!positive_definite(m, Bs))
        return fail(CDF_EINVAL, "3 D + I/2 is not positive definite (no stable relaxation matrix)");
    if (!invert(m, B, Binv)) return fail(CDF_EINVAL, "3 D + I/2 is singular");
    if (dif->r_regularised && !(dif->eps > 0.0)) return fail(CDF_EINVAL, "regularised cut-off needs eps > 0");
    const cdf_side *sides[4] = {&bc->west, &bc->east, &bc->south, &bc->north};
    for (int s = 0; s < 4; ++s) {
        if (sides[s]->kind == CDF_BC_WALL && sides[s]->fluid != CDF_FL_NOSLIP && sides[s]->fluid != CDF_FL_FREESLIP)
            return fail(CDF_EINVAL, "bad fluid boundary kind");
        for (int a = 0; a < m; ++a) {
            if (sides[s]->scalar[a] != CDF_SC_NOFLUX && sides[s]->scalar[a] != CDF_SC_DIRICHLET)
                return fail(CDF_EINVAL, "bad scalar boundary kind");
            if (sides[s]->kind == CDF_BC_PERIODIC && sides[s]->scalar[a] == CDF_SC_DIRICHLET)
                return fail(CDF_EINVAL, "Dirichlet value on a periodic side");
        }
    }
    if (!(rho0 > 0.0)) return fail(CDF_EINVAL, "rho0 must be positive");
    LbParams &P = *out;
    P.nx = grid->nx;
    P.ny = grid->ny;
    P.pitch = pitch;
    P.plane = (long long)pitch * grid->ny;
    P.m = m;
    for (int i = 0; i < m * m; ++i) P.omega[i] = (float)Binv[i];
    P.omega_f = (float)(1.0 / (3.0 * nu + 0.5));
    P.chemotaxis = dif->kind == CDF_D_CHEMOTAXIS;
    P.chi3 = (float)(3.0 * dif->chi);
    P.c_star = (float)dif->c_star;
    P.eps2 = (float)(dif->eps * dif->eps);
    P.r_regularised = dif->r_regularised != 0;
    P.skind = src->kind;
    for (int a = 0; a < m; ++a) P.S[a] = (float)src->S[a];
    P.k = (float)src->k;
    P.g[0] = (float)frc->g[0];
    P.g[1] = (float)frc->g[1];
    double Fbase = frc->F0;
    for (int a = 0; a < m; ++a) {
        P.beta[a] = (float)frc->beta[a];
        Fbase -= frc->beta[a] * frc->phi_ref[a];
        P.phi_ref[a] = (float)phi_ref[a];
    }
    P.Fbase = (float)Fbase;
    if (!std::isfinite(frc->varphi)) return fail(CDF_EINVAL, "varphi must be finite");
    P.varphi = (float)frc->varphi;
    P.varphi_p = (float)(frc->varphi * 3.0 * nu * 4.0 / 3.0);  // (1/omega_f - 1/2) = 3 nu, W_0 / cs^2 = 4/3
    // Reference pressure gradient of the fluid deviations; a linear reference
    // cannot wrap around a periodic axis, so it is used along walled axes only.
    P.gref[0] = bc->west.kind == CDF_BC_WALL ? (float)p_ref_grad[0] : 0.f;
    P.gref[1] = bc->south.kind == CDF_BC_WALL ? (float)p_ref_grad[1] : 0.f;
    if (node_reference) {  // 16-bit storage references each node's own equilibrium instead
        for (int a = 0; a < m; ++a) P.phi_ref[a] = 0.f;
        P.gref[0] = P.gref[1] = 0.f;
    }
    P.xc = 0.5f * (float)(grid->nx - 1);
    P.yc = 0.5f * (float)(grid->ny - 1);
    P.row_lo = 0;
    P.row_hi = grid->ny;
    P.check = check_word();
    P.rho0 = (float)rho0;
    P.periodic_x = bc->west.kind == CDF_BC_PERIODIC;
    P.periodic_y = bc->south.kind == CDF_BC_PERIODIC;
    for (int s = 0; s < 4; ++s) {
        P.freeslip[s] = sides[s]->kind == CDF_BC_WALL && sides[s]->fluid == CDF_FL_FREESLIP;
        P.dirichlet[s] = 0;
        for (int a = 0; a < m; ++a) {
            if (sides[s]->kind == CDF_BC_WALL && sides[s]->scalar[a] == CDF_SC_DIRICHLET) {
                P.dirichlet[s] |= 1u << a;
                P.abb[s][a] = (float)((sides[s]->value[a] - P.phi_ref[a]) / 3.0);  // 2 W_i (phi_w - phi_ref)
            }
        }
    }

    return CDF_OK;
}

extern "C" {

const char *cdf_lb_last_error(void) { return g_err; }

cdf_status cdf_lb_create(const cdf_grid *grid, int m, const cdf_diffusion *dif, double nu,
                         const cdf_source *src, const cdf_force *frc, const cdf_boundaries *bc,
                         const cdf_options *opt, cdf_lb **out) {
    g_err[0] = 0;
    if (!out) return fail(CDF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !dif || !src || !frc || !bc || !opt) return fail(CDF_EINVAL, "NULL argument");
    if (opt->storage < CDF_FP32 || opt->storage > CDF_BF16_DEV) return fail(CDF_EINVAL, "bad storage");
    if (opt->resident < -1 || opt->resident > 1 || !(opt->wait_timeout_s >= 0.0) || opt->test_stall_tile < 0)
        return fail(CDF_EINVAL, "bad resident-step options");
    if (opt->resident == 1 && opt->storage != CDF_FP32)
        return fail(CDF_EINVAL, "the resident step exists for FP32 storage only");
    if (opt->prescribed_velocity != 0 && opt->prescribed_velocity != 1)
        return fail(CDF_EINVAL, "prescribed_velocity must be 0 or 1");
    if (opt->prescribed_velocity && opt->storage != CDF_FP32)
        return fail(CDF_EINVAL, "the prescribed-velocity mode (Case 1) stores FP32 populations");
    if (opt->prescribed_velocity && opt->resident == 1)
        return fail(CDF_EINVAL, "the resident step does not run the prescribed-velocity mode");
    if (opt->prescribed_velocity && (frc->g[0] != 0.0 || frc->g[1] != 0.0))
        return fail(CDF_EINVAL, "the prescribed-velocity mode has no force: set g = 0");
    if (!(opt->rho0 > 0.0)) return fail(CDF_EINVAL, "rho0 must be positive");
    if (opt->temporal < -1 || opt->temporal > 1) return fail(CDF_EINVAL, "temporal must be -1, 0 or 1");
    if (opt->temporal_lanes < 0 || opt->temporal_lanes > 2) return fail(CDF_EINVAL, "temporal_lanes must be 0, 1 or 2");
    if (opt->temporal_lanes == 2 && opt->temporal_block_x == 0)
        return fail(CDF_EINVAL, "temporal_lanes = 2 goes with a given two-step kernel shape (32 x 8, tile_y 14 or 30)");
    if (opt->temporal_block_x != 0 || opt->temporal_block_y != 0 || opt->temporal_tile_y != 0) {
        if (opt->temporal != 1) return fail(CDF_EINVAL, "a two-step kernel shape needs temporal = 1");
        if ((opt->temporal_block_x != 32 && opt->temporal_block_x != 64) || opt->temporal_block_y < 1 ||
            opt->temporal_tile_y < 1)
            return fail(CDF_EINVAL, "two-step kernel shape: block_x 32 or 64, block_y >= 1, tile_y >= 1");
    }
    if (opt->temporal == 1 && opt->resident == 1)
        return fail(CDF_EINVAL, "two steps per launch and the resident step exclude each other");
    if (opt->halo_rows < 0 || opt->halo_rows > 3) return fail(CDF_EINVAL, "halo_rows must be 0..3");
    if (opt->halo_rows) {
        if (opt->storage != CDF_FP32 || opt->prescribed_velocity)
            return fail(CDF_EINVAL, "a slab with halo rows runs the full model with FP32 storage");
        if (opt->resident == 1 || opt->temporal == 1)
            return fail(CDF_EINVAL, "a slab with halo rows runs one step per launch (resident = temporal = 0 or -1)");
        const int halos = (opt->halo_rows & 1) + (opt->halo_rows >> 1);
        if (grid->ny < halos + 1) return fail(CDF_EINVAL, "a slab needs at least one row besides its halo rows");
        const int nyg = opt->ny_global > 0 ? opt->ny_global : grid->ny;
        if (opt->origin_y < -1 || opt->origin_y + grid->ny - halos > nyg + 1)
            return fail(CDF_EINVAL, "origin_y / ny_global do not place the slab inside the lattice");
    } else if (opt->origin_y != 0 || opt->ny_global != 0) {
        return fail(CDF_EINVAL, "origin_y and ny_global belong to a slab (halo_rows != 0)");
    }
    LbParams P0{};
    const int align = opt->storage == CDF_FP32 ? 32 : 64;  // 128-byte rows
    const int pitch = grid->nx >= 1 ? (grid->nx + align - 1) / align * align : 0;
    cdf_status st = cdflb::build_params(grid, m, dif, nu, src, frc, bc, opt->storage != CDF_FP32, opt->rho0,
                                        opt->phi_ref, opt->p_ref_grad, pitch, &P0);
    if (st != CDF_OK) return st;
    if (opt->block_x != 0 || opt->block_y != 0) {
        const int threads = opt->block_x * (opt->block_y > 0 ? opt->block_y : 1);
        if (opt->block_x <= 0 || opt->block_y < 0 || threads > 256 || opt->block_x % 32 != 0)
            return fail(CDF_EINVAL, "block must be a multiple of 32 wide and at most 256 threads");
        if (opt->block_y == 0 && opt->storage != CDF_FP32)
            return fail(CDF_EINVAL, "the flat launch (block_y = 0) exists for FP32 storage only");
    }
    if (opt->block_lanes < 0 || opt->block_lanes > 2) return fail(CDF_EINVAL, "block_lanes must be 0, 1 or 2");
    if (opt->block_lanes == 2 && (opt->block_x <= 0 || opt->block_y != 0 || opt->storage != CDF_FP32 ||
                                  opt->prescribed_velocity || m > 2))
        return fail(CDF_EINVAL, "block_lanes = 2: a given flat launch (block_y = 0), FP32 storage, full model, m <= 2");

    cdf_lb *h = new (std::nothrow) cdf_lb;
    if (!h) return fail(CDF_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return fail(CDF_ECUDA, "no CUDA device"); }
    h->nx = grid->nx;
    h->ny = grid->ny;
    h->m = m;
    h->storage = opt->storage;
    h->pitch = pitch;
    h->plane = (long long)h->pitch * h->ny;
    h->planes = 9 + 5 * m;
    h->sprev_planes = src->kind == CDF_S_CONSUMPTION ? 1 : 0;
    h->mr = opt->storage != CDF_FP32;
    h->user = static_cast<cudaStream_t>(opt->cuda_stream);

    h->P = P0;
    h->P.case1 = opt->prescribed_velocity;
    if (opt->halo_rows) {
        // a slab: its halo rows are not updated, and its pressure reference is the
        // whole lattice's (centre of ny_global rows, local row 0 at global origin_y)
        h->P.row_lo = opt->halo_rows & 1 ? 1 : 0;
        h->P.row_hi = opt->halo_rows & 2 ? h->ny - 1 : h->ny;
        const int nyg = opt->ny_global > 0 ? opt->ny_global : h->ny;
        h->P.yc = (float)(0.5 * (nyg - 1) - opt->origin_y);
        h->halo = opt->halo_rows;
    }

    DeviceGuard g(h->device);
    const size_t esz = elem_size(h->storage);
    const size_t pop_bytes = (size_t)h->planes * h->plane * esz;
    const size_t n = (size_t)h->nx * h->ny;
    auto alloc = [&](void **p, size_t bytes) -> bool { return dev_alloc(p, bytes) == cudaSuccess; };
    bool ok = alloc(&h->buf[0], pop_bytes) && alloc(&h->buf[1], pop_bytes) &&
              alloc((void **)&h->sprev_pp[0], (size_t)h->plane * 4) &&
              alloc((void **)&h->sprev_pp[1], (size_t)h->plane * 4) &&
              (!h->P.case1 || alloc((void **)&h->vel, (size_t)(2 + 2 * m) * h->plane * 4)) &&
              alloc((void **)&h->mom, (size_t)(m + 3) * h->plane * 4) &&
              alloc((void **)&h->mom_prev, (size_t)(m + 3) * h->plane * 4) &&
              (!h->mr || (alloc((void **)&h->mom_pp[0], (size_t)(m + 3) * h->plane * 4) &&
                          alloc((void **)&h->mom_pp[1], (size_t)(m + 3) * h->plane * 4))) &&
              alloc((void **)&h->dense, (size_t)h->planes * n * 4) &&
              alloc((void **)&h->partials, (size_t)reduce_quantities(m) * kReduceBlocks * sizeof(double)) &&
              alloc((void **)&h->red, (size_t)reduce_quantities(m) * sizeof(double)) &&
              cudaMallocHost((void **)&h->red_host, (size_t)reduce_quantities(m) * sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void **)&h->host_stage, (size_t)(m + 3) * n * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(h);
        return fail(CDF_ENOMEM, "device allocation of %.1f MB failed", 2.0 * pop_bytes / 1e6);
    }
    h->P.vel = h->vel;
    if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        release(h);
        return fail(CDF_ECUDA, "stream/event creation failed");
    }
    if (cudaMemsetAsync(h->buf[0], 0, pop_bytes, h->s) != cudaSuccess ||
        cudaMemsetAsync(h->buf[1], 0, pop_bytes, h->s) != cudaSuccess ||
        cudaMemsetAsync(h->sprev_pp[0], 0, (size_t)h->plane * 4, h->s) != cudaSuccess ||
        cudaMemsetAsync(h->sprev_pp[1], 0, (size_t)h->plane * 4, h->s) != cudaSuccess ||
        cudaMemsetAsync(h->mom, 0, (size_t)(m + 3) * h->plane * 4, h->s) != cudaSuccess ||
        (h->mr && (cudaMemsetAsync(h->mom_pp[0], 0, (size_t)(m + 3) * h->plane * 4, h->s) != cudaSuccess ||
                   cudaMemsetAsync(h->mom_pp[1], 0, (size_t)(m + 3) * h->plane * 4, h->s) != cudaSuccess))) {
        release(h);
        return fail(CDF_ECUDA, "memset failed");
    }
    if (opt->block_x > 0) {
        h->block = dim3(opt->block_x, opt->block_y, opt->block_lanes == 2 ? 2 : 1);
    } else if ((st = autotune(h)) != CDF_OK) {
        release(h);
        return st;
    }
    // a slab runs one step per launch: its halo rows are refreshed between steps
    if (!h->halo && ((st = setup_pair(h, opt)) != CDF_OK || (st = setup_resident(h, opt)) != CDF_OK)) {
        release(h);
        return st;
    }
    if (cudaStreamSynchronize(h->s) != cudaSuccess) {
        release(h);
        return fail(CDF_ECUDA, "set-up failed");
    }
    *out = h;
    return CDF_OK;
}

void cdf_lb_destroy(cdf_lb *h) {
    if (!h) return;
    {
        DeviceGuard g(h->device);
        cudaStreamSynchronize(h->s);
    }
    release(h);
}

static cdf_status init_from_device_fields(cdf_lb *h, const float *fields) {
    if (h->mr) {
        CK(launch_init_mr(h->P, h->storage, fields, h->nx, h->buf[0], h->mom_pp[0], h->sprev_pp[0], h->s));
    } else {
        LbParams pi = h->P;  // Case 1: phi(t - 1) = phi0 goes to the set of buf[0]
        if (pi.case1) pi.php_out = phi_set(h, 0);
        CK(launch_init(pi, h->storage, fields, h->nx, h->buf[0], h->sprev_pp[0], h->mom, h->s));
    }
    h->cur = 0;
    h->t = 0;
    h->initialised = true;
    return reset_resident(h);
}

cdf_status cdf_lb_init_moments(cdf_lb *h, const double *phi, const double *u, const double *p) {
    g_err[0] = 0;
    if (!h || !phi || !u) return fail(CDF_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    const size_t n = (size_t)h->nx * h->ny;
    // The pinned staging buffer may still feed an earlier copy.
    CK(cudaStreamSynchronize(h->s));
    float *host = h->host_stage;
    for (int a = 0; a < h->m; ++a)
        for (size_t i = 0; i < n; ++i) host[a * n + i] = (float)phi[a * n + i];
    for (size_t i = 0; i < 2 * n; ++i) host[h->m * n + i] = (float)u[i];
    for (size_t i = 0; i < n; ++i) host[(h->m + 2) * n + i] = p ? (float)p[i] : 0.f;
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    CK(cudaMemcpyAsync(h->dense, host, (size_t)(h->m + 3) * n * 4, cudaMemcpyHostToDevice, h->s));
    if ((st = init_from_device_fields(h, h->dense)) != CDF_OK) return st;
    return leave(h);
}

cdf_status cdf_lb_init_moments_device(cdf_lb *h, const float *dev_fields) {
    g_err[0] = 0;
    if (!h || !dev_fields) return fail(CDF_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    if ((st = init_from_device_fields(h, dev_fields)) != CDF_OK) return st;
    return leave(h);
}

cdf_status cdf_lb_step(cdf_lb *h, long long n) {
    g_err[0] = 0;
    if (!h) return fail(CDF_EINVAL, "NULL handle");
    if (n < 0) return fail(CDF_EINVAL, "n must be >= 0");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    if (n == 0) return CDF_OK;
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    if ((st = run_steps(h, n)) != CDF_OK) return st;
    if ((st = checks_verify(h->s)) != CDF_OK) return st;  // no-op unless built with -DCDF_CHECKS
    return leave(h);
}

cdf_status cdf_lb_run_to_steady(cdf_lb *h, double tol, long long check_every, long long max_steps,
                                long long *steps_taken, double *residual) {
    g_err[0] = 0;
    if (!h) return fail(CDF_EINVAL, "NULL handle");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    if (check_every < 1 || max_steps < 0 || !(tol > 0.0)) return fail(CDF_EINVAL, "bad tol / check_every / max_steps");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    const int m = h->m;
    const size_t mom_bytes = (size_t)(m + 3) * h->plane * 4;
    double q[3 * kMaxM + 5];
    long long taken = 0;
    double R = INFINITY;
    cdf_status result = CDF_ENOTCONVERGED;
    while (taken < max_steps) {
        CK(cudaMemcpyAsync(h->mom_prev, current_moments(h), mom_bytes, cudaMemcpyDeviceToDevice, h->s));
        const long long k = std::min(check_every, max_steps - taken);
        if ((st = run_steps(h, k)) != CDF_OK) return st;
        taken += k;
        if ((st = reduce(h, current_moments(h), h->mom_prev, q)) != CDF_OK) return st;
        if (q[3 * m + 4] > 0) { result = CDF_EUNSTABLE; break; }
        R = 0.0;
        for (int f = 0; f < m + 2; ++f) {
            const double den = std::max(q[2 * m + 2 + f], 1e-300);
            R = std::max(R, q[m + f] / den);
        }
        if (k == check_every && R < tol) { result = CDF_OK; break; }
    }
    if (steps_taken) *steps_taken = taken;
    if (residual) *residual = R;
    if ((st = checks_verify(h->s)) != CDF_OK) return st;  // no-op unless built with -DCDF_CHECKS
    if ((st = leave(h)) != CDF_OK) return st;
    if (result == CDF_EUNSTABLE) return fail(CDF_EUNSTABLE, "non-finite moments after %lld steps", taken);
    if (result == CDF_ENOTCONVERGED)
        return fail(CDF_ENOTCONVERGED, "residual %.3e above tol %.3e after %lld steps", R, tol, taken);
    return CDF_OK;
}

cdf_status cdf_lb_moments_device(cdf_lb *h, float *dev_out) {
    g_err[0] = 0;
    if (!h || !dev_out) return fail(CDF_EINVAL, "NULL argument");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    CK(launch_pack_moments(h->P, current_moments(h), dev_out, h->s));
    return leave(h);
}

cdf_status cdf_lb_moments(cdf_lb *h, double *host_out) {
    g_err[0] = 0;
    if (!h || !host_out) return fail(CDF_EINVAL, "NULL argument");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    const size_t n = (size_t)h->nx * h->ny * (h->m + 3);
    CK(launch_pack_moments(h->P, current_moments(h), h->dense, h->s));
    CK(cudaMemcpyAsync(h->host_stage, h->dense, n * 4, cudaMemcpyDeviceToHost, h->s));
    if ((st = sync(h)) != CDF_OK) return st;
    for (size_t i = 0; i < n; ++i) host_out[i] = h->host_stage[i];
    return leave(h);
}

cdf_status cdf_lb_mass(cdf_lb *h, double *sums) {
    g_err[0] = 0;
    if (!h || !sums) return fail(CDF_EINVAL, "NULL argument");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    double q[3 * kMaxM + 5];
    if ((st = reduce(h, current_moments(h), nullptr, q)) != CDF_OK) return st;
    for (int a = 0; a < h->m; ++a) sums[a] = q[a];
    return leave(h);
}

// The planes that cross a cut, in buffer order: moving down (c_y = -1: h_4, h_7,
// h_8, then f_{a,4}) or up (c_y = +1: h_2, h_5, h_6, then f_{a,2}).
static int crossing_planes(int m, bool up, int *planes) {
    const int hp[2][3] = {{4, 7, 8}, {2, 5, 6}};
    int k = 0;
    for (int j = 0; j < 3; ++j) planes[k++] = hp[up][j];
    for (int a = 0; a < m; ++a) planes[k++] = 9 + 5 * a + (up ? 2 : 4);
    return k;
}

// One halo transfer of a slab: pack (row -> buffer) or unpack (buffer -> row).
static cdf_status halo_copy(cdf_lb *h, int side, float *buf, bool pack) {
    if (!h || !buf) return fail(CDF_EINVAL, "NULL argument");
    if (side != 0 && side != 1) return fail(CDF_EINVAL, "side must be 0 (south) or 1 (north)");
    if (!((h->halo >> side) & 1)) return fail(CDF_EINVAL, "the slab has no halo row on that side");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    // south: send the first updated row down, receive the halo row from below (moving up);
    // north: send the last updated row up, receive the halo row from above (moving down)
    const bool up = pack ? side == 1 : side == 0;
    const int row = pack ? (side == 0 ? h->P.row_lo : h->P.row_hi - 1) : (side == 0 ? 0 : h->ny - 1);
    int planes[3 + kMaxM];
    const int np = crossing_planes(h->m, up, planes);
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    float *pop = static_cast<float *>(h->buf[h->cur]);
    for (int k = 0; k < np; ++k) {
        float *r = pop + planes[k] * h->plane + (long long)row * h->pitch;
        float *b = buf + (long long)k * h->nx;
        CK(cudaMemcpyAsync(pack ? b : r, pack ? r : b, (size_t)h->nx * 4, cudaMemcpyDeviceToDevice, h->s));
    }
    return leave(h);
}

cdf_status cdf_lb_halo_pack(cdf_lb *h, int side, float *dev_buf) {
    g_err[0] = 0;
    return halo_copy(h, side, dev_buf, true);
}

cdf_status cdf_lb_halo_unpack(cdf_lb *h, int side, const float *dev_buf) {
    g_err[0] = 0;
    return halo_copy(h, side, const_cast<float *>(dev_buf), false);
}

cdf_status cdf_lb_snapshot(cdf_lb *h) {
    g_err[0] = 0;
    if (!h) return fail(CDF_EINVAL, "NULL handle");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    CK(cudaMemcpyAsync(h->mom_prev, current_moments(h), (size_t)(h->m + 3) * h->plane * 4,
                       cudaMemcpyDeviceToDevice, h->s));
    return leave(h);
}

cdf_status cdf_lb_change_sums(cdf_lb *h, double *sums) {
    g_err[0] = 0;
    if (!h || !sums) return fail(CDF_EINVAL, "NULL argument");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    if ((st = reduce(h, current_moments(h), h->mom_prev, sums)) != CDF_OK) return st;
    return leave(h);
}

cdf_status cdf_lb_wall_transfer(cdf_lb *h, int side, double D_CT, double S_TC, double T_wall, double C_wall,
                                double *out) {
    g_err[0] = 0;
    if (!h || !out) return fail(CDF_EINVAL, "NULL argument");
    if (side != 0 && side != 1) return fail(CDF_EINVAL, "side must be 0 (west) or 1 (east)");
    if (h->m < 2 || h->nx < 2) return fail(CDF_EINVAL, "needs m >= 2 (T, C) and nx >= 2");
    if (h->P.case1) return fail(CDF_EINVAL, "the wall transfer needs the full model's moments");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    const long long off = (long long)h->P.row_lo * h->pitch;
    CK(launch_wall_transfer(current_moments(h) + off, h->nx, h->P.row_hi - h->P.row_lo, h->pitch, h->plane, side,
                            D_CT, S_TC, T_wall, C_wall, h->red, h->s));
    CK(cudaMemcpyAsync(h->red_host, h->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    if ((st = sync(h)) != CDF_OK) return st;
    out[0] = h->red_host[0];
    out[1] = h->red_host[1];
    return leave(h);
}

cdf_status cdf_lb_populations(cdf_lb *h, double *f, double *hf, double *s_now) {
    g_err[0] = 0;
    if (!h) return fail(CDF_EINVAL, "NULL handle");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    const size_t n = (size_t)h->nx * h->ny;
    std::vector<float> tmp((size_t)h->planes * n), sp;
    if (h->mr)
        CK(launch_export_mr(h->P, h->storage, h->buf[h->cur], h->mom_pp[h->cur], h->dense, h->s));
    else
        CK(launch_export(h->P, h->storage, h->buf[h->cur], h->dense, h->s));
    CK(cudaMemcpyAsync(tmp.data(), h->dense, tmp.size() * 4, cudaMemcpyDeviceToHost, h->s));
    if (s_now && h->sprev_planes) {
        sp.resize((size_t)h->plane);
        CK(cudaMemcpyAsync(sp.data(), h->sprev_pp[h->cur], sp.size() * 4, cudaMemcpyDeviceToHost, h->s));
    }
    if ((st = sync(h)) != CDF_OK) return st;
    if (hf)
        for (size_t i = 0; i < 9 * n; ++i) hf[i] = tmp[i];
    if (f)
        for (size_t i = 0; i < (size_t)5 * h->m * n; ++i) f[i] = tmp[9 * n + i];
    if (s_now) {
        for (size_t i = 0; i < (size_t)h->m * n; ++i) s_now[i] = 0.0;
        if (h->sprev_planes)
            for (int y = 0; y < h->ny; ++y)
                for (int x = 0; x < h->nx; ++x) s_now[n + (size_t)y * h->nx + x] = sp[(size_t)y * h->pitch + x];
    }
    return leave(h);
}

namespace {
struct FileHeader {
    char magic[8];
    int version, nx, ny, m, storage, planes, sprev_planes, pitch;
    long long t;
    int cur;
    int reserved[5];
    float phi_ref[kMaxM], gref[2];
};
const char kMagic[8] = {'C', 'D', 'F', 'L', 'B', '0', '0', '1'};
}  // namespace

cdf_status cdf_lb_save(cdf_lb *h, const char *path) {
    g_err[0] = 0;
    if (!h || !path) return fail(CDF_EINVAL, "NULL argument");
    if (!h->initialised) return fail(CDF_EINVAL, "state not initialised");
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    const size_t pop = (size_t)h->planes * h->plane * elem_size(h->storage);
    const size_t spb = (size_t)h->plane * 4, momb = (size_t)(h->m + 3) * h->plane * 4;
    const size_t velb = h->P.case1 ? (size_t)(2 + h->m) * h->plane * 4 : 0;
    std::vector<char> data(pop + spb + momb + velb);
    CK(cudaMemcpyAsync(data.data(), h->buf[h->cur], pop, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(data.data() + pop, h->sprev_pp[h->cur], spb, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(data.data() + pop + spb, current_moments(h), momb, cudaMemcpyDeviceToHost, h->s));
    if (velb) {  // Case 1: the prescribed velocity and the current phi set
        const size_t ub = (size_t)2 * h->plane * 4;
        CK(cudaMemcpyAsync(data.data() + pop + spb + momb, h->vel, ub, cudaMemcpyDeviceToHost, h->s));
        CK(cudaMemcpyAsync(data.data() + pop + spb + momb + ub, phi_set(h, h->cur), velb - ub,
                           cudaMemcpyDeviceToHost, h->s));
    }
    if ((st = sync(h)) != CDF_OK) return st;
    FileHeader hd{};
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = 1;
    hd.nx = h->nx; hd.ny = h->ny; hd.m = h->m; hd.storage = h->storage;
    hd.planes = h->planes; hd.sprev_planes = h->sprev_planes; hd.pitch = h->pitch; hd.t = h->t;
    hd.reserved[0] = h->P.case1;
    for (int a = 0; a < kMaxM; ++a) hd.phi_ref[a] = h->P.phi_ref[a];
    hd.gref[0] = h->P.gref[0];
    hd.gref[1] = h->P.gref[1];
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(CDF_EIO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&hd, sizeof hd, 1, fp) == 1 && std::fwrite(data.data(), 1, data.size(), fp) == data.size();
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(CDF_EIO, "write to %s failed", path);
    return leave(h);
}

cdf_status cdf_lb_load(cdf_lb *h, const char *path) {
    g_err[0] = 0;
    if (!h || !path) return fail(CDF_EINVAL, "NULL argument");
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(CDF_EIO, "cannot open %s", path);
    FileHeader hd{};
    if (std::fread(&hd, sizeof hd, 1, fp) != 1 || std::memcmp(hd.magic, kMagic, 8) != 0) {
        std::fclose(fp);
        return fail(CDF_EIO, "%s is not a cdf_lb checkpoint", path);
    }
    if (hd.nx != h->nx || hd.ny != h->ny || hd.m != h->m || hd.storage != h->storage ||
        hd.planes != h->planes || hd.sprev_planes != h->sprev_planes || hd.pitch != h->pitch ||
        hd.reserved[0] != h->P.case1 ||
        std::memcmp(hd.phi_ref, h->P.phi_ref, sizeof hd.phi_ref) != 0 || hd.gref[0] != h->P.gref[0] ||
        hd.gref[1] != h->P.gref[1]) {
        std::fclose(fp);
        return fail(CDF_EINVAL, "checkpoint does not match this solver's grid, m, storage or reference state");
    }
    const size_t pop = (size_t)h->planes * h->plane * elem_size(h->storage);
    const size_t spb = (size_t)h->plane * 4, momb = (size_t)(h->m + 3) * h->plane * 4;
    const size_t velb = h->P.case1 ? (size_t)(2 + h->m) * h->plane * 4 : 0;
    std::vector<char> data(pop + spb + momb + velb);
    const bool ok = std::fread(data.data(), 1, data.size(), fp) == data.size();
    std::fclose(fp);
    if (!ok) return fail(CDF_EIO, "%s is truncated", path);
    DeviceGuard g(h->device);
    cdf_status st = enter(h);
    if (st != CDF_OK) return st;
    h->cur = 0;
    CK(cudaMemcpyAsync(h->buf[0], data.data(), pop, cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(h->sprev_pp[0], data.data() + pop, spb, cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(current_moments(h), data.data() + pop + spb, momb, cudaMemcpyHostToDevice, h->s));
    if (velb) {
        const size_t ub = (size_t)2 * h->plane * 4;
        CK(cudaMemcpyAsync(h->vel, data.data() + pop + spb + momb, ub, cudaMemcpyHostToDevice, h->s));
        CK(cudaMemcpyAsync(phi_set(h, 0), data.data() + pop + spb + momb + ub, velb - ub, cudaMemcpyHostToDevice,
                           h->s));
    }
    if ((st = reset_resident(h)) != CDF_OK) return st;
    CK(cudaStreamSynchronize(h->s));
    h->t = hd.t;
    h->initialised = true;
    return leave(h);
}

cdf_status cdf_lb_get_info(const cdf_lb *h, cdf_info *out) {
    if (!h || !out) return fail(CDF_EINVAL, "NULL argument");
    out->nx = h->nx; out->ny = h->ny; out->m = h->m; out->pitch = h->pitch;
    out->storage = h->storage; out->planes = h->planes; out->sprev_planes = h->sprev_planes;
    out->block_x = (int)h->block.x; out->block_y = (int)h->block.y;  // block_y 0: flat launch
    out->resident = h->resident ? 1 : 0;
    out->tile_x = h->resident ? h->rg.tw : 0;
    out->tile_y = h->resident ? h->rg.th : 0;
    out->tiles = h->resident ? h->rg.tiles_x * h->rg.tiles_y : 0;
    out->bytes_per_lup = 2.0 * h->planes * (double)elem_size(h->storage) + 8.0 * h->sprev_planes +
                         (h->mr ? 2.0 * 4.0 * (h->m + 3) : 0.0);
    if (h->P.case1)  // scalars read and written, u read, phi(t - 1) read and written
        out->bytes_per_lup = 2.0 * 5 * h->m * 4.0 + 8.0 + 8.0 * h->m + 8.0 * h->sprev_planes;
    out->t = h->t;
    out->temporal = h->pair ? 1 : 0;
    out->lanes = h->pair ? (int)h->pair_block.z : (h->resident ? 1 : (int)h->block.z);
    if (h->pair) {
        out->block_x = (int)h->pair_block.x;
        out->block_y = (int)h->pair_block.y;
        out->tile_x = (int)h->pair_block.x - 2;
        out->tile_y = h->pair_th;
        out->tiles = ((h->nx + out->tile_x - 1) / out->tile_x) * ((h->ny + h->pair_th - 1) / h->pair_th);
    }
    return CDF_OK;
}

void *cdf_lb_stream(const cdf_lb *h) { return h ? static_cast<void *>(h->s) : nullptr; }

}  // extern "C"
