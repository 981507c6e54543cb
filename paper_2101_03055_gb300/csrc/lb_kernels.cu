// Fused stream-and-collide kernels of the CDF lattice Boltzmann model
// (Zhan, Chai & Shi, arXiv:2101.03055) for sm_103a.
//
// One thread owns one lattice node.  A step pulls the post-collision
// populations of the previous step from the neighbours (x - c_i), substitutes
// the boundary rule where the link crosses a wall, forms the moments (Eqs.
// sum-phi, sum-u, sum-p), the closures and the relaxation matrix (Eq. omega-D),
// collides (Eqs. evolution12, evolution3 with Eqs. feq-phi, heq, force,
// source, Gi) and stores the new post-collision populations: one read and one
// write of every population per step, nothing else in HBM.
//
// Storage is structure-of-arrays: plane k holds population k of every node,
// rows padded to `pitch` elements (128-byte aligned rows).  Pull loads along
// x are shifted by one element; consecutive threads still read consecutive
// addresses, and the overlap between neighbouring warps is served from L1/L2.
#include "lb_device.cuh"

#include <atomic>
#include <type_traits>

namespace cdflb {
namespace {
using namespace dev;

// Launch a step kernel with programmatic stream serialisation (see
// pdl_wait_and_release): it may begin while the previous kernel of the stream
// finishes, and waits inside for that kernel's results.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    return launch_pdl_smem(kern, grid, block, 0, s, args...);
}

// One pointer per moment plane of the stacks `in` (read) and `out` (written).
MomentPlanes moments_of(const LbParams &p, const float *in, float *out) {
    MomentPlanes mp{};
    for (int k = 0; k < p.m + 3; ++k) {
        mp.in[k] = in + k * p.plane;
        mp.out[k] = out + k * p.plane;
    }
    return mp;
}

// One pointer per population plane of the buffers `in` (read) and `out` (written).
template <typename T>
Planes<T> planes_of(const LbParams &p, const T *in, T *out) {
    Planes<T> pl{};
    for (int k = 0; k < 9 + 5 * p.m; ++k) {
        pl.in[k] = in + k * p.plane;
        pl.out[k] = out + k * p.plane;
    }
    return pl;
}

// ---- the fused step ------------------------------------------------------------
template <int M, typename T>
__global__ void __launch_bounds__(256) step_kernel(const LbParams p, const Planes<T> pl, const float *sp_in,
                                                   float *sp_out, float *__restrict__ moments) {
    pdl_wait_and_release();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    // Warp-uniform choice (every CTA holds whole warps): a warp whose 32 nodes
    // all lie inside the boundary ring runs the pull without boundary selects.
    // (halo rows of a slab, y = 0 or ny - 1, are never inner nodes)
    if (__all_sync(0xffffffffu, inner_node(p, x, y)))
        step_node_planes<M, T, true>(p, x, y, pl, sp_in, sp_out, moments);
    else if (x < p.nx && y >= p.row_lo && y < p.row_hi)
        step_node_planes<M, T>(p, x, y, pl, sp_in, sp_out, moments);
}

// Flat launch: one thread per node over nx * ny (no idle threads in ragged rows).
template <int M, typename T>
__global__ void __launch_bounds__(256) step_kernel_flat(const LbParams p, const Planes<T> pl, const float *sp_in,
                                                        float *sp_out, float *__restrict__ moments) {
    pdl_wait_and_release();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = idx < p.nx * p.ny;
    const int y = idx / p.nx, x = idx - y * p.nx;
    if (__all_sync(0xffffffffu, valid && inner_node(p, x, y)))
        step_node_planes<M, T, true>(p, x, y, pl, sp_in, sp_out, moments);
    else if (valid && y >= p.row_lo && y < p.row_hi)
        step_node_planes<M, T>(p, x, y, pl, sp_in, sp_out, moments);
}

template <int M>
__device__ __forceinline__ void pack_node(const float (&f0)[M][5], const float (&h0)[9], const float (&f1)[M][5],
                                          const float (&h1)[9], F2 (&f)[M][5], F2 (&h)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = pack2(h0[i], h1[i]);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) f[a][i] = pack2(f0[a][i], f1[a][i]);
}

template <int M>
__device__ __forceinline__ NodeOut<M> lane_out(const NodeOut<M, F2> &o, int k) {
    NodeOut<M> r;
#pragma unroll
    for (int a = 0; a < M; ++a) r.phi[a] = lane(o.phi[a], k);
    r.ux = lane(o.ux, k);
    r.uy = lane(o.uy, k);
    r.pr = lane(o.pr, k);
    r.s1 = lane(o.s1, k);
    return r;
}

// Flat launch with two nodes per thread (paired FP32 lanes): thread t updates
// nodes t and t + half of the row-major order (half a multiple of 32, so the
// second nodes of a warp are a whole warp's worth of the order too).  The two
// nodes are pulled one after the other and collide together on paired FP32
// lanes (collide<M, F2>): each lane runs the scalar update's operations in the
// same order, so every node gets the bits of step_kernel_flat.  A lattice of
// about one wave is bound by the instructions each SM issues for its share of
// the nodes, which this halves for the arithmetic; where a lane has no node to
// update (past the end, or a slab's halo row) it repeats the other lane's node
// and its result is not stored.  FP32, m <= 2, full model.
template <int M>
__global__ void __launch_bounds__(256) step_kernel_flat_x2(const LbParams p, const Planes<float> pl,
                                                           const float *sp_in, float *sp_out,
                                                           float *__restrict__ moments, int half) {
    constexpr unsigned kAll = 0xffffffffu;
    pdl_wait_and_release();
    const int n = p.nx * p.ny, nx = p.nx;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x, i1 = i0 + half;
    bool ok[2];
    int xs[2], ys[2];
    ys[0] = i0 / nx;
    xs[0] = i0 - ys[0] * nx;
    ys[1] = i1 / nx;
    xs[1] = i1 - ys[1] * nx;
#pragma unroll
    for (int k = 0; k < 2; ++k) ok[k] = i0 < half && (k ? i1 : i0) < n && ys[k] >= p.row_lo && ys[k] < p.row_hi;
    const int ka = ok[0] ? 0 : 1, kb = ok[1] ? 1 : 0;  // a lane without a node repeats the other's
    const int xa = xs[ka], ya = ys[ka], xb = xs[kb], yb = ys[kb];
    const bool any = ok[0] || ok[1];
    const bool inta = __all_sync(kAll, any && inner_node(p, xa, ya));
    const bool intb = __all_sync(kAll, any && inner_node(p, xb, yb));
    if (!any) return;
    const int pitch = p.pitch;
    const auto mk = [pitch](int sx, int sy) { return sy * pitch + sx; };
    const auto ld = [&pl, &p](int plane, int off) { return __ldg(pl.in[plane] + CDF_CHK(p, off, p.plane, 1)); };
    float h0[9], f0[M][5], h1[9], f1[M][5];
    if (inta) pull_node<M, true>(p, xa, ya, mk, ld, f0, h0);
    else pull_node<M, false>(p, xa, ya, mk, ld, f0, h0);
    if (intb) pull_node<M, true>(p, xb, yb, mk, ld, f1, h1);
    else pull_node<M, false>(p, xb, yb, mk, ld, f1, h1);
    const int oa = CDF_CHK(p, ya * pitch + xa, p.plane, 2), ob = CDF_CHK(p, yb * pitch + xb, p.plane, 2);
    const bool consume = (M >= 2 && p.skind == 2);
    F2 h[9], f[M][5];
    pack_node<M>(f0, h0, f1, h1, f, h);
    NodeOut<M, F2> o;
    collide<M>(p, f, h, pack2(pref_at(p, xa, ya), pref_at(p, xb, yb)),
               consume ? pack2(sp_in[oa], sp_in[ob]) : splat<F2>(0.f), false, o);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!ok[k]) continue;
        const int o0 = k ? ob : oa;
#pragma unroll
        for (int i = 0; i < 9; ++i) pl.out[i][o0] = lane(h[i], k);
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int i = 0; i < 5; ++i) pl.out[9 + 5 * a + i][o0] = lane(f[a][i], k);
        if (consume) sp_out[o0] = lane(o.s1, k);
        if (moments) write_moments<M>(moments, p.plane, o0, lane_out<M>(o, k));
    }
}

// ---- two time steps per launch (temporal blocking), FP32 storage ----------------
// A small lattice lives in L2 between steps, and a one-step launch is then
// bound by one full pass over the state plus the launch gap.  Here a CTA of
// W1 x BY threads owns an output tile of (W1 - 2) x TH nodes and the region R1
// around it, W1 x (TH + 2) nodes with origin (X0 - 1, Y0 - 1) (wrapped on
// periodic axes).  Step t -> t+1: every R1 node that some tile node pulls from
// is updated from the global buffer `in` into shared memory (plane stride
// W1 (TH + 2), planes h_0..h_8, f_{a,0..4}, then S_1(t)); step t+1 -> t+2:
// every tile node pulls from shared memory and stores to `out`.  The halo ring
// is computed by both neighbouring CTAs, one pass over global memory serves
// two steps, and each node runs the same pull table and collision as
// step_kernel, so two launches of step_kernel and one of this kernel give the
// same bits.  Needs nx >= W1 on a periodic x axis and ny >= TH + 2 on a
// periodic y axis (a wrapped source must not land twice in R1).  S_1 is read
// from sp_in and written to sp_out, which must be different planes: the halo
// of one CTA is the tile of another.
// FW, FY, FT != 0: a copy for one CTA shape FW x FY and tile height FT (the
// launch must match; blockDim and the TH argument are then not read).  With the
// shape known, the shared-memory plane stride is a constant, every
// shared-memory access is a register plus an immediate offset and the row
// loops unroll; the node update is the same, so are the bits.
template <int M, int FW = 0, int FY = 0, int FT = 0>
__global__ void __launch_bounds__(FW ? FW * FY : step2_max_threads(M), FW ? step2_max_threads(M) / (FW * FY) : 1)
    step2_kernel(const LbParams p, int TH, const Planes<float> pl, const float *sp_in, float *sp_out,
                 float *__restrict__ moments) {
    constexpr int NP = 9 + 5 * M;
    extern __shared__ float sm[];
    pdl_wait_and_release();
    const int W1 = FW ? FW : (int)blockDim.x, BY = FY ? FY : (int)blockDim.y, THv = FT ? FT : TH;
    const int H1 = THv + 2, SP = W1 * H1, TW = W1 - 2;
    const int X0 = blockIdx.x * TW, Y0 = blockIdx.y * THv;
    const long long P = p.plane;
    const int pitch = p.pitch, nx = p.nx, ny = p.ny;
    const bool consume = M >= 2 && p.skind == 2;
    const int lx = threadIdx.x;

    // Column lx of R1: unwrapped x = X0 - 1 + lx.  It is needed when some tile
    // node (x < min(X0 + TW, nx)) pulls from it, and it exists when it lies in
    // the lattice or wraps on a periodic axis.
    const int xu = X0 - 1 + lx;
    const bool colv = xu <= min(X0 + TW, nx) && (p.periodic_x || (xu >= 0 && xu < nx));
    const int gx = xu < 0 ? xu + nx : (xu >= nx ? xu - nx : xu);

    // ---- step 1: R1 from global memory into shared memory
    {
        const auto mk = [pitch](int sx, int sy) { return sy * pitch + sx; };
        const auto ld = [&pl, &p, P](int plane, int off) { return __ldg(pl.in[plane] + CDF_CHK(p, off, P, 1)); };
#pragma unroll
        for (int ly = threadIdx.y; ly < H1; ly += BY) {
            const int yu = Y0 - 1 + ly;
            const bool ok = colv && yu <= min(Y0 + THv, ny) && (p.periodic_y || (yu >= 0 && yu < ny));
            const int gy = yu < 0 ? yu + ny : (yu >= ny ? yu - ny : yu);
            const bool general = ok && !inner_node(p, gx, gy);
            float h[9], f[M][5];
            if (!__any_sync(0xffffffffu, general)) {
                if (!ok) continue;
                pull_node<M, true>(p, gx, gy, mk, ld, f, h);
            } else {
                if (!ok) continue;
                pull_node<M, false>(p, gx, gy, mk, ld, f, h);
            }
            const int o0 = CDF_CHK(p, gy * pitch + gx, P, 2), l0 = CDF_CHK(p, ly * W1 + lx, SP, 3);
            NodeOut<M> o;
            collide<M>(p, f, h, pref_at(p, gx, gy), consume ? sp_in[o0] : 0.f, false, o);
#pragma unroll
            for (int i = 0; i < 9; ++i) sm[i * SP + l0] = h[i];
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int i = 0; i < 5; ++i) sm[(9 + 5 * a + i) * SP + l0] = f[a][i];
            if (consume) sm[NP * SP + l0] = o.s1;
        }
    }
    __syncthreads();

    // ---- step 2: the tile from shared memory into global memory
    const auto lds = [SP, &p](int plane, int off) { return sm[plane * SP + CDF_CHK(p, off, SP, 4)]; };
    // interior nodes pull from x - c_i without wrapping
    const auto mk_in = [W1, X0, Y0](int sx, int sy) { return (sy - Y0 + 1) * W1 + (sx - X0 + 1); };
    // general nodes: wrapped source coordinates back into R1
    const auto mk_gen = [W1, H1, X0, Y0, nx, ny](int sx, int sy) {
        int a = sx - X0 + 1, b = sy - Y0 + 1;
        a = a < 0 ? a + nx : (a >= W1 ? a - nx : a);
        b = b < 0 ? b + ny : (b >= H1 ? b - ny : b);
        return b * W1 + a;
    };
#pragma unroll
    for (int ly = 1 + threadIdx.y; ly <= THv; ly += BY) {
        const int x = xu, y = Y0 - 1 + ly;
        const bool ok = lx >= 1 && lx <= TW && x < nx && y < ny;
        const bool general = ok && !inner_node(p, x, y);
        float h[9], f[M][5];
        if (!__any_sync(0xffffffffu, general)) {
            if (!ok) continue;
            pull_node<M, true>(p, x, y, mk_in, lds, f, h);
        } else {
            if (!ok) continue;
            pull_node<M, false>(p, x, y, mk_gen, lds, f, h);
        }
        const int o0 = CDF_CHK(p, y * pitch + x, P, 2);
        NodeOut<M> o;
        collide<M>(p, f, h, pref_at(p, x, y), consume ? sm[NP * SP + CDF_CHK(p, ly * W1 + lx, SP, 4)] : 0.f, false, o);
#pragma unroll
        for (int i = 0; i < 9; ++i) pl.out[i][o0] = h[i];
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int i = 0; i < 5; ++i) pl.out[9 + 5 * a + i][o0] = f[a][i];
        if (consume) sp_out[o0] = o.s1;
        if (moments) write_moments<M>(moments, P, o0, o);
    }
}

// ---- two time steps per launch, two nodes per thread (paired FP32 lanes) ---------
// The tiling of step2_kernel for CTAs of 32 x 8 threads and output tiles of
// 30 x FT (FT = 14 or 30), with every thread updating two nodes of its column
// at once: rows ly and ly + 8 of R1 (step 1) or of the tile (step 2).  The two
// nodes are pulled one after the other (pull table and loads per node) and
// then collide together on paired FP32 lanes (collide<M, F2>), which halves the
// arithmetic instructions of the node update.  Each lane performs the scalar
// update's operations in the same order with the same rounding, so every node
// gets the bits of step2_kernel and of step_kernel.  Where one of the two rows
// has no node to update (outside the lattice, or past the tile), its lane
// repeats the other row's node and its result is not stored.  256 threads,
// two CTAs per SM (up to 128 registers a thread).
template <int M, int FT>
__global__ void __launch_bounds__(256, 2)
    step2_kernel_x2(const LbParams p, int, const Planes<float> pl, const float *sp_in, float *sp_out,
                    float *__restrict__ moments) {
    constexpr int NP = 9 + 5 * M, W1 = 32, BY = 8, H1 = FT + 2, SP = W1 * H1, TW = W1 - 2;
    static_assert(H1 % (2 * BY) == 0, "the rows of R1 fill whole paired passes");
    constexpr unsigned kAll = 0xffffffffu;
    extern __shared__ float sm[];
    pdl_wait_and_release();
    const int X0 = blockIdx.x * TW, Y0 = blockIdx.y * FT;
    const long long P = p.plane;
    const int pitch = p.pitch, nx = p.nx, ny = p.ny;
    const bool consume = M >= 2 && p.skind == 2;
    const int lx = threadIdx.x;
    const int xu = X0 - 1 + lx;
    const bool colv = xu <= min(X0 + TW, nx) && (p.periodic_x || (xu >= 0 && xu < nx));
    const int gx = xu < 0 ? xu + nx : (xu >= nx ? xu - nx : xu);

    // ---- step 1: R1 from global memory into shared memory, rows ly and ly + BY
    {
        const auto mk = [pitch](int sx, int sy) { return sy * pitch + sx; };
        const auto ld = [&pl, &p, P](int plane, int off) { return __ldg(pl.in[plane] + CDF_CHK(p, off, P, 1)); };
#pragma unroll
        for (int ly = threadIdx.y; ly < H1; ly += 2 * BY) {
            bool ok[2];
            int gy[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int yu = Y0 - 1 + ly + k * BY;
                ok[k] = colv && yu <= min(Y0 + FT, ny) && (p.periodic_y || (yu >= 0 && yu < ny));
                gy[k] = yu < 0 ? yu + ny : (yu >= ny ? yu - ny : yu);
            }
            const bool any = ok[0] || ok[1];
            const int ya = ok[0] ? gy[0] : gy[1], yb = ok[1] ? gy[1] : gy[0];
            // warp votes before any lane leaves the pass
            const bool gena = __any_sync(kAll, any && !inner_node(p, gx, ya));
            const bool genb = __any_sync(kAll, any && !inner_node(p, gx, yb));
            if (!any) continue;
            float h0[9], f0[M][5], h1[9], f1[M][5];
            if (!gena) pull_node<M, true>(p, gx, ya, mk, ld, f0, h0);
            else pull_node<M, false>(p, gx, ya, mk, ld, f0, h0);
            if (!genb) pull_node<M, true>(p, gx, yb, mk, ld, f1, h1);
            else pull_node<M, false>(p, gx, yb, mk, ld, f1, h1);
            const int oa = CDF_CHK(p, ya * pitch + gx, P, 2), ob = CDF_CHK(p, yb * pitch + gx, P, 2);
            F2 h[9], f[M][5];
            pack_node<M>(f0, h0, f1, h1, f, h);
            NodeOut<M, F2> o;
            collide<M>(p, f, h, pack2(pref_at(p, gx, ya), pref_at(p, gx, yb)),
                       consume ? pack2(sp_in[oa], sp_in[ob]) : splat<F2>(0.f), false, o);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!ok[k]) continue;
                const int l0 = CDF_CHK(p, (ly + k * BY) * W1 + lx, SP, 3);
#pragma unroll
                for (int i = 0; i < 9; ++i) sm[i * SP + l0] = lane(h[i], k);
#pragma unroll
                for (int a = 0; a < M; ++a)
#pragma unroll
                    for (int i = 0; i < 5; ++i) sm[(9 + 5 * a + i) * SP + l0] = lane(f[a][i], k);
                if (consume) sm[NP * SP + l0] = lane(o.s1, k);
            }
        }
    }
    __syncthreads();

    // ---- step 2: the tile from shared memory into global memory, rows ly and ly + BY
    const auto lds = [&p](int plane, int off) { return sm[plane * SP + CDF_CHK(p, off, SP, 4)]; };
    const auto mk_in = [X0, Y0](int sx, int sy) { return (sy - Y0 + 1) * W1 + (sx - X0 + 1); };
    const auto mk_gen = [X0, Y0, nx, ny](int sx, int sy) {
        int a = sx - X0 + 1, b = sy - Y0 + 1;
        a = a < 0 ? a + nx : (a >= W1 ? a - nx : a);
        b = b < 0 ? b + ny : (b >= H1 ? b - ny : b);
        return b * W1 + a;
    };
#pragma unroll
    for (int ly = 1 + threadIdx.y; ly <= FT; ly += 2 * BY) {
        const int x = xu, ya = Y0 - 1 + ly;
        const bool oka = lx >= 1 && lx <= TW && x < nx && ya < ny;
        const bool okb = oka && ly + BY <= FT && ya + BY < ny;
        const int yb = okb ? ya + BY : ya;
        const bool gena = __any_sync(kAll, oka && !inner_node(p, x, ya));
        const bool genb = __any_sync(kAll, oka && !inner_node(p, x, yb));
        if (!oka) continue;
        float h0[9], f0[M][5], h1[9], f1[M][5];
        if (!gena) pull_node<M, true>(p, x, ya, mk_in, lds, f0, h0);
        else pull_node<M, false>(p, x, ya, mk_gen, lds, f0, h0);
        if (!genb) pull_node<M, true>(p, x, yb, mk_in, lds, f1, h1);
        else pull_node<M, false>(p, x, yb, mk_gen, lds, f1, h1);
        const int la = ly * W1 + lx, lb = (yb - Y0 + 1) * W1 + lx;
        F2 h[9], f[M][5];
        pack_node<M>(f0, h0, f1, h1, f, h);
        NodeOut<M, F2> o;
        collide<M>(p, f, h, pack2(pref_at(p, x, ya), pref_at(p, x, yb)),
                   consume ? pack2(sm[NP * SP + CDF_CHK(p, la, SP, 4)], sm[NP * SP + CDF_CHK(p, lb, SP, 4)])
                           : splat<F2>(0.f),
                   false, o);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 1 && !okb) continue;
            const int o0 = CDF_CHK(p, (k ? yb : ya) * pitch + x, P, 2);
#pragma unroll
            for (int i = 0; i < 9; ++i) pl.out[i][o0] = lane(h[i], k);
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int i = 0; i < 5; ++i) pl.out[9 + 5 * a + i][o0] = lane(f[a][i], k);
            if (consume) sp_out[o0] = lane(o.s1, k);
            if (moments) write_moments<M>(moments, P, o0, lane_out<M>(o, k));
        }
    }
}

// ---- Case 1 of Sec. 2.1: convection cross-diffusion in a prescribed velocity -----
// Scalars only: pull the 5m scalar populations, read the node's prescribed
// velocity (p.vel) and phi(t - 1) (p.php_in), collide with the Case-1
// auxiliary source, store the scalars and phi(t) (p.php_out, the other phi
// set).  Algorithmic bytes: 2 x 5m x 4 + 8 + 2 x 4m.
template <int M>
__global__ void __launch_bounds__(256) step_kernel_case1(const LbParams p, const float *__restrict__ in,
                                                         float *__restrict__ out, const float *sp_in, float *sp_out,
                                                         float *__restrict__ moments) {
    pdl_wait_and_release();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const long long P = p.plane;
    const int pitch = p.pitch;
    const auto mk = [pitch](int sx, int sy) { return sy * pitch + sx; };
    const auto ld = [in, P, &p](int plane, int off) { return __ldg(in + plane * P + CDF_CHK(p, off, P, 1)); };
    if (x >= p.nx || y >= p.ny) return;
    const int o0 = CDF_CHK(p, y * pitch + x, P, 2);
    float f[M][5];
    pull_scalars<M, false>(p, x, y, mk, ld, f);
    const float *vel = p.vel;
    const float ux = __ldg(vel + o0), uy = __ldg(vel + P + o0);
    float php[M];
#pragma unroll
    for (int a = 0; a < M; ++a) php[a] = p.php_in[a * P + o0];
    const bool consume = (M >= 2 && p.skind == 2);
    const float sp1 = consume ? sp_in[o0] : 0.f;
    NodeOut<M> o;
    collide_case1<M>(p, f, ux, uy, php, sp1, false, o);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) out[(9 + 5 * a + i) * P + o0] = f[a][i];
#pragma unroll
    for (int a = 0; a < M; ++a) p.php_out[a * P + o0] = php[a];
    if (consume) sp_out[o0] = o.s1;
    if (moments) write_moments<M>(moments, P, o0, o);
}

// Two steps of Case 1 per launch: the tiling of step2_kernel for the scalar
// populations.  Shared memory holds, per R1 node, the 5m post-collision scalar
// populations, phi(t) (the next step's phi(t - 1)) and S_1(t).  The prescribed
// velocity is read from global memory at every node; phi is read from
// p.php_in and written to p.php_out (different sets: the halo of one CTA is the
// tile of another).  Bitwise equal to two launches of step_kernel_case1.
template <int M>
__global__ void __launch_bounds__(step2_max_threads(M)) step2_kernel_case1(const LbParams p, int TH,
                                                                           const Planes<float> pl,
                                                                           const float *sp_in, float *sp_out,
                                                                           float *__restrict__ moments) {
    constexpr int NS = 5 * M;  // scalar planes; then M planes of phi(t), then S_1(t)
    extern __shared__ float sm[];
    pdl_wait_and_release();
    const int W1 = blockDim.x, H1 = TH + 2, SP = W1 * H1, TW = W1 - 2;
    const int X0 = blockIdx.x * TW, Y0 = blockIdx.y * TH;
    const long long P = p.plane;
    const int pitch = p.pitch, nx = p.nx, ny = p.ny;
    const bool consume = M >= 2 && p.skind == 2;
    const int lx = threadIdx.x;
    const int xu = X0 - 1 + lx;
    const bool colv = xu <= min(X0 + TW, nx) && (p.periodic_x || (xu >= 0 && xu < nx));
    const int gx = xu < 0 ? xu + nx : (xu >= nx ? xu - nx : xu);

    // ---- step 1: R1 from global memory into shared memory
    {
        const auto mk = [pitch](int sx, int sy) { return sy * pitch + sx; };
        const auto ld = [&pl, &p, P](int plane, int off) { return __ldg(pl.in[plane] + CDF_CHK(p, off, P, 1)); };
        for (int ly = threadIdx.y; ly < H1; ly += blockDim.y) {
            const int yu = Y0 - 1 + ly;
            const bool ok = colv && yu <= min(Y0 + TH, ny) && (p.periodic_y || (yu >= 0 && yu < ny));
            const int gy = yu < 0 ? yu + ny : (yu >= ny ? yu - ny : yu);
            if (!ok) continue;
            float f[M][5];
            pull_scalars<M, false>(p, gx, gy, mk, ld, f);
            const int o0 = CDF_CHK(p, gy * pitch + gx, P, 2), l0 = CDF_CHK(p, ly * W1 + lx, SP, 3);
            const float ux = __ldg(p.vel + o0), uy = __ldg(p.vel + P + o0);
            float php[M];
#pragma unroll
            for (int a = 0; a < M; ++a) php[a] = p.php_in[a * P + o0];
            NodeOut<M> o;
            collide_case1<M>(p, f, ux, uy, php, consume ? sp_in[o0] : 0.f, false, o);
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int i = 0; i < 5; ++i) sm[(5 * a + i) * SP + l0] = f[a][i];
#pragma unroll
            for (int a = 0; a < M; ++a) sm[(NS + a) * SP + l0] = php[a];
            if (consume) sm[(NS + M) * SP + l0] = o.s1;
        }
    }
    __syncthreads();

    // ---- step 2: the tile from shared memory into global memory
    const auto lds = [SP, &p](int plane, int off) { return sm[(plane - 9) * SP + CDF_CHK(p, off, SP, 4)]; };
    const auto mk_gen = [W1, H1, X0, Y0, nx, ny](int sx, int sy) {
        int a = sx - X0 + 1, b = sy - Y0 + 1;
        a = a < 0 ? a + nx : (a >= W1 ? a - nx : a);
        b = b < 0 ? b + ny : (b >= H1 ? b - ny : b);
        return b * W1 + a;
    };
    for (int ly = 1 + threadIdx.y; ly <= TH; ly += blockDim.y) {
        const int x = xu, y = Y0 - 1 + ly;
        if (!(lx >= 1 && lx <= TW && x < nx && y < ny)) continue;
        float f[M][5];
        pull_scalars<M, false>(p, x, y, mk_gen, lds, f);
        const int o0 = CDF_CHK(p, y * pitch + x, P, 2), l0 = CDF_CHK(p, ly * W1 + lx, SP, 4);
        const float ux = __ldg(p.vel + o0), uy = __ldg(p.vel + P + o0);
        float php[M];
#pragma unroll
        for (int a = 0; a < M; ++a) php[a] = sm[(NS + a) * SP + l0];
        NodeOut<M> o;
        collide_case1<M>(p, f, ux, uy, php, consume ? sm[(NS + M) * SP + l0] : 0.f, false, o);
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int i = 0; i < 5; ++i) pl.out[9 + 5 * a + i][o0] = f[a][i];
#pragma unroll
        for (int a = 0; a < M; ++a) p.php_out[a * P + o0] = php[a];
        if (consume) sp_out[o0] = o.s1;
        if (moments) write_moments<M>(moments, P, o0, o);
    }
}

// Case 1 initialisation: f = f^eq(phi0, u) collided once with phi(t - 1) = phi0
// (so G = 0) and S(t - 1) = S(phi0); u becomes the prescribed velocity.
template <int M>
__global__ void init_kernel_case1(const LbParams p, const float *__restrict__ fields, int fpitch,
                                  float *__restrict__ out, float *__restrict__ sprev, float *__restrict__ moments) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long P = p.plane, FP = (long long)fpitch * p.ny;
    const long long o0 = (long long)y * p.pitch + x, i0 = (long long)y * fpitch + x;
    float phi[M], phid[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        phi[a] = fields[a * FP + i0];
        phid[a] = phi[a] - p.phi_ref[a];
    }
    const float ux = fields[M * FP + i0], uy = fields[(M + 1) * FP + i0];
    float f[M][5];
    scalar_equilibrium<M>(phid, phi, ux, uy, f);
    float php[M];
    NodeOut<M> o;
    {
        // phi(t - 1) = phi0 as the scalar moments see it (sum of the populations)
        ScalarState<M> s;
        scalar_closures<M>(p, f, 0.f, true, s);
#pragma unroll
        for (int a = 0; a < M; ++a) php[a] = s.phi[a];
    }
    collide_case1<M>(p, f, ux, uy, php, 0.f, true, o);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) out[(9 + 5 * a + i) * P + o0] = f[a][i];
    p.vel[o0] = ux;
    p.vel[P + o0] = uy;
#pragma unroll
    for (int a = 0; a < M; ++a) p.php_out[a * P + o0] = php[a];
    if (M >= 2 && p.skind == 2) sprev[o0] = o.s1;
    write_moments<M>(moments, P, o0, o);
}

// ---- initialisation from moments (collide-only pass at t = 0) ------------------
template <int M, typename T>
__global__ void init_kernel(const LbParams p, const float *__restrict__ fields, int fpitch,
                            T *__restrict__ out, float *__restrict__ sprev,
                            float *__restrict__ moments) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long P = p.plane, FP = (long long)fpitch * p.ny;
    const long long o0 = (long long)y * p.pitch + x, i0 = (long long)y * fpitch + x;
    float phi[M], phid[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        phi[a] = fields[a * FP + i0];
        phid[a] = phi[a] - p.phi_ref[a];
    }
    const float ux = fields[M * FP + i0], uy = fields[(M + 1) * FP + i0];
    const float prx = pref_at(p, x, y);
    const float prd = fields[(M + 2) * FP + i0] - prx;
    float fm = p.Fbase;
#pragma unroll
    for (int a = 0; a < M; ++a) fm = fmaf(p.beta[a], phi[a], fm);
    const float Fx = p.g[0] * fm, Fy = p.g[1] * fm;
    // f = f^eq(phi, u); h = h^eq(u, p) - F_i / 2 (moments then return the inputs)
    float f[M][5], h[9];
    const float usq = usq_of(ux, uy);
    const float uF = fmaf(ux, Fx, __fmul_rn(uy, Fy));
    scalar_equilibrium<M>(phid, phi, ux, uy, f);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float Fi = (i == 0 ? 0.f : kA9(i) * cdot(kC9x(i), kC9y(i), Fx, Fy));
        if (p.varphi != 0.f) Fi = fmaf(p.varphi, force2_dir(i, ux, uy, Fx, Fy, uF), Fi);
        h[i] = fluid_equilibrium(i, prd, ux, uy, usq) - 0.5f * Fi;
    }
    NodeOut<M> o;
    collide<M>(p, f, h, prx, 0.f, true, o);
    store_node<M, T>(out, P, o0, f, h);
    if (M >= 2 && p.skind == 2) sprev[o0] = o.s1;
    write_moments<M>(moments, P, o0, o);
}

// Post-collision populations (full values) as dense FP32 planes [9 + 5m][ny][nx].
template <int M, typename T>
__global__ void export_kernel(const LbParams p, const T *__restrict__ in, float *__restrict__ dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long P = p.plane, N = (long long)p.nx * p.ny;
    const long long o0 = (long long)y * p.pitch + x, d0 = (long long)y * p.nx + x;
    const float prx = pref_at(p, x, y);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float ref = (i == 0) ? p.rho0 - kC * prx : kA9(i) * prx;
        dense[i * N + d0] = Store<T>::load(in + i * P + o0) + ref;
    }
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i)
            dense[(9 + 5 * a + i) * N + d0] = Store<T>::load(in + (9 + 5 * a + i) * P + o0) + kWs(i) * p.phi_ref[a];
}

__global__ void pack_kernel(const LbParams p, int nf, const float *__restrict__ mom,
                            float *__restrict__ dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long P = p.plane, N = (long long)p.nx * p.ny;
    for (int k = 0; k < nf; ++k) dense[k * N + (long long)y * p.nx + x] = mom[k * P + (long long)y * p.pitch + x];
}

// ---- 16-bit storage: deviations from each node's own equilibrium ----------------
// For FP16/BF16 the stored value of a post-collision population at node x is
// d_i(x) = f*_i(x) - f^eq_i(phi(x), u(x)) (h*_i - h^eq_i(p(x), u(x)) for the fluid):
// the non-equilibrium part plus the source terms, a small number that 16 bits
// resolve well.  The node's moments (phi, u, p) of the same step are stored in
// FP32 next to it, and the receiving node rebuilds the population as
// d_j(src) + f^eq_j(moments(src)).  Both ends evaluate the equilibrium with the
// same functions on the same stored moments.  The collision itself is the FP32
// one above with phi_ref = 0 and p_ref = 0 (the host sets them so).
__device__ __forceinline__ float heq_dir(int j, float pr, float ux, float uy) {
    return fluid_equilibrium(j, pr, ux, uy, usq_of(ux, uy));
}

// Reference of a stored post-collision fluid population: h^eq_j(p, u).  The
// deviation h*_j - h^eq_j then holds the viscous non-equilibrium part and the
// forcing term of Eq. force, F_j / 2 = 3 W_j c_j.F / 2, which is as small (the
// body forces of the workloads are below 1e-4 in lattice units), so leaving it
// out of the reference costs no precision and saves its evaluation at both ends.
__device__ __forceinline__ float href_dir(int j, float pr, float ux, float uy) { return heq_dir(j, pr, ux, uy); }

// Pre-collision populations of node (x, y) for 16-bit storage: the stored
// deviations of the pull sources plus the equilibria of those sources' stored
// moments (full values: the host sets phi_ref = 0 and p_ref = 0 for this
// storage).  kInterior as in step_node: with no link crossing a wall the source
// directions are compile-time constants, so the rebuilt equilibria need no
// run-time direction selects.
template <int M, typename T, bool kInterior>
__device__ __forceinline__ void pull_node_mr(const LbParams &p, int x, int y, const Planes<T> &pl,
                                             const MomentPlanes &mp, float (&f)[M][5], float (&h)[9]) {
    const int pitch = p.pitch;
    // Pull sources exactly as in step_kernel (the pressure-reference shifts are
    // zero here).
    const auto t = pull_table<kInterior>(p, x, y, [pitch](int sx, int sy) { return sy * pitch + sx; });

    // ---- loads: stored deviations and the source nodes' moments (the axis
    // sources of the fluid and of the scalars are the same nodes)
    float hu[9], hv[9], hp[9], hphi[9][M];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int src = CDF_CHK(p, t.hpos[i], p.plane, 5);
        h[i] = Store<T>::load(pl.in[t.hplane[i]] + src);
        hu[i] = __ldg(mp.in[M] + src);
        hv[i] = __ldg(mp.in[M + 1] + src);
        hp[i] = __ldg(mp.in[M + 2] + src);
#pragma unroll
        for (int a = 0; a < M; ++a) hphi[i][a] = __ldg(mp.in[a] + src);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int a = 0; a < M; ++a)
            f[a][i] = Store<T>::load(pl.in[9 + 5 * a + t.splane[i]] + CDF_CHK(p, t.spos[i], p.plane, 1));

    // ---- rebuild the pre-collision populations
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] += href_dir(t.hplane[i], hp[i], hu[i], hv[i]);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        // rest direction: from this node's own moments, rest by difference
        const float ph = hphi[0][a], t3 = 3.f * ph;
        const float e1 = feq_dir(1, ph, t3, hu[0], hv[0]), e2 = feq_dir(2, ph, t3, hu[0], hv[0]);
        const float e3 = feq_dir(3, ph, t3, hu[0], hv[0]), e4 = feq_dir(4, ph, t3, hu[0], hv[0]);
        f[a][0] += ph - ((e1 + e3) + (e2 + e4));
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            f[a][i] += feq_dir(t.splane[i], hphi[i][a], 3.f * hphi[i][a], hu[i], hv[i]);
            if (t.side[i] >= 0 && ((p.dirichlet[t.side[i]] >> a) & 1u)) f[a][i] = p.abb[t.side[i]][a] - f[a][i];
        }
    }
}

// Encoding of one node for 16-bit storage, conservative.  The deviations of the
// post-collision populations from this node's equilibrium are rounded to 16 bits;
// a receiver rebuilds each population as the rounded deviation plus the
// equilibrium of the moments stored beside it.  Rounding alone would change the
// scalar mass sum_i f*_i, the fluid momentum sum_i c_i h*_i and sum_{i!=0} h*_i
// (the pressure sum of Eq. sum-p) that leave the node by the residuals e_i =
// rounded - exact, a rounding-level source of mass and a body force that never
// averages out at a steady state.  The residuals are therefore folded into the
// FP32 moments that are stored and rebuilt from: with phi_s = phi - sum_i e_i,
// u_s = u - sum_i c_i e_i and p_s chosen so that sum_{i!=0} h^eq_i(p_s, u_s)
// absorbs the pressure residual, the rebuilt populations carry exactly (to FP32
// rounding) the mass, momentum and pressure sum of the collision's output
// (sum_i W_i (1 + 3 c_i.u) = 1, sum_i c_i h^eq_i(p, u) = u and
// sum_{i!=0} h^eq_i(p, u) = kC p' + kQ u.u in these variables).  The scalar
// deviations are taken from the equilibrium at u_s, the velocity the receivers
// rebuild with, so the shift of u leaves the scalar fluxes alone.  The stored
// moments differ from the collision's by the rounding residuals.  The deviations
// are rounded stochastically, two at a time (Store<T>::encode2): the distribution
// functions' own rounding errors then average to zero, where round-to-nearest
// would leave a steady state under a fixed rounding-level forcing of the
// non-conserved moments.
template <int M, typename T>
__device__ __forceinline__ void encode_node_mr(const float (&f)[M][5], const float (&h)[9], const NodeOut<M> &o,
                                               T (&fq)[M][5], T (&hq)[9], float (&mom)[M + 3]) {
    // fluid deviations, rounded stochastically in pairs (slots 0..4)
    float dh[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) dh[i] = h[i] - href_dir(i, o.pr, o.ux, o.uy);
#pragma unroll
    for (int i = 0; i < 8; i += 2) Store<T>::encode2(dh[i], dh[i + 1], i / 2, hq[i], hq[i + 1]);
    {
        T spare;
        Store<T>::encode2(dh[8], 0.f, 4, hq[8], spare);
    }
    float rx = 0.f, ry = 0.f, rp = 0.f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const float e = Store<T>::decode(hq[i]) - dh[i];  // exact (Sterbenz)
        if (kC9x(i) != 0) rx = kC9x(i) > 0 ? rx + e : rx - e;
        if (kC9y(i) != 0) ry = kC9y(i) > 0 ? ry + e : ry - e;
        rp += e;
    }
    const float us = o.ux - rx, vs = o.uy - ry;
    mom[M] = us;
    mom[M + 1] = vs;
    mom[M + 2] = o.pr + __fmul_rn(fmaf(kQ, usq_of(o.ux, o.uy) - usq_of(us, vs), -rp), kInvC);
    // scalar deviations from the equilibrium at the stored velocity: the receivers
    // rebuild with u_s, so taking it here keeps the shift of u out of the scalar fluxes
    float feq[M][5];
    scalar_equilibrium<M>(o.phi, o.phi, us, vs, feq);
    float df[5 * M + 1];
#pragma unroll
    for (int n = 0; n < 5 * M; ++n) df[n] = f[n / 5][n % 5] - feq[n / 5][n % 5];
    df[5 * M] = 0.f;
    T q[5 * M + 1];
#pragma unroll
    for (int n = 0; n < 5 * M; n += 2) Store<T>::encode2(df[n], df[n + 1], 5 + n / 2, q[n], q[n + 1]);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        float r = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            fq[a][i] = q[5 * a + i];
            r += Store<T>::decode(fq[a][i]) - df[5 * a + i];
        }
        mom[a] = o.phi[a] - r;
    }
}

// Store of one node for 16-bit storage: the encoded deviations and the stored
// moments of encode_node_mr.
template <int M, typename T>
__device__ __forceinline__ void store_node_mr(int o0, const Planes<T> &pl, const MomentPlanes &mp,
                                              const float (&f)[M][5], const float (&h)[9], const NodeOut<M> &o) {
    T fq[M][5], hq[9];
    float mom[M + 3];
    encode_node_mr<M, T>(f, h, o, fq, hq, mom);
#pragma unroll
    for (int i = 0; i < 9; ++i) pl.out[i][o0] = hq[i];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) pl.out[9 + 5 * a + i][o0] = fq[a][i];
#pragma unroll
    for (int k = 0; k < M + 3; ++k) mp.out[k][o0] = mom[k];
}

// One node of the 16-bit step.
template <int M, typename T, bool kInterior>
__device__ __forceinline__ void step_node_mr(const LbParams &p, int x, int y, const Planes<T> &pl,
                                             const MomentPlanes &mp, const float *sp_in, float *sp_out) {
    const int o0 = CDF_CHK(p, y * p.pitch + x, p.plane, 2);
    float f[M][5], h[9];
    pull_node_mr<M, T, kInterior>(p, x, y, pl, mp, f, h);
    const bool consume = (M >= 2 && p.skind == 2);
    const float sp1 = consume ? sp_in[o0] : 0.f;
    NodeOut<M> o;
    collide<M>(p, f, h, 0.f, sp1, false, o);
    store_node_mr<M, T>(o0, pl, mp, f, h, o);
    if (consume) sp_out[o0] = o.s1;
}

// Two time steps per launch with 16-bit storage: the tiling of step2_kernel.
// Step 1 rebuilds the populations of the R1 nodes from the stored deviations
// and moments, collides, and keeps the post-collision populations in FP32 in
// shared memory (no 16-bit rounding in between); step 2 pulls them from there,
// collides and stores deviations and moments.  Per two steps the populations
// are rounded to 16 bits once, so the results differ from two one-step
// launches by that saved rounding (both are held to the FP64 oracle).
// FW, FY, FT != 0: a copy for one CTA shape and tile height, as for step2_kernel.
template <int M, typename T, int FW = 0, int FY = 0, int FT = 0>
__global__ void __launch_bounds__(step2_mr_max_threads(M), (M <= 2 ? 3 : 1)) step2_kernel_mr(
    const LbParams p, int TH, const Planes<T> pl, const MomentPlanes mp, const float *sp_in, float *sp_out) {
    constexpr int NP = 9 + 5 * M;
    extern __shared__ float sm[];
    pdl_wait_and_release();
    const int W1 = FW ? FW : (int)blockDim.x, BY = FY ? FY : (int)blockDim.y, THv = FT ? FT : TH;
    const int H1 = THv + 2, SP = W1 * H1, TW = W1 - 2;
    const int X0 = blockIdx.x * TW, Y0 = blockIdx.y * THv;
    const int pitch = p.pitch, nx = p.nx, ny = p.ny;
    const bool consume = M >= 2 && p.skind == 2;
    const int lx = threadIdx.x;
    const int xu = X0 - 1 + lx;
    const bool colv = xu <= min(X0 + TW, nx) && (p.periodic_x || (xu >= 0 && xu < nx));
    const int gx = xu < 0 ? xu + nx : (xu >= nx ? xu - nx : xu);

    // ---- step 1: R1 from the stored deviations into shared memory (FP32)
#pragma unroll
    for (int ly = threadIdx.y; ly < H1; ly += BY) {
        const int yu = Y0 - 1 + ly;
        const bool ok = colv && yu <= min(Y0 + THv, ny) && (p.periodic_y || (yu >= 0 && yu < ny));
        const int gy = yu < 0 ? yu + ny : (yu >= ny ? yu - ny : yu);
        const bool general = ok && !inner_node(p, gx, gy);
        float h[9], f[M][5];
        if (!__any_sync(0xffffffffu, general)) {
            if (!ok) continue;
            pull_node_mr<M, T, true>(p, gx, gy, pl, mp, f, h);
        } else {
            if (!ok) continue;
            pull_node_mr<M, T, false>(p, gx, gy, pl, mp, f, h);
        }
        const int o0 = CDF_CHK(p, gy * pitch + gx, p.plane, 2), l0 = CDF_CHK(p, ly * W1 + lx, SP, 3);
        NodeOut<M> o;
        collide<M>(p, f, h, 0.f, consume ? sp_in[o0] : 0.f, false, o);
#pragma unroll
        for (int i = 0; i < 9; ++i) sm[i * SP + l0] = h[i];
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int i = 0; i < 5; ++i) sm[(9 + 5 * a + i) * SP + l0] = f[a][i];
        if (consume) sm[NP * SP + l0] = o.s1;
    }
    __syncthreads();

    // ---- step 2: the tile from shared memory into 16-bit deviations and moments
    const auto lds = [SP, &p](int plane, int off) { return sm[plane * SP + CDF_CHK(p, off, SP, 4)]; };
    const auto mk_in = [W1, X0, Y0](int sx, int sy) { return (sy - Y0 + 1) * W1 + (sx - X0 + 1); };
    const auto mk_gen = [W1, H1, X0, Y0, nx, ny](int sx, int sy) {
        int a = sx - X0 + 1, b = sy - Y0 + 1;
        a = a < 0 ? a + nx : (a >= W1 ? a - nx : a);
        b = b < 0 ? b + ny : (b >= H1 ? b - ny : b);
        return b * W1 + a;
    };
#pragma unroll
    for (int ly = 1 + threadIdx.y; ly <= THv; ly += BY) {
        const int x = xu, y = Y0 - 1 + ly;
        const bool ok = lx >= 1 && lx <= TW && x < nx && y < ny;
        const bool general = ok && !inner_node(p, x, y);
        float h[9], f[M][5];
        if (!__any_sync(0xffffffffu, general)) {
            if (!ok) continue;
            pull_node<M, true>(p, x, y, mk_in, lds, f, h);
        } else {
            if (!ok) continue;
            pull_node<M, false>(p, x, y, mk_gen, lds, f, h);
        }
        const int o0 = CDF_CHK(p, y * pitch + x, p.plane, 2);
        NodeOut<M> o;
        collide<M>(p, f, h, 0.f, consume ? sm[NP * SP + CDF_CHK(p, ly * W1 + lx, SP, 4)] : 0.f, false, o);
        store_node_mr<M, T>(o0, pl, mp, f, h, o);
        if (consume) sp_out[o0] = o.s1;
    }
}

template <int M, typename T>
__global__ void __launch_bounds__(256, (M <= 2 ? 3 : 1)) step_kernel_mr(const LbParams p, const Planes<T> pl,
                                                                       const MomentPlanes mp, const float *sp_in,
                                                                       float *sp_out) {
    pdl_wait_and_release();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    // warp-uniform interior path, as in step_kernel
    if (__all_sync(0xffffffffu, inner_node(p, x, y)))
        step_node_mr<M, T, true>(p, x, y, pl, mp, sp_in, sp_out);
    else if (x < p.nx && y < p.ny)
        step_node_mr<M, T, false>(p, x, y, pl, mp, sp_in, sp_out);
}

template <int M, typename T>
__global__ void init_kernel_mr(const LbParams p, const float *__restrict__ fields, int fpitch, T *__restrict__ out,
                               float *__restrict__ mout, float *__restrict__ sprev) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long P = p.plane, FP = (long long)fpitch * p.ny;
    const long long o0 = (long long)y * p.pitch + x, i0 = (long long)y * fpitch + x;
    float phi[M];
#pragma unroll
    for (int a = 0; a < M; ++a) phi[a] = fields[a * FP + i0];
    const float ux = fields[M * FP + i0], uy = fields[(M + 1) * FP + i0], pr = fields[(M + 2) * FP + i0];
    float fm = p.Fbase;
#pragma unroll
    for (int a = 0; a < M; ++a) fm = fmaf(p.beta[a], phi[a], fm);
    const float Fx = p.g[0] * fm, Fy = p.g[1] * fm;
    float f[M][5], h[9];
    const float uF = fmaf(ux, Fx, __fmul_rn(uy, Fy));
    scalar_equilibrium<M>(phi, phi, ux, uy, f);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float Fi = (i == 0 ? 0.f : kA9(i) * cdot(kC9x(i), kC9y(i), Fx, Fy));
        if (p.varphi != 0.f) Fi = fmaf(p.varphi, force2_dir(i, ux, uy, Fx, Fy, uF), Fi);
        h[i] = heq_dir(i, pr, ux, uy) - 0.5f * Fi;
    }
    NodeOut<M> o;
    collide<M>(p, f, h, 0.f, 0.f, true, o);
    T fq[M][5], hq[9];
    float mom[M + 3];
    encode_node_mr<M, T>(f, h, o, fq, hq, mom);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i * P + o0] = hq[i];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) out[(9 + 5 * a + i) * P + o0] = fq[a][i];
    if (M >= 2 && p.skind == 2) sprev[o0] = o.s1;
#pragma unroll
    for (int k = 0; k < M + 3; ++k) mout[k * P + o0] = mom[k];
}

template <int M, typename T>
__global__ void export_kernel_mr(const LbParams p, const T *__restrict__ in, const float *__restrict__ min,
                                 float *__restrict__ dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long P = p.plane, N = (long long)p.nx * p.ny;
    const long long o0 = (long long)y * p.pitch + x, d0 = (long long)y * p.nx + x;
    const float ux = min[M * P + o0], uy = min[(M + 1) * P + o0], pr = min[(M + 2) * P + o0];
    float phi[M];
#pragma unroll
    for (int a = 0; a < M; ++a) phi[a] = min[a * P + o0];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        dense[i * N + d0] = Store<T>::load(in + i * P + o0) + href_dir(i, pr, ux, uy) + (i == 0 ? p.rho0 : 0.f);
    float feq[M][5];
    scalar_equilibrium<M>(phi, phi, ux, uy, feq);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i)
            dense[(9 + 5 * a + i) * N + d0] = Store<T>::load(in + (9 + 5 * a + i) * P + o0) + feq[a][i];
}

template <typename T>
cudaError_t step_mr_dispatch(const LbParams &p, const void *in, const float *min, void *out, float *mout,
                             const float *sp_in, float *sp_out, dim3 block, cudaStream_t s) {
    dim3 grid((p.nx + block.x - 1) / block.x, (p.ny + block.y - 1) / block.y);
    const T *i = static_cast<const T *>(in);
    T *o = static_cast<T *>(out);
    const Planes<T> pl = planes_of(p, i, o);
    const MomentPlanes mp = moments_of(p, min, mout);
    cudaError_t e = cudaSuccess;
    switch (p.m) {
        case 1: e = launch_pdl(step_kernel_mr<1, T>, grid, block, s, p, pl, mp, sp_in, sp_out); break;
        case 2: e = launch_pdl(step_kernel_mr<2, T>, grid, block, s, p, pl, mp, sp_in, sp_out); break;
        case 3: e = launch_pdl(step_kernel_mr<3, T>, grid, block, s, p, pl, mp, sp_in, sp_out); break;
        case 4: e = launch_pdl(step_kernel_mr<4, T>, grid, block, s, p, pl, mp, sp_in, sp_out); break;
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t init_mr_dispatch(const LbParams &p, const float *fields, int fpitch, void *out, float *mout,
                             float *sprev, cudaStream_t s) {
    dim3 block(128, 2), grid((p.nx + 127) / 128, (p.ny + 1) / 2);
    T *o = static_cast<T *>(out);
    switch (p.m) {
        case 1: init_kernel_mr<1, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, mout, sprev); break;
        case 2: init_kernel_mr<2, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, mout, sprev); break;
        case 3: init_kernel_mr<3, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, mout, sprev); break;
        case 4: init_kernel_mr<4, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, mout, sprev); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t export_mr_dispatch(const LbParams &p, const void *in, const float *min, float *dense, cudaStream_t s) {
    dim3 block(128, 2), grid((p.nx + 127) / 128, (p.ny + 1) / 2);
    const T *i = static_cast<const T *>(in);
    switch (p.m) {
        case 1: export_kernel_mr<1, T><<<grid, block, 0, s>>>(p, i, min, dense); break;
        case 2: export_kernel_mr<2, T><<<grid, block, 0, s>>>(p, i, min, dense); break;
        case 3: export_kernel_mr<3, T><<<grid, block, 0, s>>>(p, i, min, dense); break;
        case 4: export_kernel_mr<4, T><<<grid, block, 0, s>>>(p, i, min, dense); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t step_dispatch(const LbParams &p, const void *in, void *out, const float *sp_in, float *sp_out, float *mom,
                          dim3 block, cudaStream_t s) {
    const T *i = static_cast<const T *>(in);
    T *o = static_cast<T *>(out);
    if (p.case1) {  // FP32 only (the host refuses other storage), 2-D blocks
        if constexpr (std::is_same<T, float>::value) {
            const dim3 b2(block.x, block.y ? block.y : 1);
            dim3 grid((p.nx + b2.x - 1) / b2.x, (p.ny + b2.y - 1) / b2.y);
            cudaError_t e = cudaSuccess;
            switch (p.m) {
                case 1: e = launch_pdl(step_kernel_case1<1>, grid, b2, s, p, i, o, sp_in, sp_out, mom); break;
                case 2: e = launch_pdl(step_kernel_case1<2>, grid, b2, s, p, i, o, sp_in, sp_out, mom); break;
                case 3: e = launch_pdl(step_kernel_case1<3>, grid, b2, s, p, i, o, sp_in, sp_out, mom); break;
                case 4: e = launch_pdl(step_kernel_case1<4>, grid, b2, s, p, i, o, sp_in, sp_out, mom); break;
                default: return cudaErrorInvalidValue;
            }
            return e != cudaSuccess ? e : cudaGetLastError();
        }
        return cudaErrorInvalidValue;
    }
    const Planes<T> pl = planes_of(p, i, o);
    if (block.y == 0 && block.z == 2) {  // flat launch, two nodes per thread (FP32, m <= 2)
        if constexpr (std::is_same<T, float>::value) {
            const long long n = (long long)p.nx * p.ny;
            const int half = (int)(((n + 1) / 2 + 31) / 32 * 32);
            dim3 fb(block.x), grid((unsigned)((half + block.x - 1) / block.x));
            cudaError_t e = cudaSuccess;
            switch (p.m) {
                case 1: e = launch_pdl(step_kernel_flat_x2<1>, grid, fb, s, p, pl, sp_in, sp_out, mom, half); break;
                case 2: e = launch_pdl(step_kernel_flat_x2<2>, grid, fb, s, p, pl, sp_in, sp_out, mom, half); break;
                default: return cudaErrorInvalidValue;
            }
            return e != cudaSuccess ? e : cudaGetLastError();
        }
        return cudaErrorInvalidValue;
    }
    if (block.y == 0) {  // flat launch
        const long long n = (long long)p.nx * p.ny;
        dim3 fb(block.x), grid((unsigned)((n + block.x - 1) / block.x));
        cudaError_t e = cudaSuccess;
        switch (p.m) {
            case 1: e = launch_pdl(step_kernel_flat<1, T>, grid, fb, s, p, pl, sp_in, sp_out, mom); break;
            case 2: e = launch_pdl(step_kernel_flat<2, T>, grid, fb, s, p, pl, sp_in, sp_out, mom); break;
            case 3: e = launch_pdl(step_kernel_flat<3, T>, grid, fb, s, p, pl, sp_in, sp_out, mom); break;
            case 4: e = launch_pdl(step_kernel_flat<4, T>, grid, fb, s, p, pl, sp_in, sp_out, mom); break;
            default: return cudaErrorInvalidValue;
        }
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    dim3 grid((p.nx + block.x - 1) / block.x, (p.ny + block.y - 1) / block.y);
    cudaError_t e = cudaSuccess;
    switch (p.m) {
        case 1: e = launch_pdl(step_kernel<1, T>, grid, block, s, p, pl, sp_in, sp_out, mom); break;
        case 2: e = launch_pdl(step_kernel<2, T>, grid, block, s, p, pl, sp_in, sp_out, mom); break;
        case 3: e = launch_pdl(step_kernel<3, T>, grid, block, s, p, pl, sp_in, sp_out, mom); break;
        case 4: e = launch_pdl(step_kernel<4, T>, grid, block, s, p, pl, sp_in, sp_out, mom); break;
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t init_dispatch(const LbParams &p, const float *fields, int fpitch, void *out, float *sprev,
                          float *mom, cudaStream_t s) {
    dim3 block(128, 2), grid((p.nx + 127) / 128, (p.ny + 1) / 2);
    T *o = static_cast<T *>(out);
    if (p.case1) {
        if constexpr (std::is_same<T, float>::value) {
            switch (p.m) {
                case 1: init_kernel_case1<1><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
                case 2: init_kernel_case1<2><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
                case 3: init_kernel_case1<3><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
                case 4: init_kernel_case1<4><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
                default: return cudaErrorInvalidValue;
            }
            return cudaGetLastError();
        }
        return cudaErrorInvalidValue;
    }
    switch (p.m) {
        case 1: init_kernel<1, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
        case 2: init_kernel<2, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
        case 3: init_kernel<3, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
        case 4: init_kernel<4, T><<<grid, block, 0, s>>>(p, fields, fpitch, o, sprev, mom); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t export_dispatch(const LbParams &p, const void *in, float *dense, cudaStream_t s) {
    dim3 block(128, 2), grid((p.nx + 127) / 128, (p.ny + 1) / 2);
    const T *i = static_cast<const T *>(in);
    switch (p.m) {
        case 1: export_kernel<1, T><<<grid, block, 0, s>>>(p, i, dense); break;
        case 2: export_kernel<2, T><<<grid, block, 0, s>>>(p, i, dense); break;
        case 3: export_kernel<3, T><<<grid, block, 0, s>>>(p, i, dense); break;
        case 4: export_kernel<4, T><<<grid, block, 0, s>>>(p, i, dense); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(const LbParams &p, int storage, const void *in, void *out, const float *sp_in, float *sp_out,
                        float *moments, dim3 block, cudaStream_t s) {
    // 16-bit storage runs the node-equilibrium kernels (launch_step_mr)
    if (storage != kFP32) return cudaErrorInvalidValue;
    return step_dispatch<float>(p, in, out, sp_in, sp_out, moments, block, s);
}

size_t step2_smem_bytes(int m, dim3 block, int th) {
    return (size_t)(9 + 5 * m + 1) * block.x * (th + 2) * sizeof(float);
}

cudaError_t launch_step2(const LbParams &p, const float *in, float *out, const float *sp_in, float *sp_out,
                         float *moments, dim3 block, int th, cudaStream_t s) {
    const size_t smem = step2_smem_bytes(p.m, block, th);
    dim3 grid((p.nx + block.x - 3) / (block.x - 2), (p.ny + th - 1) / th);
    const Planes<float> pl = planes_of(p, in, out);
    // block.z == 2 names the paired-lane kernel (two nodes per thread; CTAs of
    // 32 x 8 threads, tile heights 14 and 30)
    const bool x2 = block.z == 2;
    if (x2 && (p.case1 || block.x != 32 || block.y != 8 || (th != 14 && th != 30))) return cudaErrorInvalidValue;
    const dim3 threads(block.x, block.y, 1);
    // the opt-in to more than 48 KB of dynamic shared memory, once per device and m
    static std::atomic<bool> attr_set[64][kMaxM + 1];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    // the shape that the autotuners pick for large lattices and for the batched
    // sweep has its own copy of the kernel (constant shared-memory strides)
    const bool fixed = !p.case1 && block.x == 32 && block.y == 8 && th == 14;
    switch (p.m) {
#define CDF_STEP2_CASE(MM)                                                                               \
    case MM:                                                                                             \
        if (!attr_set[dev][MM].load()) {                                                                 \
            e = cudaFuncSetAttribute(step2_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                     kStep2MaxSmem);                                                     \
            if (e == cudaSuccess)                                                                        \
                e = cudaFuncSetAttribute(step2_kernel<MM, 32, 8, 14>,                                    \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kStep2MaxSmem);    \
            if (e == cudaSuccess)                                                                        \
                e = cudaFuncSetAttribute(step2_kernel_case1<MM>,                                         \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kStep2MaxSmem);    \
            if (e == cudaSuccess && MM <= 2)                                                             \
                e = cudaFuncSetAttribute(step2_kernel_x2<(MM <= 2 ? MM : 2), 14>,                        \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kStep2MaxSmem);    \
            if (e == cudaSuccess && MM <= 2)                                                             \
                e = cudaFuncSetAttribute(step2_kernel_x2<(MM <= 2 ? MM : 2), 30>,                        \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kStep2MaxSmem);    \
            if (e != cudaSuccess) return e;                                                              \
            attr_set[dev][MM].store(true);                                                               \
        }                                                                                                \
        if (p.case1)                                                                                     \
            e = launch_pdl_smem(step2_kernel_case1<MM>, grid, threads, smem, s, p, th, pl, sp_in, sp_out, moments); \
        else if (x2)                                                                                     \
            e = MM > 2 ? cudaErrorInvalidValue                                                           \
                       : launch_pdl_smem(th == 14 ? step2_kernel_x2<(MM <= 2 ? MM : 2), 14>              \
                                                  : step2_kernel_x2<(MM <= 2 ? MM : 2), 30>,             \
                                         grid, threads, smem, s, p, th, pl, sp_in, sp_out, moments);     \
        else if (fixed)                                                                                  \
            e = launch_pdl_smem(step2_kernel<MM, 32, 8, 14>, grid, threads, smem, s, p, th, pl, sp_in, sp_out,   \
                                moments);                                                                \
        else                                                                                             \
            e = launch_pdl_smem(step2_kernel<MM>, grid, threads, smem, s, p, th, pl, sp_in, sp_out, moments); \
        break;
        CDF_STEP2_CASE(1)
        CDF_STEP2_CASE(2)
        CDF_STEP2_CASE(3)
        CDF_STEP2_CASE(4)
#undef CDF_STEP2_CASE
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t step2_mr_dispatch(const LbParams &p, const void *in, const float *min, void *out, float *mout,
                              const float *sp_in, float *sp_out, dim3 block, int th, cudaStream_t s) {
    const size_t smem = step2_smem_bytes(p.m, block, th);
    dim3 grid((p.nx + block.x - 3) / (block.x - 2), (p.ny + th - 1) / th);
    const T *i = static_cast<const T *>(in);
    T *o = static_cast<T *>(out);
    const Planes<T> pl = planes_of(p, i, o);
    const MomentPlanes mp = moments_of(p, min, mout);
    static std::atomic<bool> attr_set[64][kMaxM + 1];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const bool fixed = block.x == 32 && block.y == 8 && th == 14;  // the shape with its own copy
    switch (p.m) {
#define CDF_STEP2MR_CASE(MM)                                                                             \
    case MM:                                                                                             \
        if (!attr_set[dev][MM].load()) {                                                                 \
            e = cudaFuncSetAttribute(step2_kernel_mr<MM, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     kStep2MaxSmem);                                                     \
            if (e == cudaSuccess)                                                                        \
                e = cudaFuncSetAttribute(step2_kernel_mr<MM, T, 32, 8, 14>,                              \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kStep2MaxSmem);    \
            if (e != cudaSuccess) return e;                                                              \
            attr_set[dev][MM].store(true);                                                               \
        }                                                                                                \
        e = fixed ? launch_pdl_smem(step2_kernel_mr<MM, T, 32, 8, 14>, grid, block, smem, s, p, th, pl, mp, sp_in, \
                                    sp_out)                                                              \
                  : launch_pdl_smem(step2_kernel_mr<MM, T>, grid, block, smem, s, p, th, pl, mp, sp_in, sp_out); \
        break;
        CDF_STEP2MR_CASE(1)
        CDF_STEP2MR_CASE(2)
        CDF_STEP2MR_CASE(3)
        CDF_STEP2MR_CASE(4)
#undef CDF_STEP2MR_CASE
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_step2_mr(const LbParams &p, int storage, const void *in, const float *moments_in, void *out,
                            float *moments_out, const float *sp_in, float *sp_out, dim3 block, int th,
                            cudaStream_t s) {
    switch (storage) {
        case kFP16:
            return step2_mr_dispatch<__half>(p, in, moments_in, out, moments_out, sp_in, sp_out, block, th, s);
        case kBF16:
            return step2_mr_dispatch<__nv_bfloat16>(p, in, moments_in, out, moments_out, sp_in, sp_out, block, th,
                                                    s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init(const LbParams &p, int storage, const float *fields, int fields_pitch,
                        void *out, float *sprev, float *moments, cudaStream_t s) {
    if (storage != kFP32) return cudaErrorInvalidValue;  // 16-bit: launch_init_mr
    return init_dispatch<float>(p, fields, fields_pitch, out, sprev, moments, s);
}

cudaError_t launch_export(const LbParams &p, int storage, const void *in, float *dense, cudaStream_t s) {
    if (storage != kFP32) return cudaErrorInvalidValue;  // 16-bit: launch_export_mr
    return export_dispatch<float>(p, in, dense, s);
}

cudaError_t launch_step_mr(const LbParams &p, int storage, const void *in, const float *moments_in, void *out,
                           float *moments_out, const float *sp_in, float *sp_out, dim3 block, cudaStream_t s) {
    switch (storage) {
        case kFP16: return step_mr_dispatch<__half>(p, in, moments_in, out, moments_out, sp_in, sp_out, block, s);
        case kBF16: return step_mr_dispatch<__nv_bfloat16>(p, in, moments_in, out, moments_out, sp_in, sp_out, block, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init_mr(const LbParams &p, int storage, const float *fields, int fields_pitch, void *out,
                           float *moments_out, float *sprev, cudaStream_t s) {
    switch (storage) {
        case kFP16: return init_mr_dispatch<__half>(p, fields, fields_pitch, out, moments_out, sprev, s);
        case kBF16: return init_mr_dispatch<__nv_bfloat16>(p, fields, fields_pitch, out, moments_out, sprev, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_export_mr(const LbParams &p, int storage, const void *in, const float *moments, float *dense,
                             cudaStream_t s) {
    switch (storage) {
        case kFP16: return export_mr_dispatch<__half>(p, in, moments, dense, s);
        case kBF16: return export_mr_dispatch<__nv_bfloat16>(p, in, moments, dense, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_pack_moments(const LbParams &p, const float *moments, float *dense, cudaStream_t s) {
    dim3 block(128, 2), grid((p.nx + 127) / 128, (p.ny + 1) / 2);
    pack_kernel<<<grid, block, 0, s>>>(p, p.m + 3, moments, dense);
    return cudaGetLastError();
}

}  // namespace cdflb
