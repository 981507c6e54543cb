// Three-dimensional fused step of the CDF lattice Boltzmann model (Zhan, Chai &
// Shi, arXiv:2101.03055): D3Q7 scalars (Eq. D3Q7, cs^2 = 1/4) and D3Q19 fluid
// (Eq. D3Q19, cs^2 = 1/3), the same collision as the 2-D kernels written for
// d = 3, and the C ABI of include/cdf_lb3d.h.
//
// One thread owns one node; a CTA covers a block_x x block_y patch of one
// z plane.  Every pull source is chosen by selects (regular link, or bounce-back
// when the link crosses a wall), so all 19 + 7m loads issue before any
// arithmetic; the node is collided in registers and stored: one read and one
// write of every population per step, 2 (19 + 7m) 4 bytes per node update.
// Populations are FP32 deviations from a reference state, as in 2-D:
// f - W_i phi_ref and h - h^eq(p_ref(x), 0) with p_ref(x) = G.(x - x_c).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/cdf_lb3d.h"
#include "lb_internal.h"

namespace cdflb {
namespace d3 {

constexpr int kMaxM3 = 3;

struct Lb3Params {
    int nx, ny, nz, pitch;
    long long plane;           // elements per plane (pitch * ny * nz)
    int m;
    float omega[kMaxM * kMaxM];  // constant D: omega; chemotaxis: inverse of the constant part
    float omega_f;
    int chemotaxis;
    float chi4;                // chi / cs_s^2
    float c_star, eps2;
    int r_regularised;
    int skind;
    float S[kMaxM];
    float k;
    float g[3];
    float beta[kMaxM];
    float Fbase;
    float rho0;
    int periodic[3];
    unsigned dirichlet[6];     // per side (x-, x+, y-, y+, z-, z+): bit a set -> scalar a Dirichlet
    float abb[6][kMaxM];       // 2 W_i (phi_w - phi_ref) = (phi_w - phi_ref) / 4
    float phi_ref[kMaxM];
    float gref[3];
    float xc, yc, zc;
};

// ---- lattice constants -----------------------------------------------------------
// D3Q7: W_0 = 1/4, W_1..6 = 1/8, 1/cs^2 = 4, all exact in FP32.
// D3Q19: kB1 = 3 W_1..6 ~ 1/6, kB2 = 3 W_7..18 ~ 1/12, chosen so that for the
// rounded values 2 kB1 + 8 kB2 = 1 (3 sum W c_x^2 = 1) and kC3 = 6 kB1 + 12 kB2
// (= (1 - W_0)/cs^2 ~ 2) hold exactly; kQ3 = 3/2 - kC3/2.  Off the exact
// weights by at most 2.4e-7 relative.
constexpr float kW7 = 0.125f;
constexpr float kB1 = 0x1.555550p-3f;
constexpr float kB2 = 0x1.555558p-4f;
constexpr float kC3 = 0x1.fffffep+0f;
constexpr float kQ3 = 0x1.000002p-1f;

__host__ __device__ constexpr int c7(int i, int d) {
    return i == 0 ? 0 : ((i - 1) % 3 == d ? (i <= 3 ? 1 : -1) : 0);
}
__host__ __device__ constexpr int opp7(int i) { return i == 0 ? 0 : (i <= 3 ? i + 3 : i - 3); }
// D3Q19 in the order of Eq. D3Q19
__host__ __device__ constexpr int c19(int i, int d) {
    return d == 0 ? (i == 1 || i == 7 || i == 9 || i == 11 || i == 14) ? 1
                    : (i == 2 || i == 8 || i == 10 || i == 12 || i == 13) ? -1 : 0
         : d == 1 ? (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
                    : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0
                  : (i == 5 || i == 11 || i == 13 || i == 15 || i == 18) ? 1
                    : (i == 6 || i == 12 || i == 14 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp19(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float kB19(int i) { return i == 0 ? 0.f : (i <= 6 ? kB1 : kB2); }
constexpr float kInvC3 = 0x1.000002p-1f;  // fl(1 / kC3): Eq. sum-p by one multiply

// c . (a0, a1, a2) for a lattice direction whose components are 0 or +-1 (at most
// two nonzero), without multiplications by the components.
__device__ __forceinline__ float cdot3(int c0, int c1, int c2, float a0, float a1, float a2) {
    const float t0 = c0 > 0 ? a0 : -a0, t1 = c1 > 0 ? a1 : -a1, t2 = c2 > 0 ? a2 : -a2;
    if (c0 != 0) return c1 != 0 ? t0 + t1 : (c2 != 0 ? t0 + t2 : t0);
    if (c1 != 0) return c2 != 0 ? t1 + t2 : t1;
    return c2 != 0 ? t2 : 0.f;
}
__device__ __forceinline__ float c19dot(int i, const float (&a)[3]) {
    return cdot3(c19(i, 0), c19(i, 1), c19(i, 2), a[0], a[1], a[2]);
}
__device__ __forceinline__ float c7dot(int i, const float (&a)[3]) {
    return cdot3(c7(i, 0), c7(i, 1), c7(i, 2), a[0], a[1], a[2]);
}

// Fluid equilibrium deviation on D3Q19 (Eq. heq): for i != 0,
// kB_i (q + 1.5 (c_i.u)^2) + kB_i c_i.u with q = p' - 0.5 u.u; the first term is even
// in c_i, the second odd, so the odd directions i = 1, 3, .., 17 and their opposites
// i + 1 share them (the collision forms them once per pair); -kC3 p' - kQ3 u.u for i = 0.
__device__ __forceinline__ float heq3_even(int i, float q, const float (&u)[3]) {
    const float cu = c19dot(i, u);
    return __fmul_rn(kB19(i), fmaf(1.5f, __fmul_rn(cu, cu), q));
}
__device__ __forceinline__ float heq3_odd(int i, const float (&u)[3]) { return __fmul_rn(kB19(i), c19dot(i, u)); }
__device__ __forceinline__ float fluid_eq3(int i, float prd, const float (&u)[3], float usq) {
    if (i == 0) return fmaf(-kC3, prd, __fmul_rn(-kQ3, usq));
    const int b = (i & 1) ? i : i - 1;
    const float E = heq3_even(b, fmaf(-0.5f, usq, prd), u), O = heq3_odd(b, u);
    return b == i ? E + O : E - O;
}

__device__ __forceinline__ float pref_at(const Lb3Params &p, int x, int y, int z) {
    return fmaf(p.gref[0], (float)x - p.xc,
                fmaf(p.gref[1], (float)y - p.yc, __fmul_rn(p.gref[2], (float)z - p.zc)));
}

__device__ __forceinline__ float cutoff(const Lb3Params &p, float c) {
    if (p.r_regularised) {
        const float d = c - p.c_star;
        return 0.5f * fmaf(d, rsqrtf(fmaf(d, d, p.eps2)), 1.f);
    }
    return c >= p.c_star ? 1.f : 0.f;
}

template <int M>
struct Out3 {
    float phi[M], u[3], pr, s1;
};

// Collision of one node (Eqs. evolution12, evolution3 for d = 3) in deviation
// variables; f, h are overwritten by the post-collision values.
template <int M>
__device__ __forceinline__ void collide3(const Lb3Params &p, float (&f)[M][7], float (&h)[19], float prx, float sp1,
                                         bool first, Out3<M> &o) {
    float phid[M], phi[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        phid[a] = ((f[a][0] + f[a][1]) + (f[a][2] + f[a][3])) + ((f[a][4] + f[a][5]) + f[a][6]);
        phi[a] = p.phi_ref[a] + phid[a];
    }
    float r = 0.f;
    if (M >= 2 && (p.chemotaxis || p.skind == 2)) r = cutoff(p, phi[M >= 2 ? 1 : 0]);
    float S[M], Sp[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        S[a] = (p.skind == 1) ? p.S[a] : 0.f;
        Sp[a] = S[a];
    }
    if (M >= 2 && p.skind == 2) {
        S[1] = -p.k * phi[0] * r;
        Sp[1] = first ? S[1] : sp1;
    }
    float fm = p.Fbase;
#pragma unroll
    for (int a = 0; a < M; ++a) fm = fmaf(p.beta[a], phi[a], fm);
    float F[3], u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F[d] = p.g[d] * fm;
        float j = 0.f;
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (c19(i, d) > 0) j += h[i];
            if (c19(i, d) < 0) j -= h[i];
        }
        u[d] = fmaf(0.5f, F[d], j);
    }
    const float usq = fmaf(u[0], u[0], fmaf(u[1], u[1], __fmul_rn(u[2], u[2])));
    float snr = 0.f;
#pragma unroll
    for (int i = 1; i < 19; ++i) snr += h[i];
    const float prd = __fmul_rn(fmaf(-kQ3, usq, snr), kInvC3);

    // Eq. omega-D (cs_s^2 = 1/4): omega^-1 = B + delta e_0 e_1^T, delta = -4 chi phi_0 r
    float om[M][M];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) om[a][b] = p.omega[a * M + b];
    if (M >= 2 && p.chemotaxis) {
        const float delta = -p.chi4 * phi[0] * r;
        const float den = 1.f / fmaf(delta, om[M >= 2 ? 1 : 0][0], 1.f);
        float col0[M], row1[M];
#pragma unroll
        for (int a = 0; a < M; ++a) { col0[a] = om[a][0]; row1[a] = om[M >= 2 ? 1 : 0][a]; }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) om[a][b] = fmaf(-__fmul_rn(__fmul_rn(delta, den), col0[a]), row1[b], om[a][b]);
    }
    // Eq. Gi: J_a = sum_b (delta_ab - omega_ab/2)(u S_b + phi_b F); G_i,a = W_i c_i.J_a / cs_s^2
    float J[M][3];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float acc = 0.f;
#pragma unroll
            for (int b = 0; b < M; ++b)
                acc = fmaf(fmaf(-0.5f, om[a][b], a == b ? 1.f : 0.f), fmaf(u[d], S[b], __fmul_rn(phi[b], F[d])), acc);
            J[a][d] = acc;
        }
    // Eq. evolution12 on D3Q7; f^eq_i - W_i phi_ref = W_i (phi' + 4 phi c_i.u),
    // the rest population by difference
    float feq[M][7];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const float t = 4.f * phi[a];
        float mv = 0.f;
#pragma unroll
        for (int i = 1; i < 7; ++i) feq[a][i] = __fmul_rn(kW7, fmaf(t, c7dot(i, u), phid[a]));
        mv = ((feq[a][1] + feq[a][4]) + (feq[a][2] + feq[a][5])) + (feq[a][3] + feq[a][6]);
        feq[a][0] = phid[a] - mv;
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        float neq[M];
#pragma unroll
        for (int b = 0; b < M; ++b) neq[b] = f[b][i] - feq[b][i];
        const float w = (i == 0) ? 0.25f : kW7;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            float coll = 0.f;
#pragma unroll
            for (int b = 0; b < M; ++b) coll = fmaf(om[a][b], neq[b], coll);
            const float G = (i == 0) ? 0.f : __fmul_rn(4.f * kW7, c7dot(i, J[a]));
            f[a][i] = (f[a][i] - coll) + fmaf(w, fmaf(1.5f, S[a], __fmul_rn(-0.5f, Sp[a])), G);
        }
    }
    // Eq. evolution3 with Eq. force (varphi = 0) on D3Q19: h*_i = h_i - wf (h_i - h^eq_i)
    // + fw F_i (the non-equilibrium part first: a node at equilibrium stays there
    // exactly).  h^eq and F_i = kB_i c_i.F split into parts even and odd in c_i, which a
    // direction i (odd) and its opposite i + 1 share.
    const float wf = p.omega_f, fw = 1.f - 0.5f * wf;
    h[0] = fmaf(-wf, h[0] - fluid_eq3(0, prd, u, usq), h[0]);
    const float q = fmaf(-0.5f, usq, prd);
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const float E = heq3_even(i, q, u), O = heq3_odd(i, u), Fo = __fmul_rn(kB19(i), c19dot(i, F));
        h[i] = fmaf(fw, Fo, fmaf(-wf, h[i] - (E + O), h[i]));
        h[i + 1] = fmaf(fw, -Fo, fmaf(-wf, h[i + 1] - (E - O), h[i + 1]));
    }
#pragma unroll
    for (int a = 0; a < M; ++a) o.phi[a] = phi[a];
#pragma unroll
    for (int d = 0; d < 3; ++d) o.u[d] = u[d];
    o.pr = prx + prd;
    o.s1 = (M >= 2) ? S[M >= 2 ? 1 : 0] : 0.f;
}

template <int M>
__device__ __forceinline__ void store3(const Lb3Params &p, float *out, float *sprev, float *moments, long long o0,
                                       const float (&f)[M][7], const float (&h)[19], const Out3<M> &o) {
    const long long P = p.plane;
#pragma unroll
    for (int i = 0; i < 19; ++i) out[i * P + o0] = h[i];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 7; ++i) out[(19 + 7 * a + i) * P + o0] = f[a][i];
    if (M >= 2 && p.skind == 2) sprev[o0] = o.s1;
    if (moments) {
#pragma unroll
        for (int a = 0; a < M; ++a) moments[a * P + o0] = o.phi[a];
#pragma unroll
        for (int d = 0; d < 3; ++d) moments[(M + d) * P + o0] = o.u[d];
        moments[(M + 3) * P + o0] = o.pr;
    }
}

template <int M>
__global__ void __launch_bounds__(256) step3d_kernel(const Lb3Params p, const float *__restrict__ in,
                                                     float *__restrict__ out, float *__restrict__ sprev,
                                                     float *__restrict__ moments) {
    // programmatic dependent launch: wait for the previous step's results, then
    // let the next step's CTAs be scheduled (hides the launch gap)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long P = p.plane;
    // neighbour coordinates (periodic wrap) and wall crossings of the pull links
    const int X[3] = {x, y, z}, N[3] = {p.nx, p.ny, p.nz};
    int lo[3], hi[3];
    bool clo[3], chi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo[d] = X[d] - 1;
        hi[d] = X[d] + 1;
        clo[d] = lo[d] < 0 && !p.periodic[d];
        chi[d] = hi[d] >= N[d] && !p.periodic[d];
        lo[d] = lo[d] < 0 ? N[d] - 1 : lo[d];
        hi[d] = hi[d] >= N[d] ? 0 : hi[d];
    }
    // in-plane offsets fit in int: the host keeps pitch * ny * nz < 2^31
    const auto off = [&](int sx, int sy, int sz) { return (sz * p.ny + sy) * p.pitch + sx; };
    const int o0 = off(x, y, z);
    // shifts of the pressure reference along links, kept out of FMA contraction
    const float gB1[3] = {__fmul_rn(kB1, p.gref[0]), __fmul_rn(kB1, p.gref[1]), __fmul_rn(kB1, p.gref[2])};
    const float gB2[3] = {__fmul_rn(kB2, p.gref[0]), __fmul_rn(kB2, p.gref[1]), __fmul_rn(kB2, p.gref[2])};

    // ---- fluid sources: x - c_i, or bounce-back from x when the link crosses a wall
    int hp[19], ho[19];
    float hs[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        bool cross = false;
        int s[3];
        float shift = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int c = c19(i, d);
            s[d] = c > 0 ? lo[d] : (c < 0 ? hi[d] : X[d]);
            cross = cross || (c > 0 && clo[d]) || (c < 0 && chi[d]);
            if (c != 0) shift -= (float)c * (i <= 6 ? gB1[d] : gB2[d]);
        }
        hp[i] = cross ? opp19(i) : i;
        ho[i] = cross ? o0 : off(s[0], s[1], s[2]);
        hs[i] = cross ? 0.f : shift;
    }
    // ---- scalar sources (axis links): bounce-back / anti-bounce-back at walls
    int sp[7], side[7], so[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        bool cross = false;
        int s[3], sd = -1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int c = c7(i, d);
            s[d] = c > 0 ? lo[d] : (c < 0 ? hi[d] : X[d]);
            if (c > 0 && clo[d]) { cross = true; sd = 2 * d; }
            if (c < 0 && chi[d]) { cross = true; sd = 2 * d + 1; }
        }
        sp[i] = cross ? opp7(i) : i;
        so[i] = cross ? o0 : off(s[0], s[1], s[2]);
        side[i] = cross ? sd : -1;
    }
    // ---- loads
    float h[19], f[M][7];
#pragma unroll
    for (int i = 0; i < 19; ++i) h[i] = __ldg(in + hp[i] * P + ho[i]);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 7; ++i) f[a][i] = __ldg(in + (19 + 7 * a + sp[i]) * P + so[i]);
    const bool consume = (M >= 2 && p.skind == 2);
    const float sp1 = consume ? sprev[o0] : 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) h[i] += hs[i];
#pragma unroll
    for (int i = 1; i < 7; ++i)
        if (side[i] >= 0)
#pragma unroll
            for (int a = 0; a < M; ++a)
                if ((p.dirichlet[side[i]] >> a) & 1u) f[a][i] = p.abb[side[i]][a] - f[a][i];
    Out3<M> o;
    collide3<M>(p, f, h, pref_at(p, x, y, z), sp1, false, o);
    store3<M>(p, out, sprev, moments, o0, f, h, o);
}

// t = 0: f = f^eq(phi0, u0), h = h^eq(u0, p0) - F_i/2, collided once (S(t-1) = S).
template <int M>
__global__ void init3d_kernel(const Lb3Params p, const float *__restrict__ fields, float *__restrict__ out,
                              float *__restrict__ sprev, float *__restrict__ moments) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long N = (long long)p.nx * p.ny * p.nz, i0 = ((long long)z * p.ny + y) * p.nx + x;
    const long long o0 = ((long long)z * p.ny + y) * p.pitch + x;
    float phi[M], phid[M], u[3];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        phi[a] = fields[a * N + i0];
        phid[a] = phi[a] - p.phi_ref[a];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = fields[(M + d) * N + i0];
    const float prx = pref_at(p, x, y, z);
    const float prd = fields[(M + 3) * N + i0] - prx;
    float fm = p.Fbase;
#pragma unroll
    for (int a = 0; a < M; ++a) fm = fmaf(p.beta[a], phi[a], fm);
    const float usq = fmaf(u[0], u[0], fmaf(u[1], u[1], __fmul_rn(u[2], u[2])));
    float f[M][7], h[19];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const float t = 4.f * phi[a];
#pragma unroll
        for (int i = 1; i < 7; ++i) f[a][i] = __fmul_rn(kW7, fmaf(t, c7dot(i, u), phid[a]));
        f[a][0] = phid[a] - (((f[a][1] + f[a][4]) + (f[a][2] + f[a][5])) + (f[a][3] + f[a][6]));
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float g[3] = {p.g[0], p.g[1], p.g[2]};
        const float cF = c19dot(i, g) * fm;
        h[i] = fluid_eq3(i, prd, u, usq) - 0.5f * __fmul_rn(kB19(i), cF);
    }
    Out3<M> o;
    collide3<M>(p, f, h, prx, 0.f, true, o);
    store3<M>(p, out, sprev, moments, o0, f, h, o);
}

// Post-collision populations as full values, dense [19 + 7m][nz][ny][nx].
template <int M>
__global__ void export3d_kernel(const Lb3Params p, const float *__restrict__ in, float *__restrict__ dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long N = (long long)p.nx * p.ny * p.nz, d0 = ((long long)z * p.ny + y) * p.nx + x;
    const long long o0 = ((long long)z * p.ny + y) * p.pitch + x;
    const float prx = pref_at(p, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float ref = (i == 0) ? p.rho0 - kC3 * prx : kB19(i) * prx;
        dense[i * N + d0] = in[i * p.plane + o0] + ref;
    }
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 7; ++i)
            dense[(19 + 7 * a + i) * N + d0] = in[(19 + 7 * a + i) * p.plane + o0] + (i == 0 ? 0.25f : kW7) * p.phi_ref[a];
}

__global__ void pack3d_kernel(const Lb3Params p, int nf, const float *__restrict__ mom, float *__restrict__ dense) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long N = (long long)p.nx * p.ny * p.nz;
    for (int k = 0; k < nf; ++k)
        dense[k * N + ((long long)z * p.ny + y) * p.nx + x] = mom[k * p.plane + ((long long)z * p.ny + y) * p.pitch + x];
}

#define DISPATCH_M(KERNEL, GRID, BLOCK, STREAM, ...)                                        \
    switch (p.m) {                                                                          \
        case 1: KERNEL<1><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                  \
        case 2: KERNEL<2><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                  \
        case 3: KERNEL<3><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;                  \
        default: return cudaErrorInvalidValue;                                              \
    }

dim3 grid_of(const Lb3Params &p, dim3 b) { return dim3((p.nx + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, p.nz); }

template <int M>
cudaError_t launch_step3_m(const Lb3Params &p, const float *in, float *out, float *sprev, float *mom, dim3 b,
                           cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid_of(p, b);
    cfg.blockDim = b;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step3d_kernel<M>, p, in, out, sprev, mom);
}

cudaError_t launch_step3(const Lb3Params &p, const float *in, float *out, float *sprev, float *mom, dim3 b,
                         cudaStream_t s) {
    switch (p.m) {
        case 1: return launch_step3_m<1>(p, in, out, sprev, mom, b, s);
        case 2: return launch_step3_m<2>(p, in, out, sprev, mom, b, s);
        case 3: return launch_step3_m<3>(p, in, out, sprev, mom, b, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_init3(const Lb3Params &p, const float *fields, float *out, float *sprev, float *mom,
                         cudaStream_t s) {
    const dim3 b(128, 2);
    DISPATCH_M(init3d_kernel, grid_of(p, b), b, s, p, fields, out, sprev, mom)
    return cudaGetLastError();
}
cudaError_t launch_export3(const Lb3Params &p, const float *in, float *dense, cudaStream_t s) {
    const dim3 b(128, 2);
    DISPATCH_M(export3d_kernel, grid_of(p, b), b, s, p, in, dense)
    return cudaGetLastError();
}
cudaError_t launch_pack3(const Lb3Params &p, const float *mom, float *dense, cudaStream_t s) {
    const dim3 b(128, 2);
    pack3d_kernel<<<grid_of(p, b), b, 0, s>>>(p, p.m + 4, mom, dense);
    return cudaGetLastError();
}

// ---- host helpers -----------------------------------------------------------------
bool invert(int n, const double *a_in, double *inv) {
    double a[kMaxM * kMaxM];
    std::memcpy(a, a_in, sizeof(double) * n * n);
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

constexpr int kGraphSteps = 32;
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, dim3> g_tune;

}  // namespace d3
}  // namespace cdflb

using namespace cdflb;
using namespace cdflb::d3;

struct cdf_lb3d {
    int device = 0;
    int nx = 0, ny = 0, nz = 0, m = 0, pitch = 0;
    long long plane = 0;
    int planes = 0, sprev_planes = 0;
    Lb3Params P{};
    float *buf[2] = {nullptr, nullptr};
    int cur = 0;
    float *sprev = nullptr, *mom = nullptr, *mom_prev = nullptr, *dense = nullptr, *host_stage = nullptr;
    double *partials = nullptr, *red = nullptr, *red_host = nullptr;
    cudaStream_t s = nullptr, user = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    dim3 block{128, 1, 1};
    long long t = 0;
    bool initialised = false;
};

namespace {

cdf_status fail3(cdf_status st, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return cdflb::report_error(st, msg);
}

#define CK3(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail3(CDF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void release3(cdf_lb3d *h) {
    if (!h) return;
    Guard g(h->device);
    for (auto &row : h->graph)
        for (auto &ge : row)
            if (ge) cudaGraphExecDestroy(ge);
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->sprev);
    cudaFree(h->mom);
    cudaFree(h->mom_prev);
    cudaFree(h->dense);
    cudaFree(h->partials);
    cudaFree(h->red);
    if (h->red_host) cudaFreeHost(h->red_host);
    if (h->host_stage) cudaFreeHost(h->host_stage);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->s) cudaStreamDestroy(h->s);
    delete h;
}

cdf_status enter3(cdf_lb3d *h) {
    CK3(cudaEventRecord(h->ev_in, h->user));
    CK3(cudaStreamWaitEvent(h->s, h->ev_in, 0));
    return CDF_OK;
}
cdf_status leave3(cdf_lb3d *h) {
    CK3(cudaEventRecord(h->ev_out, h->s));
    CK3(cudaStreamWaitEvent(h->user, h->ev_out, 0));
    return CDF_OK;
}

cudaError_t launch_any3(cdf_lb3d *h, int src, bool with_moments) {
    return launch_step3(h->P, h->buf[src], h->buf[src ^ 1], h->sprev, with_moments ? h->mom : nullptr, h->block, h->s);
}

cdf_status run_steps3(cdf_lb3d *h, long long n) {
    while (n > 0) {
        if (n >= kGraphSteps) {
            const int wm = n == kGraphSteps ? 1 : 0;
            cudaGraphExec_t &ge = h->graph[h->cur][wm];
            if (!ge) {
                cudaGraph_t graph = nullptr;
                CK3(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
                int src = h->cur;
                cudaError_t e = cudaSuccess;
                for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k, src ^= 1)
                    e = launch_any3(h, src, wm && k == kGraphSteps - 1);
                cudaError_t e2 = cudaStreamEndCapture(h->s, &graph);
                if (e != cudaSuccess || e2 != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    return fail3(CDF_ECUDA, "step capture failed: %s",
                                 cudaGetErrorString(e != cudaSuccess ? e : e2));
                }
                e = cudaGraphInstantiate(&ge, graph, 0);
                cudaGraphDestroy(graph);
                CK3(e);
            }
            CK3(cudaGraphLaunch(ge, h->s));
            n -= kGraphSteps;
            h->t += kGraphSteps;
        } else {
            for (long long j = 0; j < n; ++j) {
                CK3(launch_any3(h, h->cur, j == n - 1));
                h->cur ^= 1;
            }
            h->t += n;
            n = 0;
        }
    }
    return CDF_OK;
}

// FP64 sums through the 2-D reduction: the 3-D moment stack [phi.., u_x, u_y, u_z, p]
// read as a 2-D stack of (ny nz) rows with m + 1 "scalars" (phi_0..phi_{m-1}, u_x).
cdf_status reduce3(cdf_lb3d *h, const float *nw, const float *od, double *host_out) {
    CK3(launch_reduce(nw, od, h->nx, h->ny * h->nz, h->pitch, h->plane, h->m + 1, h->partials, h->red, h->s));
    const int nq = reduce_quantities(h->m + 1);
    CK3(cudaMemcpyAsync(h->red_host, h->red, nq * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK3(cudaStreamSynchronize(h->s));
    std::memcpy(host_out, h->red_host, nq * sizeof(double));
    return CDF_OK;
}

cdf_status autotune3(cdf_lb3d *h) {
    auto key = std::make_tuple(h->nx, h->ny, h->nz, h->m, h->P.chemotaxis);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) { h->block = it->second; return CDF_OK; }
    }
    const dim3 cands[] = {dim3(32, 4), dim3(32, 8), dim3(64, 2), dim3(64, 4), dim3(128, 1), dim3(128, 2),
                          dim3(256, 1)};
    cudaEvent_t a, b;
    CK3(cudaEventCreate(&a));
    CK3(cudaEventCreate(&b));
    float best = 1e30f;
    dim3 best_b = h->block;
    const long long nodes = (long long)h->nx * h->ny * h->nz;
    const int reps = nodes >= (1 << 22) ? 4 : 16;
    for (const dim3 &c : cands) {
        if ((int)c.x > 2 * h->nx && c.x > 32) continue;
        h->block = c;
        for (int w = 0; w < 2; ++w) CK3(launch_any3(h, 0, false));
        CK3(cudaEventRecord(a, h->s));
        for (int r = 0; r < reps; ++r) CK3(launch_any3(h, r & 1, false));
        CK3(cudaEventRecord(b, h->s));
        CK3(cudaEventSynchronize(b));
        float ms = 0;
        CK3(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) { best = ms; best_b = c; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->block = best_b;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best_b;
    return CDF_OK;
}

}  // namespace

extern "C" {

cdf_status cdf_lb3d_create(const cdf_grid3 *grid, int m, const cdf_diffusion *dif, double nu, const cdf_source *src,
                           const cdf_force3 *frc, const cdf_boundaries3 *bc, const cdf_options3 *opt,
                           cdf_lb3d **out) {
    if (!out) return fail3(CDF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !dif || !src || !frc || !bc || !opt) return fail3(CDF_EINVAL, "NULL argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail3(CDF_EINVAL, "grid sizes must be >= 1");
    if (m < 1 || m > kMaxM3) return fail3(CDF_EINVAL, "3-D solver: 1 <= m <= 3");
    if ((long long)((grid->nx + 31) / 32 * 32) * grid->ny * grid->nz >= (1LL << 31))
        return fail3(CDF_EINVAL, "3-D lattice too large (pitch x ny x nz must stay below 2^31)");
    if (!(nu > 0.0)) return fail3(CDF_EINVAL, "nu must be positive");
    if (!(opt->rho0 > 0.0)) return fail3(CDF_EINVAL, "rho0 must be positive");
    if ((dif->kind == CDF_D_CHEMOTAXIS || src->kind == CDF_S_CONSUMPTION) && m < 2)
        return fail3(CDF_EINVAL, "chemotaxis and consumption need m >= 2");
    if (dif->kind != CDF_D_CONST && dif->kind != CDF_D_CHEMOTAXIS) return fail3(CDF_EINVAL, "bad diffusion kind");
    if (src->kind < CDF_S_NONE || src->kind > CDF_S_CONSUMPTION) return fail3(CDF_EINVAL, "bad source kind");
    for (int a = 0; a < 3; ++a)
        if ((bc->side[2 * a].kind == CDF_BC_PERIODIC) != (bc->side[2 * a + 1].kind == CDF_BC_PERIODIC))
            return fail3(CDF_EINVAL, "opposite sides must both be periodic or both walls");
    if (opt->block_x < 0 || opt->block_y < 0 || (opt->block_x > 0 && (opt->block_x % 32 != 0 || opt->block_y < 1 ||
                                                                    opt->block_x * opt->block_y > 256)))
        return fail3(CDF_EINVAL, "block must be a multiple of 32 wide and at most 256 threads");

    Lb3Params P{};
    P.nx = grid->nx;
    P.ny = grid->ny;
    P.nz = grid->nz;
    P.pitch = (grid->nx + 31) / 32 * 32;
    P.plane = (long long)P.pitch * grid->ny * grid->nz;
    P.m = m;
    // Eq. omega-D with cs_s^2 = 1/4: B = 4 D + I/2 (constant part), omega = B^-1
    double B[kMaxM * kMaxM], Binv[kMaxM * kMaxM];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) B[a * m + b] = 4.0 * dif->D[a * m + b] + (a == b ? 0.5 : 0.0);
    if (!invert(m, B, Binv)) return fail3(CDF_EINVAL, "D / cs^2 + I / 2 is singular");
    for (int k = 0; k < m * m; ++k) P.omega[k] = (float)Binv[k];
    P.omega_f = (float)(1.0 / (3.0 * nu + 0.5));
    P.chemotaxis = dif->kind == CDF_D_CHEMOTAXIS;
    P.chi4 = (float)(4.0 * dif->chi);
    P.c_star = (float)dif->c_star;
    P.eps2 = (float)(dif->eps * dif->eps);
    P.r_regularised = dif->r_regularised;
    P.skind = src->kind;
    for (int a = 0; a < m; ++a) P.S[a] = (float)src->S[a];
    P.k = (float)src->k;
    double fb = frc->F0;
    for (int a = 0; a < m; ++a) {
        P.beta[a] = (float)frc->beta[a];
        fb -= frc->beta[a] * frc->phi_ref[a];
    }
    P.Fbase = (float)fb;
    for (int d = 0; d < 3; ++d) P.g[d] = (float)frc->g[d];
    P.rho0 = (float)opt->rho0;
    for (int a = 0; a < m; ++a) P.phi_ref[a] = (float)opt->phi_ref[a];
    for (int d = 0; d < 3; ++d) {
        P.periodic[d] = bc->side[2 * d].kind == CDF_BC_PERIODIC;
        P.gref[d] = P.periodic[d] ? 0.f : (float)opt->p_ref_grad[d];
    }
    P.xc = 0.5f * (float)(grid->nx - 1);
    P.yc = 0.5f * (float)(grid->ny - 1);
    P.zc = 0.5f * (float)(grid->nz - 1);
    for (int sdx = 0; sdx < 6; ++sdx) {
        const cdf_side &sd = bc->side[sdx];
        P.dirichlet[sdx] = 0u;
        if (sd.kind != CDF_BC_WALL) continue;
        for (int a = 0; a < m; ++a) {
            if (sd.scalar[a] == CDF_SC_DIRICHLET) P.dirichlet[sdx] |= 1u << a;
            P.abb[sdx][a] = (float)(0.25 * (sd.value[a] - opt->phi_ref[a]));
        }
    }

    cdf_lb3d *h = new (std::nothrow) cdf_lb3d;
    if (!h) return fail3(CDF_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return fail3(CDF_ECUDA, "no CUDA device"); }
    h->nx = grid->nx;
    h->ny = grid->ny;
    h->nz = grid->nz;
    h->m = m;
    h->pitch = P.pitch;
    h->plane = P.plane;
    h->planes = 19 + 7 * m;
    h->sprev_planes = src->kind == CDF_S_CONSUMPTION ? 1 : 0;
    h->user = static_cast<cudaStream_t>(opt->cuda_stream);
    h->P = P;
    Guard g(h->device);
    const size_t n = (size_t)h->nx * h->ny * h->nz;
    const size_t pop = (size_t)h->planes * h->plane * 4, momb = (size_t)(m + 4) * h->plane * 4;
    const int nq = reduce_quantities(m + 1);
    bool ok = cudaMalloc((void **)&h->buf[0], pop) == cudaSuccess && cudaMalloc((void **)&h->buf[1], pop) == cudaSuccess &&
              cudaMalloc((void **)&h->sprev, (size_t)h->plane * 4) == cudaSuccess &&
              cudaMalloc((void **)&h->mom, momb) == cudaSuccess && cudaMalloc((void **)&h->mom_prev, momb) == cudaSuccess &&
              cudaMalloc((void **)&h->dense, (size_t)h->planes * n * 4) == cudaSuccess &&
              cudaMalloc((void **)&h->partials, (size_t)nq * kReduceBlocks * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&h->red, (size_t)nq * sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void **)&h->red_host, (size_t)nq * sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void **)&h->host_stage, (size_t)(m + 4) * n * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release3(h);
        return fail3(CDF_ENOMEM, "device allocation of %.1f MB failed", 2.0 * pop / 1e6);
    }
    if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaMemsetAsync(h->buf[0], 0, pop, h->s) != cudaSuccess || cudaMemsetAsync(h->buf[1], 0, pop, h->s) != cudaSuccess ||
        cudaMemsetAsync(h->sprev, 0, (size_t)h->plane * 4, h->s) != cudaSuccess ||
        cudaMemsetAsync(h->mom, 0, momb, h->s) != cudaSuccess) {
        release3(h);
        return fail3(CDF_ECUDA, "stream / memset set-up failed");
    }
    cdf_status st = CDF_OK;
    if (opt->block_x > 0)
        h->block = dim3(opt->block_x, opt->block_y, 1);
    else if ((st = autotune3(h)) != CDF_OK) {
        release3(h);
        return st;
    }
    if (cudaStreamSynchronize(h->s) != cudaSuccess) {
        release3(h);
        return fail3(CDF_ECUDA, "set-up failed");
    }
    *out = h;
    return CDF_OK;
}

void cdf_lb3d_destroy(cdf_lb3d *h) {
    if (!h) return;
    {
        Guard g(h->device);
        cudaStreamSynchronize(h->s);
    }
    release3(h);
}

cdf_status cdf_lb3d_init_moments(cdf_lb3d *h, const double *phi, const double *u, const double *p) {
    if (!h || !phi || !u) return fail3(CDF_EINVAL, "NULL argument");
    Guard g(h->device);
    const size_t n = (size_t)h->nx * h->ny * h->nz;
    CK3(cudaStreamSynchronize(h->s));  // the staging buffer may still feed an earlier copy
    float *host = h->host_stage;
    for (int a = 0; a < h->m; ++a)
        for (size_t i = 0; i < n; ++i) host[a * n + i] = (float)phi[a * n + i];
    for (size_t i = 0; i < 3 * n; ++i) host[h->m * n + i] = (float)u[i];
    for (size_t i = 0; i < n; ++i) host[(h->m + 3) * n + i] = p ? (float)p[i] : 0.f;
    cdf_status st = enter3(h);
    if (st != CDF_OK) return st;
    CK3(cudaMemcpyAsync(h->dense, host, (size_t)(h->m + 4) * n * 4, cudaMemcpyHostToDevice, h->s));
    CK3(launch_init3(h->P, h->dense, h->buf[0], h->sprev, h->mom, h->s));
    h->cur = 0;
    h->t = 0;
    h->initialised = true;
    return leave3(h);
}

cdf_status cdf_lb3d_step(cdf_lb3d *h, long long n) {
    if (!h) return fail3(CDF_EINVAL, "NULL handle");
    if (n < 0) return fail3(CDF_EINVAL, "n must be >= 0");
    if (!h->initialised) return fail3(CDF_EINVAL, "state not initialised");
    if (n == 0) return CDF_OK;
    Guard g(h->device);
    cdf_status st = enter3(h);
    if (st != CDF_OK) return st;
    if ((st = run_steps3(h, n)) != CDF_OK) return st;
    return leave3(h);
}

cdf_status cdf_lb3d_run_to_steady(cdf_lb3d *h, double tol, long long check_every, long long max_steps,
                                  long long *steps_taken, double *residual) {
    if (!h) return fail3(CDF_EINVAL, "NULL handle");
    if (!h->initialised) return fail3(CDF_EINVAL, "state not initialised");
    if (check_every < 1 || max_steps < 0 || !(tol > 0.0)) return fail3(CDF_EINVAL, "bad tol / check_every / max_steps");
    Guard g(h->device);
    cdf_status st = enter3(h);
    if (st != CDF_OK) return st;
    const int m1 = h->m + 1;  // the reduction's view: phi.., u_x as scalars, then u_y, u_z
    const size_t momb = (size_t)(h->m + 4) * h->plane * 4;
    double q[3 * kMaxM + 5];
    long long taken = 0;
    double R = INFINITY;
    cdf_status result = CDF_ENOTCONVERGED;
    while (taken < max_steps) {
        CK3(cudaMemcpyAsync(h->mom_prev, h->mom, momb, cudaMemcpyDeviceToDevice, h->s));
        const long long k = std::min(check_every, max_steps - taken);
        if ((st = run_steps3(h, k)) != CDF_OK) return st;
        taken += k;
        if ((st = reduce3(h, h->mom, h->mom_prev, q)) != CDF_OK) return st;
        if (q[3 * m1 + 4] > 0) { result = CDF_EUNSTABLE; break; }
        // scalars one by one, the velocity as one vector field (a component that
        // stays at round-off level, e.g. u_z of a z-independent flow, has no
        // meaningful relative change of its own)
        R = 0.0;
        for (int f = 0; f < h->m; ++f) R = std::max(R, q[m1 + f] / std::max(q[2 * m1 + 2 + f], 1e-300));
        double du = 0.0, su = 0.0;
        for (int f = h->m; f < m1 + 2; ++f) {
            du += q[m1 + f];
            su += q[2 * m1 + 2 + f];
        }
        R = std::max(R, du / std::max(su, 1e-300));
        if (k == check_every && R < tol) { result = CDF_OK; break; }
    }
    if (steps_taken) *steps_taken = taken;
    if (residual) *residual = R;
    if ((st = leave3(h)) != CDF_OK) return st;
    if (result == CDF_EUNSTABLE) return fail3(CDF_EUNSTABLE, "non-finite moments after %lld steps", taken);
    if (result == CDF_ENOTCONVERGED)
        return fail3(CDF_ENOTCONVERGED, "residual %.3e above tol %.3e after %lld steps", R, tol, taken);
    return CDF_OK;
}

cdf_status cdf_lb3d_moments(cdf_lb3d *h, double *host_out) {
    if (!h || !host_out) return fail3(CDF_EINVAL, "NULL argument");
    if (!h->initialised) return fail3(CDF_EINVAL, "state not initialised");
    Guard g(h->device);
    cdf_status st = enter3(h);
    if (st != CDF_OK) return st;
    const size_t n = (size_t)h->nx * h->ny * h->nz * (h->m + 4);
    CK3(launch_pack3(h->P, h->mom, h->dense, h->s));
    CK3(cudaMemcpyAsync(h->host_stage, h->dense, n * 4, cudaMemcpyDeviceToHost, h->s));
    CK3(cudaStreamSynchronize(h->s));
    for (size_t i = 0; i < n; ++i) host_out[i] = h->host_stage[i];
    return leave3(h);
}

cdf_status cdf_lb3d_mass(cdf_lb3d *h, double *sums) {
    if (!h || !sums) return fail3(CDF_EINVAL, "NULL argument");
    if (!h->initialised) return fail3(CDF_EINVAL, "state not initialised");
    Guard g(h->device);
    cdf_status st = enter3(h);
    if (st != CDF_OK) return st;
    double q[3 * kMaxM + 5];
    if ((st = reduce3(h, h->mom, nullptr, q)) != CDF_OK) return st;
    for (int a = 0; a < h->m; ++a) sums[a] = q[a];
    return leave3(h);
}

cdf_status cdf_lb3d_populations(cdf_lb3d *h, double *f, double *hf) {
    if (!h) return fail3(CDF_EINVAL, "NULL handle");
    if (!h->initialised) return fail3(CDF_EINVAL, "state not initialised");
    Guard g(h->device);
    cdf_status st = enter3(h);
    if (st != CDF_OK) return st;
    const size_t n = (size_t)h->nx * h->ny * h->nz;
    std::vector<float> tmp((size_t)h->planes * n);
    CK3(launch_export3(h->P, h->buf[h->cur], h->dense, h->s));
    CK3(cudaMemcpyAsync(tmp.data(), h->dense, tmp.size() * 4, cudaMemcpyDeviceToHost, h->s));
    CK3(cudaStreamSynchronize(h->s));
    if (hf)
        for (size_t i = 0; i < 19 * n; ++i) hf[i] = tmp[i];
    if (f)
        for (size_t i = 0; i < (size_t)7 * h->m * n; ++i) f[i] = tmp[19 * n + i];
    return leave3(h);
}

cdf_status cdf_lb3d_get_info(const cdf_lb3d *h, cdf_info3 *out) {
    if (!h || !out) return fail3(CDF_EINVAL, "NULL argument");
    out->nx = h->nx;
    out->ny = h->ny;
    out->nz = h->nz;
    out->m = h->m;
    out->pitch = h->pitch;
    out->block_x = (int)h->block.x;
    out->block_y = (int)h->block.y;
    out->bytes_per_lup = 2.0 * h->planes * 4.0 + 8.0 * h->sprev_planes;
    out->t = h->t;
    return CDF_OK;
}

void *cdf_lb3d_stream(const cdf_lb3d *h) { return h ? static_cast<void *>(h->s) : nullptr; }

}  // extern "C"
