// Device-side building blocks of the fused lattice Boltzmann step (Zhan, Chai &
// Shi, arXiv:2101.03055): FP32 lattice constants, storage types, equilibria, the
// node collision and the node update of the pull scheme.  Included by the
// single-lattice kernels (lb_kernels.cu) and the batched kernel (lb_batch.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>
#include <utility>

#include "lb_internal.h"

namespace cdflb {
namespace dev {

// Lattice constants of Eq. D2Q5 and Eq. D2Q9 in FP32.  Rounding 1/3, 1/6,
// 1/9, 1/36 independently would break the discrete conservation identities by
// a few 1e-8 per collision, and because scalar mass, fluid momentum and the
// mean pressure are neutral (conserved) modes the error would pile up linearly
// over the run.  The constants below are chosen so that, for the rounded
// values themselves, sum W = 1 (scalars), 3 sum W c_x^2 = 1 and
// 3 sum_{i!=0} W = kC (fluid) hold exactly; they differ from the exact
// weights by at most 1.2e-7 relative.
//   kW5  = fl(1/6)                W_1..4 of D2Q5;   kW50 = 1 - 4 kW5
//   kA1  = 3 W_1..4 of D2Q9 ~ 1/3; kA5 = 3 W_5..8 ~ 1/12;  2 kA1 + 4 kA5 = 1
//   kC   = 4 kA1 + 4 kA5 ~ 5/3 (= (1 - W_0)/cs^2);  kQ = 3/2 - kC/2 ~ 2/3
constexpr float kW5 = 0x1.555556p-3f;
constexpr float kW50 = 0x1.555554p-2f;
constexpr float kA1 = 0x1.555554p-2f;
constexpr float kA5 = 0x1.555558p-4f;
constexpr float kC = 0x1.aaaaaap+0f;
constexpr float kQ = 0x1.555556p-1f;
constexpr float kInvC = 0x1.333334p-1f;  // fl(1 / kC): Eq. sum-p by one multiply
__host__ __device__ constexpr float kWs(int i) { return i == 0 ? kW50 : kW5; }
__host__ __device__ constexpr float kA9(int i) { return i == 0 ? 0.f : (i < 5 ? kA1 : kA5); }
__host__ __device__ constexpr int kC5x(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
__host__ __device__ constexpr int kC5y(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
__host__ __device__ constexpr int kC9x(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int kC9y(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }

// Nanoseconds of the GPU's global timer: the clock of every bounded wait.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Programmatic dependent launch: a step kernel launched with the programmatic
// stream-serialisation attribute may start while the previous step is still
// running; griddepcontrol.wait holds it until that grid has completed and its
// memory is visible (a no-op without the attribute), and
// griddepcontrol.launch_dependents lets the next step's CTAs be scheduled
// early, which hides the launch gap between the short steps of a small lattice.
__device__ __forceinline__ void pdl_wait_and_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- offset checks (checks builds) -------------------------------------------------
// CDF_CHK(p, off, lim, site) is `off` itself in a normal build.  With
// -DCDF_CHECKS it first tests 0 <= off < lim: an offset outside is recorded in
// the word p.check -- bit 63, the access site in bits 48..62, the offset's low
// 48 bits -- unless an earlier one is there already, and replaced by 0, so the
// access that follows stays inside its buffer and the launch completes.  Sites:
// 1 population load, 2 a node's store offset, 3 shared-memory store,
// 4 shared-memory load, 5 moment-plane load (16-bit storage), 6 batched-step
// load, 7 tile-resident global load, 8 tile-resident shared-memory offset.
#ifdef CDF_CHECKS
__device__ __forceinline__ long long checked_offset(unsigned long long *word, long long off, long long lim,
                                                    int site) {
    if (off >= 0 && off < lim) return off;
    if (word)
        atomicCAS(word, 0ull,
                  (1ull << 63) | ((unsigned long long)(site & 0x7fff) << 48) |
                      ((unsigned long long)off & 0xffffffffffffull));
    return 0;
}
#define CDF_CHK(p, off, lim, site) \
    ((decltype(off))::cdflb::dev::checked_offset((p).check, (long long)(off), (long long)(lim), (site)))
#else
#define CDF_CHK(p, off, lim, site) (off)
#endif

// ---- storage types ---------------------------------------------------------------
// Populations are stored as deviations from a reference state (below) in FP32,
// FP16 or BF16; every collision is computed in FP32.
template <typename T> struct Store;
template <> struct Store<float> {
    __device__ static float load(const float *p) { return __ldg(p); }
    __device__ static void store(float *p, float v) { *p = v; }
};
// FP16 holds the small deviations scaled by 2^12 (exactly invertible), which
// moves them out of FP16's subnormal range: normal numbers then cover
// |d| in [1.5e-8, 16].
constexpr float kHalfScale = 4096.f, kHalfUnscale = 1.f / 4096.f;
// Random bits for the stochastic rounding of the value pair (x, y) in slot k of a
// node's encoding: the lowbias32 integer hash (C. Wellons' published constants) of
// the two FP32 bit patterns and the slot.  The rounding is then a deterministic
// function of the values (bitwise reproducible, independent of where the node
// sits in the lattice), while its errors are uncorrelated between populations and
// nodes and average to zero.
__device__ __forceinline__ unsigned sr_bits(float x, float y, unsigned k) {
    unsigned h = __float_as_uint(x) ^ (__float_as_uint(y) * 0x9E3779B1u) ^ (k * 0x85EBCA77u);
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}
// encode2: the pair (x, y) rounded stochastically to the 16-bit type with one
// cvt.rs (sm_100 and later): each value goes to one of its two 16-bit neighbours
// with the probabilities that make the expected rounded value the value itself,
// so the rounding of the stored deviations acts as a zero-mean perturbation
// instead of a fixed forcing at a steady state.
template <> struct Store<__half> {
    __device__ static __half encode(float v) { return __float2half_rn(v * kHalfScale); }
    __device__ static float decode(__half q) { return __half2float(q) * kHalfUnscale; }
    __device__ static float load(const __half *p) { return decode(__ldg(p)); }
    __device__ static void store(__half *p, float v) { *p = encode(v); }
    __device__ static void encode2(float x, float y, unsigned k, __half &qx, __half &qy) {
        unsigned d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;"
            : "=r"(d)
            : "f"(y * kHalfScale), "f"(x * kHalfScale), "r"(sr_bits(x, y, k)));
        qx = __ushort_as_half((unsigned short)(d & 0xffffu));
        qy = __ushort_as_half((unsigned short)(d >> 16));
    }
};
template <> struct Store<__nv_bfloat16> {
    __device__ static __nv_bfloat16 encode(float v) { return __float2bfloat16_rn(v); }
    __device__ static float decode(__nv_bfloat16 q) { return __bfloat162float(q); }
    __device__ static float load(const __nv_bfloat16 *p) { return decode(__ldg(p)); }
    __device__ static void store(__nv_bfloat16 *p, float v) { *p = encode(v); }
    __device__ static void encode2(float x, float y, unsigned k, __nv_bfloat16 &qx, __nv_bfloat16 &qy) {
        unsigned d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(y), "f"(x), "r"(sr_bits(x, y, k)));
        qx = __ushort_as_bfloat16((unsigned short)(d & 0xffffu));
        qy = __ushort_as_bfloat16((unsigned short)(d >> 16));
    }
};

// Population load of the step.  A kernel that runs one step per launch reads
// data that is read-only for the launch (non-coherent path).  The persistent
// batched kernel reads buffers that other blocks wrote earlier in the same
// launch, which the non-coherent path may not do: it uses ordinary cached
// loads (ld.global.ca), made current by the acquire fence of its grid barrier.
template <typename T, bool kCoherent>
__device__ __forceinline__ float load_pop(const T *p) {
    if constexpr (kCoherent) return __ldca(p);
    else return Store<T>::load(p);
}

// Reference state of the deviation variables at node x (FP32 storage):
//   scalars  f_ref_i,a = W_i phi_ref_a                      (constant)
//   fluid    h_ref_i   = h^eq_i(p_ref(x), u = 0)            (Eq. heq)
//            p_ref(x)  = G . (x - x_c), G the hydrostatic gradient of the mean force
// The collision below is written in these variables; it is the same update as
// Eqs. evolution12/evolution3 term by term, with phi = phi_ref + sum_i f'_i,
// u = sum_i c_i h'_i + F/2 (sum_i c_i h_ref_i = 0) and p = p_ref(x) + p'.
__device__ __forceinline__ float pref_at(const LbParams &p, int x, int y) {
    return fmaf(p.gref[0], (float)x - p.xc, __fmul_rn(p.gref[1], (float)y - p.yc));
}

// ---- paired FP32 lanes -----------------------------------------------------------
// F2 carries one FP32 value of each of two nodes.  Its arithmetic is the paired
// FP32 instructions of sm_100 and later (__ffma2_rn, __fadd2_rn, __fmul2_rn):
// one instruction for both lanes, each lane rounded exactly as the scalar
// fmaf / __fadd_rn / __fmul_rn rounds it.  a - b is fma(b, -1, a) and -a is
// a * -1, both exact.  The node update below is written once for a value type
// V, float or F2, so a kernel that updates two nodes per thread with V = F2
// gives every node the bits of the scalar update with half of its arithmetic
// instructions (the loads, stores and pull table stay per node).
struct F2 {
    float2 v;
};
template <class T>
struct IsF2 {
    static constexpr bool value = false;
};
template <>
struct IsF2<F2> {
    static constexpr bool value = true;
};
template <class A, class B, class C = float>
using IfF2 = typename std::enable_if<IsF2<A>::value || IsF2<B>::value || IsF2<C>::value, F2>::type;

__device__ __forceinline__ float2 as2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 as2(F2 a) { return a.v; }
template <class V>
__device__ __forceinline__ V splat(float a) {
    if constexpr (IsF2<V>::value) return F2{make_float2(a, a)};
    else return a;
}
__device__ __forceinline__ F2 pack2(float a, float b) { return F2{make_float2(a, b)}; }
__device__ __forceinline__ float lane(float a, int) { return a; }
__device__ __forceinline__ float lane(F2 a, int k) { return k ? a.v.y : a.v.x; }

// vfma / vmul: fmaf / __fmul_rn for float, their paired forms for F2 (a float
// operand is used in both lanes)
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
template <class A, class B, class C>
__device__ __forceinline__ IfF2<A, B, C> vfma(A a, B b, C c) {
    return F2{__ffma2_rn(as2(a), as2(b), as2(c))};
}
template <class A, class B>
__device__ __forceinline__ IfF2<A, B> vmul(A a, B b) {
    return F2{__fmul2_rn(as2(a), as2(b))};
}
template <class A, class B>
__device__ __forceinline__ IfF2<A, B> operator*(A a, B b) {
    return F2{__fmul2_rn(as2(a), as2(b))};
}
template <class A, class B>
__device__ __forceinline__ IfF2<A, B> operator+(A a, B b) {
    return F2{__fadd2_rn(as2(a), as2(b))};
}
template <class A, class B>
__device__ __forceinline__ IfF2<A, B> operator-(A a, B b) {
    return F2{__ffma2_rn(as2(b), make_float2(-1.f, -1.f), as2(a))};
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2{__fmul2_rn(a.v, make_float2(-1.f, -1.f))}; }
// per lane: 1 / a, 1 / sqrt(a), and the step a >= t ? 1 : 0
__device__ __forceinline__ float vrcp(float a) { return 1.f / a; }
__device__ __forceinline__ F2 vrcp(F2 a) { return pack2(1.f / a.v.x, 1.f / a.v.y); }
__device__ __forceinline__ float vrsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ F2 vrsqrt(F2 a) { return pack2(rsqrtf(a.v.x), rsqrtf(a.v.y)); }
__device__ __forceinline__ float vstep(float a, float t) { return a >= t ? 1.f : 0.f; }
__device__ __forceinline__ F2 vstep(F2 a, float t) { return pack2(vstep(a.v.x, t), vstep(a.v.y, t)); }

// c_i . (ax, ay) for a lattice direction (components 0 or +-1, at least one
// nonzero), without multiplications by the components.
template <class V>
__device__ __forceinline__ V cdot(int cx, int cy, V ax, V ay) {
    if (cx == 0) return cy > 0 ? ay : -ay;
    if (cy == 0) return cx > 0 ? ax : -ax;
    if (cx > 0) return cy > 0 ? ax + ay : ax - ay;
    return cy > 0 ? ay - ax : -(ax + ay);
}

template <class V>
__device__ __forceinline__ V cutoff(const LbParams &p, V c) {
    // r(c): step (Sec. 3.1.3) or regularised (Sec. 3.1.2)
    if (p.r_regularised) {
        const V d = c - p.c_star;
        return 0.5f * vfma(d, vrsqrt(vfma(d, d, p.eps2)), 1.f);
    }
    return vstep(c, p.c_star);
}

template <int M, class V = float>
struct NodeOut {
    V phi[M], ux, uy, pr, s1;
};

// Scalar equilibrium deviation, Eq. feq-phi with lambda = I, vartheta = 0:
// f^eq_i - W_i phi_ref = W_i (phi' + 3 phi c_i.u) for the moving directions; the
// rest direction is phi' minus the moving ones, so the sum is phi' up to one rounding.
// One moving direction j = 1..4 of the scalar equilibrium deviation
// W_j (phi' + 3 phi c_j.u); shared by the collision and by the pull of the
// 16-bit storage so both evaluate it bit for bit the same way.
template <class V>
__device__ __forceinline__ V feq_dir(int j, V phid, V t3phi, V ux, V uy) {
    return vmul(kW5, vfma(t3phi, cdot(kC5x(j), kC5y(j), ux, uy), phid));
}

template <int M, class V>
__device__ __forceinline__ void scalar_equilibrium(const V (&phid)[M], const V (&phi)[M], V ux, V uy,
                                                   V (&feq)[M][5]) {
#pragma unroll
    for (int b = 0; b < M; ++b) {
        const V t = 3.f * phi[b];
#pragma unroll
        for (int j = 1; j < 5; ++j) feq[b][j] = feq_dir(j, phid[b], t, ux, uy);
        feq[b][0] = phid[b] - ((feq[b][1] + feq[b][3]) + (feq[b][2] + feq[b][4]));
    }
}

// u.u with a fixed rounding.  The kernels share these device functions but are
// compiled in different contexts; every multiply-add whose FMA contraction the
// compiler could decide differently in each context is written out (fmaf,
// __fmul_rn), so all kernels round identically and agree bit for bit.
template <class V>
__device__ __forceinline__ V usq_of(V ux, V uy) { return vfma(ux, ux, vmul(uy, uy)); }

// Fluid equilibrium deviation (Eq. heq): h^eq_i(p, u) - h^eq_i(p_ref, 0)
//   = kA_i (q + 1.5 (c_i.u)^2) + kA_i c_i.u,  q = p' - 0.5 u.u  (i != 0),   -kC p' - kQ u.u  (i = 0).
// The first term is even in c_i, the second odd: heq_even / heq_odd give them for the
// directions i = 1, 2, 5, 6, whose opposites 3, 4, 7, 8 take the odd part with the
// other sign.  Every user (the collision, which forms them once per pair of
// opposite directions, the initialisation and the 16-bit storage) evaluates them
// with these functions, so all agree bit for bit.
template <class V>
__device__ __forceinline__ V heq_even(int i, V q, V ux, V uy) {
    const V cu = cdot(kC9x(i), kC9y(i), ux, uy);
    return vmul(kA9(i), vfma(1.5f, vmul(cu, cu), q));
}
template <class V>
__device__ __forceinline__ V heq_odd(int i, V ux, V uy) { return vmul(kA9(i), cdot(kC9x(i), kC9y(i), ux, uy)); }
template <class V>
__device__ __forceinline__ V fluid_equilibrium(int i, V prd, V ux, V uy, V usq) {
    if (i == 0) return vfma(-kC, prd, vmul(-kQ, usq));
    const int b = (i == 3 || i == 4 || i == 7 || i == 8) ? i - 2 : i;  // the direction of the pair in 1, 2, 5, 6
    const V E = heq_even(b, vfma(-0.5f, usq, prd), ux, uy), O = heq_odd(b, ux, uy);
    return b == i ? E + O : E - O;
}

// The second-order part of Eq. force per unit varphi, W_i (uF + Fu):(c_i c_i -
// cs^2 I) / (2 cs^4): 3 W_i (3 (c_i.u)(c_i.F) - u.F) for i != 0 and, so that the
// nine sum to zero with the exact-identity weights, -(3 - kC) u.F for i = 0.
template <class V>
__device__ __forceinline__ V force2_dir(int i, V ux, V uy, V Fx, V Fy, V uF) {
    if (i == 0) return vmul(-(3.f - kC), uF);
    const V cu = cdot(kC9x(i), kC9y(i), ux, uy), cF = cdot(kC9x(i), kC9y(i), Fx, Fy);
    return vmul(kA9(i), vfma(vmul(3.f, cu), cF, -uF));
}

// Scalar moments of one node (Eq. sum-phi) and the closures of Sec. 3 that
// depend on them: the cut-off r(phi_1), the source S(phi) and S(t - 1).
// sp1: S_1(t-1) of the consumption closure; `first` uses S(t-1) = S(t).
template <int M, class V = float>
struct ScalarState {
    V phid[M], phi[M], S[M], Sp[M], r;
};
template <int M, class V>
__device__ __forceinline__ void scalar_closures(const LbParams &p, const V (&f)[M][5], V sp1, bool first,
                                                ScalarState<M, V> &s) {
#pragma unroll
    for (int a = 0; a < M; ++a) {
        s.phid[a] = ((f[a][0] + f[a][1]) + (f[a][2] + f[a][3])) + f[a][4];
        s.phi[a] = p.phi_ref[a] + s.phid[a];
    }
    s.r = splat<V>(0.f);
    if (M >= 2 && (p.chemotaxis || p.skind == 2)) s.r = cutoff(p, s.phi[M >= 2 ? 1 : 0]);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        s.S[a] = splat<V>((p.skind == 1) ? p.S[a] : 0.f);
        s.Sp[a] = s.S[a];
    }
    if (M >= 2 && p.skind == 2) {
        s.S[1] = -p.k * s.phi[0] * s.r;
        s.Sp[1] = first ? s.S[1] : sp1;
    }
}

// Eq. omega-D.  Constant D: omega from the host.  Chemotaxis: omega^-1 =
// B + delta e_0 e_1^T with delta = -3 chi phi_0 r, inverted by Sherman-Morrison.
template <int M, class V>
__device__ __forceinline__ void relaxation_matrix(const LbParams &p, const ScalarState<M, V> &s, V (&om)[M][M]) {
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) om[a][b] = splat<V>(p.omega[a * M + b]);
    if (M >= 2 && p.chemotaxis) {
        const V delta = -p.chi3 * s.phi[0] * s.r;
        // 1 / (1 + delta omega_10); omega_10 = 0 (a diagonal constant part, as in
        // the benchmark closures) makes it exactly 1, so the quotient is skipped
        // by a branch that is uniform over the launch
        const float o10 = p.omega[(M >= 2 ? 1 : 0) * M];
        V den = splat<V>(1.f);
        if (o10 != 0.f) den = vrcp(vfma(delta, o10, 1.f));
        float col0[M], row1[M];
#pragma unroll
        for (int a = 0; a < M; ++a) {
            col0[a] = p.omega[a * M];
            row1[a] = p.omega[(M >= 2 ? 1 : 0) * M + a];
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) om[a][b] = vfma(-vmul(vmul(delta, den), col0[a]), row1[b], om[a][b]);
    }
}

// Eq. evolution12 for the scalars of one node: f*_i,a = f_i,a - sum_b omega_ab
// (f_i,b - f^eq_i,b) + W_i S_a + (W_i S_a - W_i S_a(t-1)) / 2 + G_i,a with the
// auxiliary source G_i,a = 3 W_i c_i . J_a (J from Eq. Gi, or from the time
// difference of phi u in Case 1 of Sec. 2.1).  The non-equilibrium part f - f^eq
// is formed first, so a node at equilibrium stays there exactly (no rounding-level
// forcing of the conserved scalar mass).
template <int M, class V>
__device__ __forceinline__ void scalar_collide(V (&f)[M][5], const ScalarState<M, V> &s, V ux, V uy,
                                               const V (&om)[M][M], const V (&Jx)[M], const V (&Jy)[M]) {
    V feq[M][5];
    scalar_equilibrium<M>(s.phid, s.phi, ux, uy, feq);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        V neq[M];
#pragma unroll
        for (int b = 0; b < M; ++b) neq[b] = f[b][i] - feq[b][i];
#pragma unroll
        for (int a = 0; a < M; ++a) {
            V coll = splat<V>(0.f);
#pragma unroll
            for (int b = 0; b < M; ++b) coll = vfma(om[a][b], neq[b], coll);
            const V G = (i == 0) ? splat<V>(0.f) : vmul(3.f * kW5, cdot(kC5x(i), kC5y(i), Jx[a], Jy[a]));
            f[a][i] = (f[a][i] - coll) + vfma(kWs(i), vfma(1.5f, s.S[a], vmul(-0.5f, s.Sp[a])), G);
        }
    }
}

// Collision of one node (Eqs. evolution12, evolution3) in deviation variables.
// f, h: pre-collision deviations, overwritten by the post-collision ones.  prx:
// p_ref at the node.  sp1: S_1(t-1) of the consumption closure; `first` uses
// S(t-1) = S(t) (initialisation).  V = F2: two nodes, one per lane.
template <int M, class V>
__device__ __forceinline__ void collide(const LbParams &p, V (&f)[M][5], V (&h)[9], V prx, V sp1, bool first,
                                        NodeOut<M, V> &o) {
    ScalarState<M, V> s;
    scalar_closures<M>(p, f, sp1, first, s);
    V fm = splat<V>(p.Fbase);
#pragma unroll
    for (int a = 0; a < M; ++a) fm = vfma(p.beta[a], s.phi[a], fm);
    const V Fx = p.g[0] * fm, Fy = p.g[1] * fm;

    // Eq. sum-u and Eq. sum-p (varphi = 0):
    // p = cs^2/(1 - W0) [sum_{i!=0} h_i - W0 u.u / (2 cs^2)] = (sum_{i!=0} h_i - kQ u.u) / kC,
    // taken as a product with fl(1 / kC) (one rounding more than the quotient)
    const V jx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
    const V jy = (h[2] - h[4]) + (h[5] - h[8]) + (h[6] - h[7]);
    const V ux = vfma(0.5f, Fx, jx), uy = vfma(0.5f, Fy, jy);
    const V usq = usq_of(ux, uy);
    const V snr = ((h[1] + h[2]) + (h[3] + h[4])) + ((h[5] + h[6]) + (h[7] + h[8]));
    V prd = vmul(vfma(-kQ, usq, snr), kInvC);
    // varphi != 0 (a branch uniform over the launch): the appendix's pressure,
    // p = (sum_{i!=0} h_i - kQ u.u - varphi (1/omega - 1/2) (W_0/cs^2) u.F) / kC
    const V uF = vfma(ux, Fx, vmul(uy, Fy));
    if (p.varphi != 0.f) prd = vmul(vfma(-p.varphi_p, uF, vfma(-kQ, usq, snr)), kInvC);

    V om[M][M];
    relaxation_matrix<M>(p, s, om);

    // Eq. Gi: G_{i,a} = 3 W_i c_i . J_a,  J_a = sum_b (delta_ab - omega_ab / 2)(u S_b + phi_b F)
    V Jx[M], Jy[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        V jxa = splat<V>(0.f), jya = splat<V>(0.f);
#pragma unroll
        for (int b = 0; b < M; ++b) {
            const V c = vfma(-0.5f, om[a][b], a == b ? 1.f : 0.f);
            jxa = vfma(c, vfma(ux, s.S[b], s.phi[b] * Fx), jxa);
            jya = vfma(c, vfma(uy, s.S[b], s.phi[b] * Fy), jya);
        }
        Jx[a] = jxa;
        Jy[a] = jya;
    }
    scalar_collide<M>(f, s, ux, uy, om, Jx, Jy);

    // Eq. evolution3 with Eq. force, weighted by (1 - omega_f / 2):
    //   h*_i = h_i - wf (h_i - h^eq_i) + fw F_i,   fw = 1 - wf / 2,
    //   F_i = 3 W_i c_i.F  +  varphi [3 W_i (3 (c_i.u)(c_i.F) - u.F)  (i != 0),  -(3 - kC) u.F  (i = 0)].
    // The non-equilibrium part h - h^eq is formed first, so a node at equilibrium stays
    // there exactly.  For i != 0, h^eq_i = kA_i (q + 1.5 (c_i.u)^2) + kA_i c_i.u with
    // q = p' - u.u / 2 (Eq. heq), and the first-order force kA_i c_i.F is odd in c_i:
    // a direction and its opposite share the even parts and take the odd parts with
    // opposite signs, so each pair forms them once.
    const float wf = p.omega_f, fw = 1.f - 0.5f * wf;
    {
        V F0 = splat<V>(0.f);
        if (p.varphi != 0.f) F0 = vmul(p.varphi, force2_dir(0, ux, uy, Fx, Fy, uF));
        h[0] = vfma(fw, F0, vfma(-wf, h[0] - fluid_equilibrium(0, prd, ux, uy, usq), h[0]));
    }
    const V q = vfma(-0.5f, usq, prd);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = k < 2 ? k + 1 : k + 3, io = i + 2;  // i = 1, 2, 5, 6 and their opposites io = 3, 4, 7, 8
        const float kA = kA9(i);
        const V cu = cdot(kC9x(i), kC9y(i), ux, uy), cF = cdot(kC9x(i), kC9y(i), Fx, Fy);
        const V E = heq_even(i, q, ux, uy), O = heq_odd(i, ux, uy), Fo = vmul(kA, cF);
        V Fi = Fo, Fopp = -Fo;
        if (p.varphi != 0.f) {
            const V f2 = vmul(kA, vfma(vmul(3.f, cu), cF, -uF));  // even in c_i
            Fi = vfma(p.varphi, f2, Fo);
            Fopp = vfma(p.varphi, f2, -Fo);
        }
        h[i] = vfma(fw, Fi, vfma(-wf, h[i] - (E + O), h[i]));
        h[io] = vfma(fw, Fopp, vfma(-wf, h[io] - (E - O), h[io]));
    }
#pragma unroll
    for (int a = 0; a < M; ++a) o.phi[a] = s.phi[a];
    o.ux = ux;
    o.uy = uy;
    o.pr = prx + prd;
    o.s1 = (M >= 2) ? s.S[M >= 2 ? 1 : 0] : splat<V>(0.f);
}

// Case 1 of Sec. 2.1: the convection cross-diffusion equations in a prescribed
// steady velocity (ux, uy), no fluid.  The auxiliary source is
// G_i,a = sum_b (delta_ab - omega_ab / 2) W_i c_i . d_t(phi_b u) / cs^2 with the
// first-order explicit difference d_t(phi_b u) = u (phi_b - phi_prev_b).
// phi_prev: phi(t - 1), overwritten with phi(t).
template <int M>
__device__ __forceinline__ void collide_case1(const LbParams &p, float (&f)[M][5], float ux, float uy,
                                              float (&phi_prev)[M], float sp1, bool first, NodeOut<M> &o) {
    ScalarState<M> s;
    scalar_closures<M>(p, f, sp1, first, s);
    float om[M][M];
    relaxation_matrix<M>(p, s, om);
    float Jx[M], Jy[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        float ja = 0.f;
#pragma unroll
        for (int b = 0; b < M; ++b) ja = fmaf(fmaf(-0.5f, om[a][b], a == b ? 1.f : 0.f), s.phi[b] - phi_prev[b], ja);
        Jx[a] = __fmul_rn(ux, ja);
        Jy[a] = __fmul_rn(uy, ja);
    }
    scalar_collide<M>(f, s, ux, uy, om, Jx, Jy);
#pragma unroll
    for (int a = 0; a < M; ++a) {
        o.phi[a] = s.phi[a];
        phi_prev[a] = s.phi[a];
    }
    o.ux = ux;
    o.uy = uy;
    o.pr = 0.f;
    o.s1 = (M >= 2) ? s.S[M >= 2 ? 1 : 0] : 0.f;
}

template <int M>
__device__ __forceinline__ void write_moments(float *moments, long long P, long long o0, const NodeOut<M> &o) {
#pragma unroll
    for (int a = 0; a < M; ++a) moments[a * P + o0] = o.phi[a];
    moments[M * P + o0] = o.ux;
    moments[(M + 1) * P + o0] = o.uy;
    moments[(M + 2) * P + o0] = o.pr;
}

template <int M, typename T>
__device__ __forceinline__ void store_node(T *out, long long P, long long o0, const float (&f)[M][5],
                                           const float (&h)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<T>::store(out + i * P + o0, h[i]);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) Store<T>::store(out + (9 + 5 * a + i) * P + o0, f[a][i]);
}

// ---- the pull of one node -------------------------------------------------------
// Where the pre-collision populations of node (x, y) come from: for each fluid
// direction i the source plane, node and pressure-reference shift; for each
// scalar direction the source plane and node and the wall side whose rule
// applies (-1 for a regular link).  mk(sx, sy) names a source node (an element
// offset, a pair of coordinates, ...), so the same rules serve the
// global-memory kernels, the tile-resident kernel and the 16-bit storage.
// kInterior: the caller guarantees that no link of the node crosses a wall or
// wraps; every source is then x - c_i and the selects fold away.
// Is node (x, y) at least one node away from every edge of the lattice?
__device__ __forceinline__ bool inner_node(const LbParams &p, int x, int y) {
    return x >= 1 && x + 1 < p.nx && y >= 1 && y + 1 < p.ny;
}

template <class Pos>
struct PullTable {
    int hplane[9];
    Pos hpos[9];
    float hshift[9];
    int splane[5];
    Pos spos[5];
    int side[5];
};

template <bool kInterior, class MakePos>
__device__ __forceinline__ PullTable<decltype(std::declval<MakePos>()(0, 0))> pull_table(const LbParams &p, int x,
                                                                                           int y, const MakePos &mk) {
    using Pos = decltype(mk(0, 0));
    struct Src {
        int plane;
        Pos pos;
        float shift;
    };
    // Neighbour coordinates (periodic wrap) and wall crossings of the pull links.
    int xw = x - 1, xe = x + 1, ys = y - 1, yn = y + 1;
    bool cw = false, ce = false, cs = false, cn = false;
    if (!kInterior) {
        cw = xw < 0 && !p.periodic_x;
        ce = xe >= p.nx && !p.periodic_x;
        cs = ys < 0 && !p.periodic_y;
        cn = yn >= p.ny && !p.periodic_y;
        xw = xw < 0 ? p.nx - 1 : xw;
        xe = xe >= p.nx ? 0 : xe;
        ys = ys < 0 ? p.ny - 1 : ys;
        yn = yn >= p.ny ? 0 : yn;
    }
    const Pos o0 = mk(x, y), pw = mk(xw, y), pe = mk(xe, y), ps = mk(x, ys), pn = mk(x, yn);
    const Pos psw = mk(xw, ys), pse = mk(xe, ys), pne = mk(xe, yn), pnw = mk(xw, yn);
    // axis- and diagonal-link shifts (products kept out of FMA contraction so that
    // every kernel adds them with the same rounding)
    const float ax = __fmul_rn(kA1, p.gref[0]), ay = __fmul_rn(kA1, p.gref[1]);
    const float dx5 = __fmul_rn(kA5, p.gref[0]), dy5 = __fmul_rn(kA5, p.gref[1]);
    const bool fw = p.freeslip[0], fe = p.freeslip[1], fs = p.freeslip[2], fn = p.freeslip[3];

    // Fluid, D2Q9: h_i(x) = h*_j(src).  Regular link: j = i, src = x - c_i.  No-slip
    // wall: bounce-back j = opp(i), src = x.  Free-slip wall: the specular image j
    // from the neighbour along the wall.  Corner links: bounce-back.  Every
    // source is chosen by selects, so all loads can issue before any arithmetic.
    // The shift is the change of the pressure reference, kA_j G.(src - x).
    Src sh[9];
    sh[0] = Src{0, o0, 0.f};
    sh[1] = cw ? Src{3, o0, 0.f} : Src{1, pw, -ax};
    sh[2] = cs ? Src{4, o0, 0.f} : Src{2, ps, -ay};
    sh[3] = ce ? Src{1, o0, 0.f} : Src{3, pe, ax};
    sh[4] = cn ? Src{2, o0, 0.f} : Src{4, pn, ay};
    {   // (1,1) from (x-1, y-1)
        Src v{5, psw, -dx5 - dy5};
        v = (cw || cs) ? Src{7, o0, 0.f} : v;
        v = (cw && !cs && fw) ? Src{6, ps, -dy5} : v;
        v = (cs && !cw && fs) ? Src{8, pw, -dx5} : v;
        sh[5] = v;
    }
    {   // (-1,1) from (x+1, y-1)
        Src v{6, pse, dx5 - dy5};
        v = (ce || cs) ? Src{8, o0, 0.f} : v;
        v = (ce && !cs && fe) ? Src{5, ps, -dy5} : v;
        v = (cs && !ce && fs) ? Src{7, pe, dx5} : v;
        sh[6] = v;
    }
    {   // (-1,-1) from (x+1, y+1)
        Src v{7, pne, dx5 + dy5};
        v = (ce || cn) ? Src{5, o0, 0.f} : v;
        v = (ce && !cn && fe) ? Src{8, pn, dy5} : v;
        v = (cn && !ce && fn) ? Src{6, pe, dx5} : v;
        sh[7] = v;
    }
    {   // (1,-1) from (x-1, y+1)
        Src v{8, pnw, -dx5 + dy5};
        v = (cw || cn) ? Src{6, o0, 0.f} : v;
        v = (cw && !cn && fw) ? Src{7, pn, dy5} : v;
        v = (cn && !cw && fn) ? Src{5, pw, -dx5} : v;
        sh[8] = v;
    }
    PullTable<Pos> t;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        t.hplane[i] = sh[i].plane;
        t.hpos[i] = sh[i].pos;
        t.hshift[i] = sh[i].shift;
    }
    // Scalars, D2Q5: bounce-back f*_opp(i)(x) (no flux) or anti-bounce-back
    // -f*_opp(i)(x) + 2 W_i phi_w (Dirichlet) at the wall `side`.  The axis
    // sources are the nodes of the fluid's axis sources.
    t.splane[0] = 0;
    t.splane[1] = cw ? 3 : 1;
    t.splane[2] = cs ? 4 : 2;
    t.splane[3] = ce ? 1 : 3;
    t.splane[4] = cn ? 2 : 4;
#pragma unroll
    for (int i = 0; i < 5; ++i) t.spos[i] = sh[i].pos;
    t.side[0] = -1;
    t.side[1] = cw ? 0 : -1;
    t.side[2] = cs ? 2 : -1;
    t.side[3] = ce ? 1 : -1;
    t.side[4] = cn ? 3 : -1;
    return t;
}

// Pre-collision populations of node (x, y) in deviation variables: the loads of
// the pull table through ld(plane, pos), then the pressure-reference shifts and,
// in deviations, the anti-bounce-back value -f'*_opp(i)(x) + 2 W_i (phi_w - phi_ref).
template <int M, bool kInterior, class MakePos, class Load>
__device__ __forceinline__ void pull_node(const LbParams &p, int x, int y, const MakePos &mk, const Load &ld,
                                          float (&f)[M][5], float (&h)[9]) {
    const auto t = pull_table<kInterior>(p, x, y, mk);
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = ld(t.hplane[i], t.hpos[i]);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) f[a][i] = ld(9 + 5 * a + t.splane[i], t.spos[i]);
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] += t.hshift[i];
    if (!kInterior) {
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            if (t.side[i] >= 0) {
#pragma unroll
                for (int a = 0; a < M; ++a)
                    if ((p.dirichlet[t.side[i]] >> a) & 1u) f[a][i] = p.abb[t.side[i]][a] - f[a][i];
            }
        }
    }
}

// The scalar part of pull_node (Case 1 of Sec. 2.1 has no fluid populations).
template <int M, bool kInterior, class MakePos, class Load>
__device__ __forceinline__ void pull_scalars(const LbParams &p, int x, int y, const MakePos &mk, const Load &ld,
                                             float (&f)[M][5]) {
    const auto t = pull_table<kInterior>(p, x, y, mk);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) f[a][i] = ld(9 + 5 * a + t.splane[i], t.spos[i]);
    if (!kInterior) {
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            if (t.side[i] >= 0) {
#pragma unroll
                for (int a = 0; a < M; ++a)
                    if ((p.dirichlet[t.side[i]] >> a) & 1u) f[a][i] = p.abb[t.side[i]][a] - f[a][i];
            }
        }
    }
}

// ---- the fused step ------------------------------------------------------------
// One node of the fused step (x < nx, y < ny) on global-memory buffers: pull,
// moments, collision, store.  kInterior: the caller guarantees that the node is
// at least one node away from every edge of the lattice (no link crosses a wall
// or wraps); the pull then reads x - c_i directly.  Both forms give the same
// bits for such a node.
// sp_in / sp_out: S_1(t - 1) of the consumption closure in, S_1(t) out (the
// same plane, or two planes that alternate with the population buffers).
template <int M, typename T, bool kL2 = false, bool kInterior = false>
__device__ __forceinline__ void step_node(const LbParams &p, int x, int y, const T *__restrict__ in,
                                          T *__restrict__ out, const float *sp_in, float *sp_out,
                                          float *__restrict__ moments) {
    const long long P = p.plane;
    const int pitch = p.pitch;
    const auto mk = [pitch](int sx, int sy) { return sy * pitch + sx; };
    const auto ld = [in, P, &p](int plane, int off) {
        return load_pop<T, kL2>(in + plane * P + CDF_CHK(p, off, P, 6));
    };
    const int o0 = CDF_CHK(p, y * pitch + x, P, 2);
    const bool consume = (M >= 2 && p.skind == 2);
    const float sp1 = consume ? (kL2 ? __ldca(sp_in + o0) : sp_in[o0]) : 0.f;
    float h[9], f[M][5];
    pull_node<M, kInterior>(p, x, y, mk, ld, f, h);

    NodeOut<M> o;
    collide<M>(p, f, h, pref_at(p, x, y), sp1, false, o);
    store_node<M, T>(out, P, o0, f, h);
    if (consume) sp_out[o0] = o.s1;
    if (moments) write_moments<M>(moments, P, o0, o);
}

// step_node with the planes given one pointer each (Planes): the form of the
// single-lattice step kernels.  Same node update, same bits.
template <int M, typename T, bool kInterior = false>
__device__ __forceinline__ void step_node_planes(const LbParams &p, int x, int y, const Planes<T> &pl,
                                                 const float *sp_in, float *sp_out, float *__restrict__ moments) {
    const int pitch = p.pitch;
    const auto mk = [pitch](int sx, int sy) { return sy * pitch + sx; };
    const auto ld = [&pl, &p](int plane, int off) {
        return Store<T>::load(pl.in[plane] + CDF_CHK(p, off, p.plane, 1));
    };
    const int o0 = CDF_CHK(p, y * pitch + x, p.plane, 2);
    const bool consume = (M >= 2 && p.skind == 2);
    const float sp1 = consume ? sp_in[o0] : 0.f;
    float h[9], f[M][5];
    pull_node<M, kInterior>(p, x, y, mk, ld, f, h);

    NodeOut<M> o;
    collide<M>(p, f, h, pref_at(p, x, y), sp1, false, o);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<T>::store(pl.out[i] + o0, h[i]);
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int i = 0; i < 5; ++i) Store<T>::store(pl.out[9 + 5 * a + i] + o0, f[a][i]);
    if (consume) sp_out[o0] = o.s1;
    if (moments) write_moments<M>(moments, p.plane, o0, o);
}

}  // namespace dev
}  // namespace cdflb
