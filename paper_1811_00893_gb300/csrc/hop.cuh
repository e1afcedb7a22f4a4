// Device building blocks of the hopping term (Eq. 1) shared by the
// single-lattice kernels (dslash.cu) and the multi-lattice batch (batch.cu):
// spin projection and reconstruction, neighbour indices, the per-site sum
// over the eight hops, the fused epilogue and shared-memory link staging.
#pragma once

#include "clover.cuh"
#include "internal.cuh"

namespace wl {

// (1 + S gamma_mu) projection / reconstruction in the chiral basis
// (gamma_5 = diag(1,1,-1,-1)); S = -1 is Eq. 1's forward projector
// (1 - gamma_mu), S = +1 the backward one.  With u0 = W h0, u1 = W h1 the
// four spin rows of (1 + S gamma_mu) W psi are (u0, u1, r2, r3):
//   mu=x: h0 = psi0 + S i psi3, h1 = psi1 + S i psi2, r2 = -S i u1, r3 = -S i u0
//   mu=y: h0 = psi0 - S psi3,   h1 = psi1 + S psi2,   r2 =  S u1,   r3 = -S u0
//   mu=z: h0 = psi0 + S i psi2, h1 = psi1 - S i psi3, r2 = -S i u0, r3 =  S i u1
//   mu=t: h0 = psi0 + S psi2,   h1 = psi1 + S psi3,   r2 =  S u0,   r3 =  S u1
// The signs are compile-time: a +-1 factor is an add or a subtract, never a
// multiply (which matters for the double-float type).

// a + S b for S = +1 / -1
template <int S, typename T>
__device__ __forceinline__ cx<T> add_s(cx<T> a, cx<T> b)
{
    if constexpr (S > 0) return a + b;
    else return a - b;
}

template <int MU, int S, typename T>
__device__ __forceinline__ void project(cx<T> (&h0)[3], cx<T> (&h1)[3], const cx<T> (&q)[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<T> p0 = q[c], p1 = q[3 + c], p2 = q[6 + c], p3 = q[9 + c];
        if constexpr (MU == 0) {
            h0[c] = add_s<S>(p0, mul_i(p3));
            h1[c] = add_s<S>(p1, mul_i(p2));
        } else if constexpr (MU == 1) {
            h0[c] = add_s<-S>(p0, p3);
            h1[c] = add_s<S>(p1, p2);
        } else if constexpr (MU == 2) {
            h0[c] = add_s<S>(p0, mul_i(p2));
            h1[c] = add_s<-S>(p1, mul_i(p3));
        } else {
            h0[c] = add_s<S>(p0, p2);
            h1[c] = add_s<S>(p1, p3);
        }
    }
}

// add colour row a of the reconstructed (1 + S gamma_mu) W psi to acc
template <int MU, int S, typename T>
__device__ __forceinline__ void reconstruct(cx<T> (&acc)[12], int a, cx<T> u0, cx<T> u1)
{
    acc[a] = acc[a] + u0;
    acc[3 + a] = acc[3 + a] + u1;
    if constexpr (MU == 0) {
        acc[6 + a] = add_s<-S>(acc[6 + a], mul_i(u1));
        acc[9 + a] = add_s<-S>(acc[9 + a], mul_i(u0));
    } else if constexpr (MU == 1) {
        acc[6 + a] = add_s<S>(acc[6 + a], u1);
        acc[9 + a] = add_s<-S>(acc[9 + a], u0);
    } else if constexpr (MU == 2) {
        acc[6 + a] = add_s<-S>(acc[6 + a], mul_i(u0));
        acc[9 + a] = add_s<S>(acc[9 + a], mul_i(u1));
    } else {
        acc[6 + a] = add_s<S>(acc[6 + a], u0);
        acc[9 + a] = add_s<S>(acc[9 + a], u1);
    }
}

// w0 h0 + w1 h1 + w2 h2 (one row of the SU(3) matrix-vector product).  The
// first product is written with explicit fused multiply-adds, like the two
// after it (cmac), so that the compiler has no contraction left to choose:
// every kernel that inlines it rounds alike (the decomposed kernels rely on
// this to reproduce the undivided result bit for bit).
template <typename T>
__device__ __forceinline__ cx<T> dot3(cx<T> w0, cx<T> w1, cx<T> w2, const cx<T> (&h)[3])
{
    cx<T> u = {fma(w0.re, h[0].re, -(w0.im * h[0].im)), fma(w0.re, h[0].im, w0.im * h[0].re)};
    cmac(u, w1, h[1]);
    cmac(u, w2, h[2]);
    return u;
}

// Double-float: the six real products of each output component are summed
// with their rounding errors collected in one FP32 word and folded in once at
// the end (exact TwoProd of the high parts, the cross terms hi*lo in FP32,
// TwoSum for each addition) -- about 12 FP32 operations per product instead
// of ~17 for a normalised df64 multiply-add.
struct LazySum {
    float s, e;  // value = s + e, unnormalised
};
__device__ __forceinline__ void lazy_start(LazySum& L, df64 a, df64 b)
{
    L.s = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -L.s);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    L.e = __fmaf_rn(a.lo, b.hi, pe);
}
__device__ __forceinline__ void lazy_mac(LazySum& L, df64 a, df64 b)  // L += a b
{
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s, t;
    two_sum(L.s, p, s, t);
    L.s = s;
    L.e = __fadd_rn(L.e, __fadd_rn(t, pe));
}
__device__ __forceinline__ df64 lazy_value(const LazySum& L)
{
    df64 r;
    two_sum(L.s, L.e, r.hi, r.lo);
    return r;
}

template <>
__device__ __forceinline__ cx<df64> dot3<df64>(cx<df64> w0, cx<df64> w1, cx<df64> w2,
                                               const cx<df64> (&h)[3])
{
    LazySum re, im;
    lazy_start(re, w0.re, h[0].re);
    lazy_mac(re, -w0.im, h[0].im);
    lazy_mac(re, w1.re, h[1].re);
    lazy_mac(re, -w1.im, h[1].im);
    lazy_mac(re, w2.re, h[2].re);
    lazy_mac(re, -w2.im, h[2].im);
    lazy_start(im, w0.re, h[0].im);
    lazy_mac(im, w0.im, h[0].re);
    lazy_mac(im, w1.re, h[1].im);
    lazy_mac(im, w1.im, h[1].re);
    lazy_mac(im, w2.re, h[2].im);
    lazy_mac(im, w2.im, h[2].re);
    return {lazy_value(re), lazy_value(im)};
}

template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate(cx<T> (&acc)[12], const cx<T> (&q)[12],
                                           const cx<T> (&W)[9])
{
    cx<T> h0[3], h1[3];
    project<MU, S>(h0, h1, q);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        reconstruct<MU, S>(acc, a, dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h0),
                           dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h1));
}

// Row a (entries 3a .. 3a+2) of link d for the FP64-sized layouts (nine
// 16-byte planes per link): the wide types read one row at a time to keep
// fewer registers live.
template <int P>
__device__ __forceinline__ void load_link_row(cx<typename Prec<P>::real> (&w)[3], const void* base,
                                              long long Vh, int d, long long i, int a);
template <>
__device__ __forceinline__ void load_link_row<WL_F64>(cx<double> (&w)[3], const void* base,
                                                      long long Vh, int d, long long i, int a)
{
    const double2* p = (const double2*)base + ((long long)d * 9 + 3 * a) * Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 v = p[k * Vh + i];
        w[k] = {v.x, v.y};
    }
}
template <>
__device__ __forceinline__ void load_link_row<WL_DF64>(cx<df64> (&w)[3], const void* base,
                                                       long long Vh, int d, long long i, int a)
{
    const float4* p = (const float4*)base + ((long long)d * 9 + 3 * a) * Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 v = p[k * Vh + i];
        w[k] = {df64(v.x, v.y), df64(v.z, v.w)};
    }
}

// n / (Lxh, Ly, Lz)[k] without an integer divide (Geom::dm, ds);
// WL_FAST_DIV=0 builds the plain division instead (for comparisons)
#ifndef WL_FAST_DIV
#define WL_FAST_DIV 1
#endif
__device__ __forceinline__ int geo_div(const Geom& g, int k, int n)
{
#if WL_FAST_DIV
    return g.dm[k] ? (int)(__umulhi((unsigned)n, g.dm[k]) >> g.ds[k]) : n;
#else
    return n / (k == 0 ? g.Lxh : g.L[k]);
#endif
}

// Half indices of the eight neighbours (order +x, -x, +y, -y, +z, -z, +t, -t)
// of output site i on parity p, with periodic wrap-around.
__device__ __forceinline__ void neighbours(const Geom& g, int p, int i, int (&nb)[8])
{
    const int r0 = geo_div(g, 0, i);  // (y, z, t) row
    const int xh = i - r0 * g.Lxh;
    const int r1 = geo_div(g, 1, r0);
    const int y = r0 - r1 * g.L[1];
    const int t = geo_div(g, 2, r1);
    const int z = r1 - t * g.L[2];
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int row = i - xh;
    const int sy = (int)g.sy, sz = (int)g.sz, st = (int)g.st;
    nb[0] = row + ((x + 1 == g.L[0] ? 0 : x + 1) >> 1);
    nb[1] = row + ((x == 0 ? g.L[0] - 1 : x - 1) >> 1);
    nb[2] = (y == g.L[1] - 1) ? i - (g.L[1] - 1) * sy : i + sy;
    nb[3] = (y == 0) ? i + (g.L[1] - 1) * sy : i - sy;
    nb[4] = (z == g.L[2] - 1) ? i - (g.L[2] - 1) * sz : i + sz;
    nb[5] = (z == 0) ? i + (g.L[2] - 1) * sz : i - sz;
    nb[6] = (t == g.L[3] - 1) ? i - (g.L[3] - 1) * st : i + st;
    nb[7] = (t == 0) ? i + (g.L[3] - 1) * st : i - st;
}

// neighbours() plus a mask of the hops that cross the lattice boundary (bit
// d set for hop d): forward hops leaving x_mu = L_mu - 1, backward hops
// leaving x_mu = 0.  Used by the compressed-link kernels, whose stored links
// carry no boundary phase.
__device__ __forceinline__ void neighbours(const Geom& g, int p, int i, int (&nb)[8], unsigned& cross)
{
    neighbours(g, p, i, nb);
    const int r0 = geo_div(g, 0, i);
    const int xh = i - r0 * g.Lxh;
    const int r1 = geo_div(g, 1, r0);
    const int y = r0 - r1 * g.L[1];
    const int t = geo_div(g, 2, r1);
    const int z = r1 - t * g.L[2];
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int c[4] = {x, y, z, t};
    cross = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        if (c[mu] == g.L[mu] - 1) cross |= 1u << (2 * mu);
        if (c[mu] == 0) cross |= 1u << (2 * mu + 1);
    }
}

// ---------------------------------------------------------------------------
// Link storage formats of the hopping kernels.  LF = 0: all nine entries of
// each hop matrix, boundary phase folded in.  LF = 1 (FP32 / FP16 only): the
// first two rows of the SU(3) matrix without the phase; the third row is
// rebuilt as conj(row0 x row1) (unitarity with det = 1), and the phase is
// applied to the projected half spinor of boundary-crossing hops.  Twelve
// reals instead of eighteen per hop: 384 instead of 576 bytes per site in
// FP32 (192 instead of 288 in FP16).  LF = 2 (FP32, single-RHS launches): eight
// reals per hop (load_link_r8), 256 bytes per site.
// ---------------------------------------------------------------------------

template <int P, int LF>
struct LinkLayout;  // 16-byte planes, then narrower planes; bytes per site
template <>
struct LinkLayout<WL_F64, 0> {
    static constexpr int n16 = 72, nsmall = 0, small_bytes = 8, bytes = 1152;
};
template <>
struct LinkLayout<WL_F32, 0> {
    static constexpr int n16 = 32, nsmall = 8, small_bytes = 8, bytes = 576;
};
template <>
struct LinkLayout<WL_DF64, 0> {
    static constexpr int n16 = 72, nsmall = 0, small_bytes = 8, bytes = 1152;
};
template <>
struct LinkLayout<WL_F16, 0> {
    static constexpr int n16 = 16, nsmall = 8, small_bytes = 4, bytes = 288;
};
template <>
struct LinkLayout<WL_F32, 1> {  // per hop: 3 float4 = rows 0 and 1
    static constexpr int n16 = 24, nsmall = 0, small_bytes = 8, bytes = 384;
};
template <>
struct LinkLayout<WL_F16, 1> {  // per hop: 1 uint4 (4 half2) + 1 uint2 (2 half2)
    static constexpr int n16 = 8, nsmall = 8, small_bytes = 8, bytes = 192;
};
template <>
struct LinkLayout<WL_F32, 2> {  // per hop: 2 float4 (8 reals)
    static constexpr int n16 = 16, nsmall = 0, small_bytes = 8, bytes = 256;
};

// row 2 = conj(row 0 x row 1)
template <typename T>
__device__ __forceinline__ void su3_third_row(cx<T> (&w)[9])
{
    w[6] = conj(w[1] * w[5] - w[2] * w[4]);
    w[7] = conj(w[2] * w[3] - w[0] * w[5]);
    w[8] = conj(w[0] * w[4] - w[1] * w[3]);
}

// Compressed link of hop d at index i of planes with stride Vh.
template <int P>
__device__ __forceinline__ void load_link_r12(cx<float> (&w)[9], const void* base, long long Vh, int d,
                                              long long i);
template <>
__device__ __forceinline__ void load_link_r12<WL_F32>(cx<float> (&w)[9], const void* base, long long Vh,
                                                      int d, long long i)
{
    const float4* p = (const float4*)base + (long long)d * 3 * Vh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 t = p[k * Vh + i];
        w[2 * k] = {t.x, t.y};
        w[2 * k + 1] = {t.z, t.w};
    }
    su3_third_row(w);
}
template <>
__device__ __forceinline__ void load_link_r12<WL_F16>(cx<float> (&w)[9], const void* base, long long Vh,
                                                      int d, long long i)
{
    const uint4 t = ((const uint4*)base)[(long long)d * Vh + i];
    const uint2 u = ((const uint2*)((const uint4*)base + 8 * Vh))[(long long)d * Vh + i];
    const float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), e = h2f(t.w), f = h2f(u.x), h = h2f(u.y);
    w[0] = {a.x, a.y};
    w[1] = {b.x, b.y};
    w[2] = {c.x, c.y};
    w[3] = {e.x, e.y};
    w[4] = {f.x, f.y};
    w[5] = {h.x, h.y};
    su3_third_row(w);
}

// Eight reals per SU(3) matrix.  With rows (a, b, c) taken in the cyclic order
// that puts the smaller of |W_00|, |W_10| first -- (W0, W1, W2), or (W1, W2, W0)
// ("shifted") -- so that n = |a2|^2 + |a3|^2 = 1 - |a1|^2 >= 1/2, a hop stores
// two planes of float4:
//   (a2.re, a2.im, a3.re, a3.im), (b1.re, b1.im, t_a + 3 [shifted], t_c),
// t_x = tan(arg(x1) / 4) in [-1, 1].  The rest follows from unitarity and
// det = 1: |a1| = sqrt(1 - n); |c1| = sqrt(n - |b1|^2) (the first column is a
// unit vector); b2, b3 solve the two linear equations (a, b) = 0 and
// conj(c1) = a2 b3 - a3 b2 (row c is conj(a x b)), whose determinant is n;
// then c2, c3 from c = conj(a x b).  The phases come back from t by the
// tangent half-angle and double-angle formulas (rational: one reciprocal).
// Elements near zero come back with ~sqrt of the FP32 rounding as absolute
// error (a square root of a small difference); everything else to FP32
// rounding.
__device__ __forceinline__ cx<float> unit_from_tan4(float t)
{
    const float d = __frcp_rn(fmaf(t, t, 1.0f));
    const float c = (1.0f - t * t) * d, s = 2.0f * t * d;  // cos, sin of 2 atan(t)
    return {(c - s) * (c + s), 2.0f * s * c};
}

template <int P>
__device__ __forceinline__ void load_link_r8(cx<float> (&w)[9], const void* base, long long Vh, int d,
                                             long long i);
template <>
__device__ __forceinline__ void load_link_r8<WL_F32>(cx<float> (&w)[9], const void* base, long long Vh,
                                                     int d, long long i)
{
    const float4* p = (const float4*)base + (long long)d * 2 * Vh;
    const float4 q0 = p[i], q1 = p[Vh + i];
    const bool shift = q1.z > 1.5f;  // t_a + 3 >= 2 when shifted, t_a <= 1 otherwise
    const cx<float> a2 = {q0.x, q0.y}, a3 = {q0.z, q0.w}, b1 = {q1.x, q1.y};
    const float n = fmaf(a2.re, a2.re, fmaf(a2.im, a2.im, fmaf(a3.re, a3.re, a3.im * a3.im)));
    const float nb = fmaf(b1.re, b1.re, b1.im * b1.im);
    const cx<float> a1 = sqrtf(fmaxf(0.0f, 1.0f - n)) * unit_from_tan4(shift ? q1.z - 3.0f : q1.z);
    const cx<float> c1 = sqrtf(fmaxf(0.0f, n - nb)) * unit_from_tan4(q1.w);
    const float inv = __frcp_rn(n);
    const cx<float> ab = conj(a1) * b1;
    const cx<float> b2 = (-inv) * (ab * a2 + conj(a3) * conj(c1));
    const cx<float> b3 = inv * (conj(a2) * conj(c1) - ab * a3);
    const cx<float> c2 = conj(a3 * b1 - a1 * b3), c3 = conj(a1 * b2 - a2 * b1);
    const cx<float> ra[3] = {a1, a2, a3}, rb[3] = {b1, b2, b3}, rc[3] = {c1, c2, c3};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        w[k] = shift ? rc[k] : ra[k];
        w[3 + k] = shift ? ra[k] : rb[k];
        w[6 + k] = shift ? rb[k] : rc[k];
    }
}

// FP16 spinor without its per-site norm applied (the caller scales the
// projected half spinor instead: 12 multiplies per hop instead of 24)
__device__ __forceinline__ void load_spinor_ro_f16_unscaled(cx<float> (&v)[12], float& nrm,
                                                           const void* base, long long Vh, long long i)
{
    const uint4* p = (const uint4*)base;
    nrm = __ldg((const float*)(p + 3 * Vh) + i) * kSpin16Unit;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 t = __ldg(p + k * Vh + i);
        const float2 a = s16_dec(t.x), b = s16_dec(t.y), c = s16_dec(t.z), d = s16_dec(t.w);
        v[4 * k + 0] = {a.x, a.y};
        v[4 * k + 1] = {b.x, b.y};
        v[4 * k + 2] = {c.x, c.y};
        v[4 * k + 3] = {d.x, d.y};
    }
}

// The same with plain loads, for the epilogue's operands (which may be the
// field the launch writes)
__device__ __forceinline__ void load_spinor_f16_unscaled(cx<float> (&v)[12], float& nrm, const void* base,
                                                         long long Vh, long long i)
{
    const uint4* p = (const uint4*)base;
    nrm = ((const float*)(p + 3 * Vh))[i] * kSpin16Unit;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 t = p[k * Vh + i];
        const float2 a = s16_dec(t.x), b = s16_dec(t.y), c = s16_dec(t.z), d = s16_dec(t.w);
        v[4 * k + 0] = {a.x, a.y};
        v[4 * k + 1] = {b.x, b.y};
        v[4 * k + 2] = {c.x, c.y};
        v[4 * k + 3] = {d.x, d.y};
    }
}

// FP16 half h plus the FP32 value c, rounded once in FP32: the result of
// converting h (exactly) and adding in FP32, as one mixed-precision add
// (sm_100 and later) instead of a conversion and an add.
__device__ __forceinline__ float add_f16_f32(unsigned short h, float c)
{
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(h), "f"(c));
    return d;
}

// The projection above on an FP16 spinor given as 12 words (complex entry
// spin * 3 + colour, real part in the low half): spins 2 and 3 are converted
// to FP32 and enter the mixed adds with spins 0 and 1, which stay FP16.  The
// sums are the FP32 sums of the converted values, rounded once.
#ifndef WL_F16_MIXED_ADD
#define WL_F16_MIXED_ADD (!WL_SPINOR16_FIXED)
#endif
template <int MU, int S>
__device__ __forceinline__ void project_f16(cx<float> (&h0)[3], cx<float> (&h1)[3], const unsigned (&w)[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 f2 = h2f(w[6 + c]), f3 = h2f(w[9 + c]);
        const cx<float> p2 = {f2.x, f2.y}, p3 = {f3.x, f3.y};
        cx<float> b0, b1;  // the terms added to spins 0 and 1
        if constexpr (MU == 0) {
            b0 = S > 0 ? mul_i(p3) : -mul_i(p3);
            b1 = S > 0 ? mul_i(p2) : -mul_i(p2);
        } else if constexpr (MU == 1) {
            b0 = S > 0 ? -p3 : p3;
            b1 = S > 0 ? p2 : -p2;
        } else if constexpr (MU == 2) {
            b0 = S > 0 ? mul_i(p2) : -mul_i(p2);
            b1 = S > 0 ? -mul_i(p3) : mul_i(p3);
        } else {
            b0 = S > 0 ? p2 : -p2;
            b1 = S > 0 ? p3 : -p3;
        }
        const unsigned p0 = w[c], p1 = w[3 + c];
        h0[c] = {add_f16_f32((unsigned short)(p0 & 0xffffu), b0.re), add_f16_f32((unsigned short)(p0 >> 16), b0.im)};
        h1[c] = {add_f16_f32((unsigned short)(p1 & 0xffffu), b1.re), add_f16_f32((unsigned short)(p1 >> 16), b1.im)};
    }
}

// The projected half spinor of the FP16 neighbour spinor at index nb, not
// yet multiplied by the neighbour's per-site norm, which is returned in nrm:
// the hop applies it in its reconstruction (one FFMA per value instead of a
// multiply here and an add there).
template <int MU, int S>
__device__ __forceinline__ void load_project_f16(cx<float> (&h0)[3], cx<float> (&h1)[3], float& nrm, const void* in,
                                                 long long Vh, int nb)
{
#if WL_F16_MIXED_ADD && !WL_SPINOR16_FIXED
    unsigned w[12];
    {
        const uint4* p = (const uint4*)in;
        nrm = __ldg((const float*)(p + 3 * Vh) + nb);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 t = __ldg(p + k * Vh + nb);
            w[4 * k + 0] = t.x;
            w[4 * k + 1] = t.y;
            w[4 * k + 2] = t.z;
            w[4 * k + 3] = t.w;
        }
    }
    project_f16<MU, S>(h0, h1, w);
#else
    cx<float> q[12];
    load_spinor_ro_f16_unscaled(q, nrm, in, Vh, nb);
    project<MU, S>(h0, h1, q);
#endif
}

// the projected half spinor of the neighbour spinor at index nb
template <int P, int MU, int S>
__device__ __forceinline__ void load_project(cx<typename Prec<P>::real> (&h0)[3],
                                             cx<typename Prec<P>::real> (&h1)[3], const void* in,
                                             long long Vh, int nb)
{
    using T = typename Prec<P>::real;
    if constexpr (P == WL_F16) {
        float nrm;
        load_project_f16<MU, S>(h0, h1, nrm, in, Vh, nb);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h0[c] = nrm * h0[c];
            h1[c] = nrm * h1[c];
        }
    } else {
        cx<T> q[12];
        load_spinor_ro<P>(q, in, Vh, nb);
        project<MU, S>(h0, h1, q);
    }
}

// acc += s i^K u (K = 0: u, 1: i u, 2: -u, 3: -i u), as two FFMAs
template <int K>
__device__ __forceinline__ void fma_ik(cx<float>& acc, float s, cx<float> u)
{
    if constexpr (K == 0) {
        acc.re = fmaf(s, u.re, acc.re);
        acc.im = fmaf(s, u.im, acc.im);
    } else if constexpr (K == 1) {
        acc.re = fmaf(-s, u.im, acc.re);
        acc.im = fmaf(s, u.re, acc.im);
    } else if constexpr (K == 2) {
        acc.re = fmaf(-s, u.re, acc.re);
        acc.im = fmaf(-s, u.im, acc.im);
    } else {
        acc.re = fmaf(s, u.im, acc.re);
        acc.im = fmaf(-s, u.re, acc.im);
    }
}

// reconstruct() of s (u0, u1): the four spin rows of s (1 + S gamma_mu) W psi
// added with FFMAs (the FP16 hops pass the neighbour's norm as s)
template <int MU, int S>
__device__ __forceinline__ void reconstruct_scaled(cx<float> (&acc)[12], int a, cx<float> u0, cx<float> u1, float s)
{
    fma_ik<0>(acc[a], s, u0);
    fma_ik<0>(acc[3 + a], s, u1);
    if constexpr (MU == 0) {  // rows 2, 3 += -S i (u1, u0)
        fma_ik<(S > 0 ? 3 : 1)>(acc[6 + a], s, u1);
        fma_ik<(S > 0 ? 3 : 1)>(acc[9 + a], s, u0);
    } else if constexpr (MU == 1) {  // rows 2, 3 += (S u1, -S u0)
        fma_ik<(S > 0 ? 0 : 2)>(acc[6 + a], s, u1);
        fma_ik<(S > 0 ? 2 : 0)>(acc[9 + a], s, u0);
    } else if constexpr (MU == 2) {  // rows 2, 3 += (-S i u0, S i u1)
        fma_ik<(S > 0 ? 3 : 1)>(acc[6 + a], s, u0);
        fma_ik<(S > 0 ? 1 : 3)>(acc[9 + a], s, u1);
    } else {  // rows 2, 3 += S (u0, u1)
        fma_ik<(S > 0 ? 0 : 2)>(acc[6 + a], s, u0);
        fma_ik<(S > 0 ? 0 : 2)>(acc[9 + a], s, u1);
    }
}

template <int P, int D, int MU, int S, int LF>
__device__ __forceinline__ void hop_one(cx<typename Prec<P>::real> (&acc)[12], const void* in,
                                        long long Vh, int nb, const void* links, long long lVh,
                                        int li, unsigned cross, const cx<float>* ph)
{
    using T = typename Prec<P>::real;
    if constexpr (P == WL_F16) {  // the neighbour's norm enters the reconstruction
        cx<T> h0[3], h1[3], W[9];
        float nrm;
        load_project_f16<MU, S>(h0, h1, nrm, in, Vh, nb);
        if constexpr (LF == 1) {
            if (cross & (1u << D)) {  // boundary phase: phi forward, conj(phi) backward
                const cx<T> f = (D & 1) ? conj(ph[MU]) : ph[MU];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    h0[c] = f * h0[c];
                    h1[c] = f * h1[c];
                }
            }
            load_link_r12<P>(W, links, lVh, D, li);
        } else {
            load_link<P>(W, links, lVh, D, li);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            reconstruct_scaled<MU, S>(acc, a, dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h0),
                                      dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h1), nrm);
    } else if constexpr (LF >= 1) {
        cx<T> h0[3], h1[3], W[9];
        load_project<P, MU, S>(h0, h1, in, Vh, nb);
        if (cross & (1u << D)) {  // boundary phase: phi forward, conj(phi) backward
            const cx<T> f = (D & 1) ? conj(ph[MU]) : ph[MU];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                h0[c] = f * h0[c];
                h1[c] = f * h1[c];
            }
        }
        if constexpr (LF == 1) load_link_r12<P>(W, links, lVh, D, li);
        else load_link_r8<P>(W, links, lVh, D, li);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            reconstruct<MU, S>(acc, a, dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h0),
                               dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h1));
    } else if constexpr (P == WL_F64) {  // links one row at a time: fewer live registers
        cx<T> h0[3], h1[3];
        load_project<P, MU, S>(h0, h1, in, Vh, nb);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> w[3];
            load_link_row<P>(w, links, lVh, D, li, a);
            reconstruct<MU, S>(acc, a, dot3(w[0], w[1], w[2], h0), dot3(w[0], w[1], w[2], h1));
        }
    } else {  // FP32 (df64 takes hop_site_loop instead)
        cx<T> q[12], W[9];
        load_spinor_ro<P>(q, in, Vh, nb);
        load_link<P>(W, links, lVh, D, li);
        accumulate<MU, S, T>(acc, q, W);
    }
}

// The part of hop_one after the spin projection: given the projected half
// spinor (h0, h1) of hop D, apply the boundary phase (compressed links), the
// link and the reconstruction (scaled by the neighbour's norm s for FP16
// storage, whose h arrive unscaled).  The domain-decomposed kernels use it for
// hops whose half spinor arrives from a neighbouring block; it performs the
// same operations as hop_one.
template <int P, int D, int MU, int S, int LF>
__device__ __forceinline__ void hop_apply(cx<typename Prec<P>::real> (&acc)[12], cx<typename Prec<P>::real> (&h0)[3],
                                          cx<typename Prec<P>::real> (&h1)[3], const void* links, long long lVh,
                                          long long li, unsigned cross, const cx<float>* ph, float s = 1.0f)
{
    using T = typename Prec<P>::real;
    if constexpr (LF >= 1) {
        if (cross & (1u << D)) {
            const cx<T> f = (D & 1) ? conj(ph[MU]) : ph[MU];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                h0[c] = f * h0[c];
                h1[c] = f * h1[c];
            }
        }
    }
    if constexpr (P == WL_F64 && LF == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> w[3];
            load_link_row<P>(w, links, lVh, D, li, a);
            reconstruct<MU, S>(acc, a, dot3(w[0], w[1], w[2], h0), dot3(w[0], w[1], w[2], h1));
        }
    } else {
        cx<T> W[9];
        if constexpr (LF == 1) load_link_r12<P>(W, links, lVh, D, li);
        else if constexpr (LF == 2) load_link_r8<P>(W, links, lVh, D, li);
        else load_link<P>(W, links, lVh, D, li);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if constexpr (P == WL_F16)
                reconstruct_scaled<MU, S>(acc, a, dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h0),
                                          dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h1), s);
            else
                reconstruct<MU, S>(acc, a, dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h0),
                                   dot3(W[3 * a], W[3 * a + 1], W[3 * a + 2], h1));
        }
    }
}

// i^k x for k = 0..3 (multiplication by 1, i, -1, -i: swaps and negations,
// exact in every arithmetic type)
template <typename T>
__device__ __forceinline__ cx<T> mul_ik(cx<T> x, int k)
{
    const bool swap = k & 1, neg_re = k == 1 || k == 2, neg_im = k >= 2;
    cx<T> r = swap ? cx<T>{x.im, x.re} : x;
    if (neg_re) r.re = -r.re;
    if (neg_im) r.im = -r.im;
    return r;
}

// The projection / reconstruction table above as data, for a runtime loop
// over the hops: per direction mu (12 bits each), with S = +1,
//   h0 = psi0 + i^k0 psi[2 + a0],  h1 = psi1 + i^k1 psi[2 + a1],
//   row 2 += i^k2 u[b2],           row 3 += i^k3 u[b3]
// (bits: a0 | k0 << 1 | a1 << 3 | k1 << 4 | b2 << 6 | k2 << 7 | b3 << 9 | k3 << 10);
// S = -1 adds 2 to every k.
__device__ __forceinline__ unsigned hop_code(int mu)
{
    constexpr unsigned long long kTable =
        (1ull | 1ull << 1 | 0ull << 3 | 1ull << 4 | 1ull << 6 | 3ull << 7 | 0ull << 9 | 3ull << 10) |
        (1ull | 2ull << 1 | 0ull << 3 | 0ull << 4 | 1ull << 6 | 0ull << 7 | 0ull << 9 | 2ull << 10) << 12 |
        (0ull | 1ull << 1 | 1ull << 3 | 3ull << 4 | 0ull << 6 | 3ull << 7 | 1ull << 9 | 1ull << 10) << 24 |
        (0ull | 0ull << 1 | 1ull << 3 | 0ull << 4 | 0ull << 6 | 0ull << 7 | 1ull << 9 | 0ull << 10) << 36;
    return (unsigned)(kTable >> (12 * mu)) & 0xfffu;
}

// The double-float type is ALU-bound, and its arithmetic makes a fully
// unrolled eight-hop body too large for the instruction cache (ncu: "no
// instruction" stalls dominated; the loop form runs 2.7x faster).  It runs the
// hops as a loop with the spin structure from hop_code(), the link one row at
// a time.  (Plain FP64 keeps the unrolled form: looped it ran 25 % slower.)
template <int P, bool DAG>
__device__ __forceinline__ void hop_site_loop(cx<typename Prec<P>::real> (&acc)[12], const int (&nb)[8],
                                              long long Vh, const void* in, const void* links,
                                              long long lVh, int li)
{
    using T = typename Prec<P>::real;
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = {(T)0, (T)0};
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const unsigned code = hop_code(d >> 1);
        // forward hops use Eq. 1's (1 - gamma) (S = -1), backward (1 + gamma);
        // the adjoint flips both
        const int sflip = ((d & 1) ? DAG == false : DAG == true) ? 0 : 2;
        const int a0 = code & 1, k0 = ((code >> 1) + sflip) & 3;
        const int a1 = (code >> 3) & 1, k1 = ((code >> 4) + sflip) & 3;
        const int b2 = (code >> 6) & 1, k2 = ((code >> 7) + sflip) & 3;
        const int b3 = (code >> 9) & 1, k3 = ((code >> 10) + sflip) & 3;
        cx<T> h0[3], h1[3];
        {
            cx<T> q[12];
            load_spinor_ro<P>(q, in, Vh, nb[d]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                h0[c] = q[c] + mul_ik(a0 ? q[9 + c] : q[6 + c], k0);
                h1[c] = q[3 + c] + mul_ik(a1 ? q[9 + c] : q[6 + c], k1);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> w[3];
            load_link_row<P>(w, links, lVh, d, li, a);
            const cx<T> u0 = dot3(w[0], w[1], w[2], h0), u1 = dot3(w[0], w[1], w[2], h1);
            acc[a] = acc[a] + u0;
            acc[3 + a] = acc[3 + a] + u1;
            acc[6 + a] = acc[6 + a] + mul_ik(b2 ? u1 : u0, k2);
            acc[9 + a] = acc[9 + a] + mul_ik(b3 ? u1 : u0, k3);
        }
    }
}

// acc = H_{p,1-p} in at the output site whose neighbours are nb.  The links
// are read from planes of stride lVh at index li (the global link field, or a
// tile of it staged in shared memory).  DAG flips the projector signs.
// With LF = 1 the links are the compressed form and `cross` / `ph` give the
// boundary-crossing hops and the four boundary phases.
template <int P, bool DAG, int LF = 0>
__device__ __forceinline__ void hop_site(cx<typename Prec<P>::real> (&acc)[12], const int (&nb)[8],
                                         long long Vh, const void* in, const void* links,
                                         long long lVh, int li, unsigned cross = 0,
                                         const cx<float>* ph = nullptr)
{
    using T = typename Prec<P>::real;
    if constexpr (P == WL_DF64 && LF == 0) {
        hop_site_loop<P, DAG>(acc, nb, Vh, in, links, lVh, li);
    } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = {(T)0, (T)0};
        constexpr int F = DAG ? +1 : -1;  // forward projector sign
        constexpr int B = -F;             // backward projector sign
        hop_one<P, 0, 0, F, LF>(acc, in, Vh, nb[0], links, lVh, li, cross, ph);
        hop_one<P, 1, 0, B, LF>(acc, in, Vh, nb[1], links, lVh, li, cross, ph);
        hop_one<P, 2, 1, F, LF>(acc, in, Vh, nb[2], links, lVh, li, cross, ph);
        hop_one<P, 3, 1, B, LF>(acc, in, Vh, nb[3], links, lVh, li, cross, ph);
        hop_one<P, 4, 2, F, LF>(acc, in, Vh, nb[4], links, lVh, li, cross, ph);
        hop_one<P, 5, 2, B, LF>(acc, in, Vh, nb[5], links, lVh, li, cross, ph);
        hop_one<P, 6, 3, F, LF>(acc, in, Vh, nb[6], links, lVh, li, cross, ph);
        hop_one<P, 7, 3, B, LF>(acc, in, Vh, nb[7], links, lVh, li, cross, ph);
    }
}

struct HopArgs {
    Geom g;
    const void* links[2];
    const char* in[2];
    char* out[2];
    const char* x1[2];
    const char* x2[2];
    const char* w[2];
    const void* cl[2];  // clover matrix (A or A^-1) per launch parity, see CL below
    cx<float> ph[4];    // boundary phases (used by the compressed-link kernels)
    long long rs_in, rs_out, rs_x1, rs_x2, rs_w;
    double a, b1;
    int parity0, nparity, blocks_per_parity;
    double* dot_out;
    int dot_stride;
    const int* active;
    int active_stride;
    RedScratch red;
    // reducing single-RHS kernel: 0 = grid of resident blocks, the last block
    // adds the partials; 1 = one site per thread, every block leaves its
    // partial and a finishing launch adds them (no grid-stride loop)
    int partials_only;
};

// Clover modes of the epilogue (Eq. 2's site-diagonal A = 1 + F or its
// inverse, packed as in clover.cuh, at the output site):
//   CL = 0: out = x1 + b1 x2 + a acc
//   CL = 1: out = x1 + b1 C x2 + a acc          (A x in the Schur operator)
//   CL = 2: out = C (x1 + b1 x2 + a acc)        (A^-1 H in)
enum { kClNone = 0, kClX2 = 1, kClOut = 2 };

// (w, out) and ||out||^2 of one site into part.  The double-float kernels
// produce outer residuals: the residual itself needs the 48-bit arithmetic (a
// small difference of large terms), its norm and dots only a few digits, so
// they are summed from the high words in FP32 (~2^-24 relative, a tenth of
// the double-float cost).
template <int P>
__device__ __forceinline__ void site_dots(const cx<typename Prec<P>::real> (&acc)[12],
                                          const cx<typename Prec<P>::real>* ww,
                                          typename Prec<P>::real (&part)[3])
{
    using T = typename Prec<P>::real;
    if constexpr (P == WL_DF64) {
        float cr = 0.f, ci = 0.f, nn = 0.f;
        if (ww)
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                cr = fmaf(ww[c].re.hi, acc[c].re.hi, fmaf(ww[c].im.hi, acc[c].im.hi, cr));
                ci = fmaf(ww[c].re.hi, acc[c].im.hi, fmaf(-ww[c].im.hi, acc[c].re.hi, ci));
            }
#pragma unroll
        for (int c = 0; c < 12; ++c)
            nn = fmaf(acc[c].re.hi, acc[c].re.hi, fmaf(acc[c].im.hi, acc[c].im.hi, nn));
        part[0] = T(cr);
        part[1] = T(ci);
        part[2] = T(nn);
    } else {
        T cr = 0, ci = 0, nn = 0;
        if (ww)
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                cr = fma(ww[c].re, acc[c].re, fma(ww[c].im, acc[c].im, cr));
                ci = fma(ww[c].re, acc[c].im, fma(-ww[c].im, acc[c].re, ci));
            }
#pragma unroll
        for (int c = 0; c < 12; ++c) nn = fma(acc[c].re, acc[c].re, fma(acc[c].im, acc[c].im, nn));
        part[0] = cr;
        part[1] = ci;
        part[2] = nn;
    }
}

// out = x1 + b1 x2 + a acc at site i (x1, x2 optional; clover per CL); with
// DOT the thread's contributions to (w, out) (w optional) and ||out||^2 go to
// part.
template <int P, bool DOT, int CL = kClNone>
__device__ __forceinline__ void epilogue_ptrs(cx<typename Prec<P>::real> (&acc)[12], double a_,
                                              const char* x1, const char* x2, double b1_,
                                              const char* w, char* out, long long Vh, int i,
                                              typename Prec<P>::real (&part)[3],
                                              const void* cl = nullptr)
{
    using T = typename Prec<P>::real;
    const T a = (T)a_;
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = a * acc[c];
    // FP16 operands enter unscaled, their per-site norm folded into one FFMA
    // per value (n = 1 for the other types)
    if (x1) {
        cx<T> x[12];
        T n = (T)1;
        if constexpr (P == WL_F16) load_spinor_f16_unscaled(x, n, x1, Vh, i);
        else load_spinor<P>(x, x1, Vh, i);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            if constexpr (P == WL_F16) acc[c] = {fmaf(n, x[c].re, acc[c].re), fmaf(n, x[c].im, acc[c].im)};
            else acc[c] = acc[c] + x[c];
        }
    }
    if (x2) {
        cx<T> x[12];
        T b1 = (T)b1_;
        if constexpr (P == WL_F16) {
            float n;
            load_spinor_f16_unscaled(x, n, x2, Vh, i);
            b1 = b1 * n;  // the clover multiply below is linear
        } else {
            load_spinor<P>(x, x2, Vh, i);
        }
        if (CL == kClX2) clover_mul<P>(x, cl, Vh, i);
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = acc[c] + b1 * x[c];
    }
    if (CL == kClOut) clover_mul<P>(acc, cl, Vh, i);
    store_spinor<P>(out, Vh, i, acc);
    if (DOT) {
        if (w) {
            cx<T> ww[12];
            if constexpr (P == WL_F16) {
                float n;
                load_spinor_f16_unscaled(ww, n, w, Vh, i);
                site_dots<P>(acc, ww, part);
                part[0] *= n;
                part[1] *= n;
            } else {
                load_spinor<P>(ww, w, Vh, i);
                site_dots<P>(acc, ww, part);
            }
        } else {
            site_dots<P>(acc, nullptr, part);
        }
    }
}

template <int P, bool DOT, int CL = kClNone>
__device__ __forceinline__ void epilogue(cx<typename Prec<P>::real> (&acc)[12], const HopArgs& A,
                                         int pidx, int rhs, int i, typename Prec<P>::real (&part)[3])
{
    auto at = [&](const char* q, long long rs) -> const char* { return q ? q + rhs * rs : nullptr; };
    epilogue_ptrs<P, DOT, CL>(acc, A.a, at(A.x1[pidx], A.rs_x1), at(A.x2[pidx], A.rs_x2), A.b1,
                              at(A.w[pidx], A.rs_w), A.out[pidx] + rhs * A.rs_out, A.g.Vh, i, part,
                              A.cl[pidx]);
}

// ---------------------------------------------------------------------------
// Many right-hand sides: a block owns kTile output sites of one parity.  It
// copies their links (all eight hops) into shared memory once, then its
// warps sweep the right-hand sides, lane = site, reading the links from
// shared memory: the links leave HBM once for all right-hand sides.
// ---------------------------------------------------------------------------

static constexpr int kTile = 32;
static constexpr int kMaxRhsLaunch = 32;

// Copy the links of sites [base, base + n) into a kTile-stride tile.
template <int P, int LF = 0>
__device__ __forceinline__ void stage_links(char* sm, const char* gl, long long Vh, int base, int n)
{
    using LP = LinkLayout<P, LF>;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int e = tid; e < LP::n16 * kTile; e += nt) {
        const int q = e / kTile, j = e - q * kTile;
        if (j < n) ((uint4*)sm)[q * kTile + j] = __ldg((const uint4*)gl + q * Vh + base + j);
    }
    if (LP::nsmall) {
        const char* gs = gl + (size_t)LP::n16 * 16 * Vh;
        char* ss = sm + LP::n16 * 16 * kTile;
        for (int e = tid; e < LP::nsmall * kTile; e += nt) {
            const int q = e / kTile, j = e - q * kTile;
            if (j >= n) continue;
            if (LP::small_bytes == 8)
                ((uint2*)ss)[q * kTile + j] = __ldg((const uint2*)gs + q * Vh + base + j);
            else
                ((unsigned*)ss)[q * kTile + j] = __ldg((const unsigned*)gs + q * Vh + base + j);
        }
    }
}


// Asynchronous variant (cp.async, sm_80+): the copies of the tile are issued
// without waiting; the caller commits them as one group and waits for the
// group before reading the tile.  Lets a block fetch the next tile's links
// while it computes on the current one.
__device__ __forceinline__ void cp_async16(void* sm, const void* gl)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sm);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gl) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sm, const void* gl)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sm);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(gl) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sm, const void* gl)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sm);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gl) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int P, int LF = 0>
__device__ __forceinline__ void stage_links_async(char* sm, const char* gl, long long Vh, int base, int n)
{
    using LP = LinkLayout<P, LF>;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int e = tid; e < LP::n16 * kTile; e += nt) {
        const int q = e / kTile, j = e - q * kTile;
        if (j < n) cp_async16((uint4*)sm + q * kTile + j, (const uint4*)gl + q * Vh + base + j);
    }
    if (LP::nsmall) {
        const char* gs = gl + (size_t)LP::n16 * 16 * Vh;
        char* ss = sm + LP::n16 * 16 * kTile;
        for (int e = tid; e < LP::nsmall * kTile; e += nt) {
            const int q = e / kTile, j = e - q * kTile;
            if (j >= n) continue;
            if (LP::small_bytes == 8)
                cp_async8((uint2*)ss + q * kTile + j, (const uint2*)gs + q * Vh + base + j);
            else
                cp_async4((unsigned*)ss + q * kTile + j, (const unsigned*)gs + q * Vh + base + j);
        }
    }
}

}  // namespace wl
