// Packed storage of the clover term and its site-local multiply.
//
// Sec. 2, Eq. 2: D_clov = D_W + F(x) delta_xy, where F(x) is a 12x12
// Hermitian matrix that is block diagonal with two 6x6 Hermitian blocks in
// the chiral basis; block b acts on spins {2b, 2b+1}, i.e. on the spinor
// components c = 6b .. 6b+5 (c = spin*3 + colour).  The library stores the
// site-diagonal operator A = 1 + F and its inverse, each block as 36 reals:
//   [0..5]   the real diagonal d_0 .. d_5
//   [6..35]  the strictly lower triangle L_rj (r > j) as (re, im) pairs in the
//            order (1,0), (2,0), (2,1), (3,0), ..., (5,4); the upper triangle
//            is its Hermitian conjugate.
// 72 reals per site, in structure-of-arrays planes of 16 bytes [q][Vh]:
//   F64:  36 double2 planes  (block b: planes 18b .. 18b+17)       576 B/site
//   F32:  18 float4 planes   (block b: planes  9b ..  9b+8)        288 B/site
//   DF64: 36 float4 planes   (hi, lo, hi, lo: two reals per plane) 576 B/site
//   F16:   9 uint4 planes    (8 halves per plane, unscaled)        144 B/site
// FP16 entries are stored without a norm: |A_ij| and |A^-1_ij| are O(1) for
// any usable clover term, and the set-up rejects entries outside the FP16
// range.  The FP32 layout is Table 1's 288 extra bytes per site (72 floats).
#pragma once

#include "common.cuh"

namespace wl {

static constexpr int kCloverReals = 72;

inline size_t clover_site_bytes(int prec)
{
    return prec == WL_F32 ? 288 : prec == WL_F16 ? 144 : 576;
}
inline size_t clover_field_bytes(int prec, long long Vh) { return clover_site_bytes(prec) * (size_t)Vh; }

// The 36 reals of block b at half-site i, in the arithmetic type of P.
template <int P>
__device__ __forceinline__ void load_clover_block(typename Prec<P>::real (&c)[36], const void* base,
                                                  long long Vh, long long i, int b);

template <>
__device__ __forceinline__ void load_clover_block<WL_F64>(double (&c)[36], const void* base,
                                                          long long Vh, long long i, int b)
{
    const double2* p = (const double2*)base + (long long)18 * b * Vh;
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        const double2 t = __ldg(p + q * Vh + i);
        c[2 * q] = t.x;
        c[2 * q + 1] = t.y;
    }
}

template <>
__device__ __forceinline__ void load_clover_block<WL_F32>(float (&c)[36], const void* base,
                                                          long long Vh, long long i, int b)
{
    const float4* p = (const float4*)base + (long long)9 * b * Vh;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float4 t = __ldg(p + q * Vh + i);
        c[4 * q] = t.x;
        c[4 * q + 1] = t.y;
        c[4 * q + 2] = t.z;
        c[4 * q + 3] = t.w;
    }
}

template <>
__device__ __forceinline__ void load_clover_block<WL_DF64>(df64 (&c)[36], const void* base,
                                                           long long Vh, long long i, int b)
{
    const float4* p = (const float4*)base + (long long)18 * b * Vh;
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        const float4 t = __ldg(p + q * Vh + i);
        c[2 * q] = df64(t.x, t.y);
        c[2 * q + 1] = df64(t.z, t.w);
    }
}

template <>
__device__ __forceinline__ void load_clover_block<WL_F16>(float (&c)[36], const void* base,
                                                          long long Vh, long long i, int b)
{
    // block b is halves 36b .. 36b+35: planes 4.5b .. 4.5b+4.5
    const uint4* p = (const uint4*)base;
    const int h0 = 36 * b, q0 = h0 / 8;
    unsigned w[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const uint4 t = __ldg(p + (q0 + q) * Vh + i);
        w[4 * q] = t.x;
        w[4 * q + 1] = t.y;
        w[4 * q + 2] = t.z;
        w[4 * q + 3] = t.w;
    }
    // block 0 starts at word 0 of plane 0, block 1 at word 2 of plane 4
#pragma unroll
    for (int k = 0; k < 18; ++k) {
        const float2 f = h2f(b ? w[k + 2] : w[k]);
        c[2 * k] = f.x;
        c[2 * k + 1] = f.y;
    }
}

// v <- C v for the packed Hermitian block-diagonal C at half-site i.
template <int P>
__device__ __forceinline__ void clover_mul(cx<typename Prec<P>::real> (&v)[12], const void* cl,
                                           long long Vh, long long i)
{
    using T = typename Prec<P>::real;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        T c[36];
        load_clover_block<P>(c, cl, Vh, i, b);
        cx<T> y[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) y[r] = c[r] * v[6 * b + r];
        int k = 6;
#pragma unroll
        for (int r = 1; r < 6; ++r)
#pragma unroll
            for (int j = 0; j < r; ++j) {
                const cx<T> L = {c[k], c[k + 1]};
                k += 2;
                cmac(y[r], L, v[6 * b + j]);        // lower triangle
                cmac(y[j], conj(L), v[6 * b + r]);  // its Hermitian conjugate above
            }
#pragma unroll
        for (int r = 0; r < 6; ++r) v[6 * b + r] = y[r];
    }
}

}  // namespace wl
