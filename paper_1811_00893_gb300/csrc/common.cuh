// Device-side building blocks shared by every kernel of the library:
// complex arithmetic, the structure-of-arrays field layouts per storage
// precision, block/grid reductions and host-side error plumbing.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "df64.cuh"
#include "wilson.h"

// ---------------------------------------------------------------------------
// host-side errors and launch accounting
// ---------------------------------------------------------------------------

namespace wl {

int set_error(int code, const std::string& msg);
extern std::atomic<long long> g_launches;
extern std::atomic<long long> g_bytes;  // algorithmic bytes of every launched kernel

inline void count_launch(long long n = 1, double bytes = 0.0)
{
    g_launches.fetch_add(n, std::memory_order_relaxed);
    g_bytes.fetch_add((long long)bytes, std::memory_order_relaxed);
}

}  // namespace wl

// A failed runtime call is reported and its (non-sticky) error consumed, so it
// cannot resurface in a later launch check.
#define WL_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            cudaGetLastError();                                                           \
            return wl::set_error(WL_ERR_CUDA, std::string(#call) + ": " +                 \
                                                  cudaGetErrorString(e_));                \
        }                                                                                 \
    } while (0)

// Entry points start from a clean error state: an earlier failure elsewhere in
// the process must not be reported as this call's launch error.
#define WL_ENTRY() cudaGetLastError()

// Check a kernel launch and account for it with its algorithmic bytes.
#define WL_CHECK_LAUNCH(bytes)                                                            \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return wl::set_error(WL_ERR_CUDA, std::string("kernel launch: ") +            \
                                                  cudaGetErrorString(e_));                \
        wl::count_launch(1, (bytes));                                                     \
    } while (0)

#define WL_TRY(expr)             \
    do {                         \
        int rc_ = (expr);        \
        if (rc_ != WL_OK) return rc_; \
    } while (0)

namespace wl {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------

template <typename T>
struct cx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T r, T i) { return {r, i}; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a) { return {-a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.re, -a.im}; }
// i * a
template <typename T>
__device__ __forceinline__ cx<T> mul_i(cx<T> a) { return {-a.im, a.re}; }
// acc += a * b
template <typename T>
__device__ __forceinline__ void cmac(cx<T>& acc, cx<T> a, cx<T> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}

// ---------------------------------------------------------------------------
// storage layouts (one half-lattice field = one parity, one right-hand side)
//
//   F64 spinor: 12 double2 planes    [c][Vh]         c = spin*3 + colour
//   F32 spinor:  6 float4 planes     [k][Vh]         float4 k holds c = 2k, 2k+1
//   F16 spinor:  3 uint4 planes      [k][Vh]         uint4 k holds c = 4k..4k+3 (half2)
//                + float norm[Vh]                    value = half * norm
//   Link field for output parity p: for each of the 8 hops d = 2*mu (+mu) and
//   d = 2*mu+1 (-mu) the 3x3 matrix W_d(x) applied to the neighbour spinor,
//   with the backward link already daggered and the boundary phase folded in:
//   F64: [d][9][Vh] double2; F32: [d][4][Vh] float4 + [d][Vh] float2;
//   F16: [d][2][Vh] uint4 + [d][Vh] half2.  Entry order a*3 + b (row, col).
// ---------------------------------------------------------------------------

template <int P>
struct Prec;

template <>
struct Prec<WL_F64> {
    using real = double;
    static constexpr size_t spinor_bytes = 192;  // per site
    static constexpr size_t link_bytes = 8 * 9 * 16;
};
template <>
struct Prec<WL_F32> {
    using real = float;
    static constexpr size_t spinor_bytes = 96;
    static constexpr size_t link_bytes = 8 * (64 + 8);
};
template <>
struct Prec<WL_F16> {
    using real = float;  // arithmetic precision of the FP16-storage path
    static constexpr size_t spinor_bytes = 52;
    static constexpr size_t link_bytes = 8 * (32 + 4);
};
template <>
struct Prec<WL_DF64> {
    using real = df64;
    static constexpr size_t spinor_bytes = 192;
    static constexpr size_t link_bytes = 8 * 9 * 16;
};

inline size_t spinor_field_bytes(int prec, long long Vh)
{
    return (prec == WL_F64 || prec == WL_DF64 ? 192 : prec == WL_F32 ? 96 : 52) * (size_t)Vh;
}
inline size_t link_field_bytes(int prec, long long Vh)
{
    return (prec == WL_F64 || prec == WL_DF64 ? 8 * 9 * 16 : prec == WL_F32 ? 8 * 72 : 8 * 36) *
           (size_t)Vh;
}

// --- spinor loads/stores --------------------------------------------------

template <int P>
__device__ __forceinline__ void load_spinor(cx<typename Prec<P>::real> (&v)[12], const void* base,
                                            long long Vh, long long i);
template <int P>
__device__ __forceinline__ void store_spinor(void* base, long long Vh, long long i,
                                             const cx<typename Prec<P>::real> (&v)[12]);

template <>
__device__ __forceinline__ void load_spinor<WL_F64>(cx<double> (&v)[12], const void* base,
                                                    long long Vh, long long i)
{
    const double2* p = (const double2*)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 t = p[c * Vh + i];
        v[c] = {t.x, t.y};
    }
}
template <>
__device__ __forceinline__ void store_spinor<WL_F64>(void* base, long long Vh, long long i,
                                                     const cx<double> (&v)[12])
{
    double2* p = (double2*)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c * Vh + i] = make_double2(v[c].re, v[c].im);
}

template <>
__device__ __forceinline__ void load_spinor<WL_F32>(cx<float> (&v)[12], const void* base,
                                                    long long Vh, long long i)
{
    const float4* p = (const float4*)base;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 t = p[k * Vh + i];
        v[2 * k] = {t.x, t.y};
        v[2 * k + 1] = {t.z, t.w};
    }
}
template <>
__device__ __forceinline__ void store_spinor<WL_F32>(void* base, long long Vh, long long i,
                                                     const cx<float> (&v)[12])
{
    float4* p = (float4*)base;
#pragma unroll
    for (int k = 0; k < 6; ++k)
        p[k * Vh + i] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
}

template <>
__device__ __forceinline__ void load_spinor<WL_DF64>(cx<df64> (&v)[12], const void* base,
                                                     long long Vh, long long i)
{
    const float4* p = (const float4*)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        float4 t = p[c * Vh + i];
        v[c] = {df64(t.x, t.y), df64(t.z, t.w)};
    }
}
template <>
__device__ __forceinline__ void store_spinor<WL_DF64>(void* base, long long Vh, long long i,
                                                      const cx<df64> (&v)[12])
{
    float4* p = (float4*)base;
#pragma unroll
    for (int c = 0; c < 12; ++c)
        p[c * Vh + i] = make_float4(v[c].re.hi, v[c].re.lo, v[c].im.hi, v[c].im.lo);
}

__device__ __forceinline__ float2 h2f(unsigned u)
{
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ unsigned f2h(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned*>(&h);
}

// Codec of the 16-bit spinor words (two values per word, real part in the
// low half), applied to the value divided by the site's max |component|, so
// that it lies in [-1, 1].  Default: IEEE binary16 (2^-11 relative
// rounding).  WL_SPINOR16_FIXED=1 builds int16 fixed point instead: the value
// times 32767, rounded to nearest, which is 2^-16 of the site scale absolute.
// It is stored biased by 32768 so that decoding is a byte permute into the
// mantissa of 2^23 and one subtraction, both exact.  kSpin16Unit is the value
// of one decoded unit; the kernels fold it into the site norm.
#ifndef WL_SPINOR16_FIXED
#define WL_SPINOR16_FIXED 0
#endif
constexpr float kSpin16Unit = WL_SPINOR16_FIXED ? 1.0f / 32767.0f : 1.0f;
__device__ __forceinline__ float2 s16_dec(unsigned u)
{
#if WL_SPINOR16_FIXED
    const float bias = 8421376.0f;  // 2^23 + 32768
    return make_float2(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7610)) - bias,
                       __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7632)) - bias);
#else
    return h2f(u);
#endif
}
__device__ __forceinline__ unsigned s16_enc(float a, float b)
{
#if WL_SPINOR16_FIXED
    const int qa = min(32767, max(-32767, __float2int_rn(a * 32767.0f)));
    const int qb = min(32767, max(-32767, __float2int_rn(b * 32767.0f)));
    return (unsigned)(qa + 32768) | ((unsigned)(qb + 32768) << 16);
#else
    return f2h(a, b);
#endif
}

template <>
__device__ __forceinline__ void load_spinor<WL_F16>(cx<float> (&v)[12], const void* base,
                                                    long long Vh, long long i)
{
    const uint4* p = (const uint4*)base;
    const float nrm = ((const float*)(p + 3 * Vh))[i] * kSpin16Unit;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 t = p[k * Vh + i];
        float2 a = s16_dec(t.x), b = s16_dec(t.y), c = s16_dec(t.z), d = s16_dec(t.w);
        v[4 * k + 0] = {a.x * nrm, a.y * nrm};
        v[4 * k + 1] = {b.x * nrm, b.y * nrm};
        v[4 * k + 2] = {c.x * nrm, c.y * nrm};
        v[4 * k + 3] = {d.x * nrm, d.y * nrm};
    }
}
template <>
__device__ __forceinline__ void store_spinor<WL_F16>(void* base, long long Vh, long long i,
                                                     const cx<float> (&v)[12])
{
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(v[c].re), fabsf(v[c].im)));
    const float s = m > 0.f ? 1.f / m : 0.f;
    uint4* p = (uint4*)base;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 t;
        t.x = s16_enc(v[4 * k + 0].re * s, v[4 * k + 0].im * s);
        t.y = s16_enc(v[4 * k + 1].re * s, v[4 * k + 1].im * s);
        t.z = s16_enc(v[4 * k + 2].re * s, v[4 * k + 2].im * s);
        t.w = s16_enc(v[4 * k + 3].re * s, v[4 * k + 3].im * s);
        p[k * Vh + i] = t;
    }
    ((float*)(p + 3 * Vh))[i] = m;
}

// Read-only variants for fields that no thread of the launch writes (the
// hopping kernels' neighbour spinors): loads go through the non-coherent
// read-only path, whose caching serves the stencil's neighbour reuse.
template <int P>
__device__ __forceinline__ void load_spinor_ro(cx<typename Prec<P>::real> (&v)[12],
                                               const void* base, long long Vh, long long i);

template <>
__device__ __forceinline__ void load_spinor_ro<WL_F64>(cx<double> (&v)[12], const void* base,
                                                       long long Vh, long long i)
{
    const double2* p = (const double2*)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 t = __ldg(p + c * Vh + i);
        v[c] = {t.x, t.y};
    }
}
template <>
__device__ __forceinline__ void load_spinor_ro<WL_F32>(cx<float> (&v)[12], const void* base,
                                                       long long Vh, long long i)
{
    const float4* p = (const float4*)base;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 t = __ldg(p + k * Vh + i);
        v[2 * k] = {t.x, t.y};
        v[2 * k + 1] = {t.z, t.w};
    }
}
template <>
__device__ __forceinline__ void load_spinor_ro<WL_F16>(cx<float> (&v)[12], const void* base,
                                                       long long Vh, long long i)
{
    const uint4* p = (const uint4*)base;
    const float nrm = __ldg((const float*)(p + 3 * Vh) + i) * kSpin16Unit;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 t = __ldg(p + k * Vh + i);
        float2 a = s16_dec(t.x), b = s16_dec(t.y), c = s16_dec(t.z), d = s16_dec(t.w);
        v[4 * k + 0] = {a.x * nrm, a.y * nrm};
        v[4 * k + 1] = {b.x * nrm, b.y * nrm};
        v[4 * k + 2] = {c.x * nrm, c.y * nrm};
        v[4 * k + 3] = {d.x * nrm, d.y * nrm};
    }
}

template <>
__device__ __forceinline__ void load_spinor_ro<WL_DF64>(cx<df64> (&v)[12], const void* base,
                                                        long long Vh, long long i)
{
    const float4* p = (const float4*)base;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        float4 t = __ldg(p + c * Vh + i);
        v[c] = {df64(t.x, t.y), df64(t.z, t.w)};
    }
}

// --- link loads -----------------------------------------------------------

template <int P>
__device__ __forceinline__ void load_link(cx<typename Prec<P>::real> (&w)[9], const void* base,
                                          long long Vh, int d, long long i);

template <>
__device__ __forceinline__ void load_link<WL_F64>(cx<double> (&w)[9], const void* base,
                                                  long long Vh, int d, long long i)
{
    const double2* p = (const double2*)base + (long long)d * 9 * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 t = p[k * Vh + i];
        w[k] = {t.x, t.y};
    }
}
template <>
__device__ __forceinline__ void load_link<WL_F32>(cx<float> (&w)[9], const void* base,
                                                  long long Vh, int d, long long i)
{
    const float4* p = (const float4*)base + (long long)d * 4 * Vh;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 t = p[k * Vh + i];
        w[2 * k] = {t.x, t.y};
        w[2 * k + 1] = {t.z, t.w};
    }
    const float2* q = (const float2*)((const float4*)base + 8 * 4 * Vh) + (long long)d * Vh;
    float2 t = q[i];
    w[8] = {t.x, t.y};
}
template <>
__device__ __forceinline__ void load_link<WL_DF64>(cx<df64> (&w)[9], const void* base,
                                                   long long Vh, int d, long long i)
{
    const float4* p = (const float4*)base + (long long)d * 9 * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float4 t = p[k * Vh + i];
        w[k] = {df64(t.x, t.y), df64(t.z, t.w)};
    }
}
template <>
__device__ __forceinline__ void load_link<WL_F16>(cx<float> (&w)[9], const void* base,
                                                  long long Vh, int d, long long i)
{
    const uint4* p = (const uint4*)base + (long long)d * 2 * Vh;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint4 t = p[k * Vh + i];
        float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), e = h2f(t.w);
        w[4 * k + 0] = {a.x, a.y};
        w[4 * k + 1] = {b.x, b.y};
        w[4 * k + 2] = {c.x, c.y};
        w[4 * k + 3] = {e.x, e.y};
    }
    const unsigned* q = (const unsigned*)((const uint4*)base + 8 * 2 * Vh) + (long long)d * Vh;
    float2 t = h2f(q[i]);
    w[8] = {t.x, t.y};
}

// ---------------------------------------------------------------------------
// reductions: warp shuffle -> shared memory -> per-block partial in FP64 ->
// the last block to finish (atomic ticket) sums the partials in a fixed
// order, so results do not depend on block scheduling.
// ---------------------------------------------------------------------------

// Type in which per-warp partial sums are shuffled: FP32 for FP32 arithmetic,
// FP64 for the wider types.
template <typename T>
struct RedType {
    using type = double;
};
template <>
struct RedType<float> {
    using type = float;
};

template <int N, typename T>
__device__ __forceinline__ void warp_sum(T (&v)[N])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// Sum v over the block; the total is valid in thread 0.  `sh` holds
// N * 32 doubles.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* sh)
{
    warp_sum<N>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k * 32 + w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = lane < nw ? sh[k * 32 + lane] : 0.0;
        warp_sum<N>(v);
    }
}

// Block sum of per-warp totals already formed in a narrower type: lane 0 of
// every warp holds its warp's total in v; the result is valid in thread 0.
// (The kernels sum their sites in the arithmetic type, then go to FP64 at
// the warp level: GB300 runs FP64 at 1/64 of the FP32 rate.)
template <int N>
__device__ __forceinline__ void block_sum_warps(double (&v)[N], double* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k * 32 + w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = lane < nw ? sh[k * 32 + lane] : 0.0;
        warp_sum<N>(v);
    }
}

// This thread's share of the sum of nblocks partial N-tuples (stride N),
// four independent loads in flight so the loop is not one L2 latency per step.
template <int N>
__device__ __forceinline__ void sum_partials(const double* part, int nblocks, double (&v)[N],
                                             long long tstride = N)
{
    double a[4][N];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < N; ++k) a[u][k] = 0.0;
    const int step = blockDim.x;
    int b = threadIdx.x;
    for (; b + 3 * step < nblocks; b += 4 * step)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < N; ++k) a[u][k] += __ldcg(&part[(long long)(b + u * step) * tstride + k]);
    for (; b < nblocks; b += step)
#pragma unroll
        for (int k = 0; k < N; ++k) a[0][k] += __ldcg(&part[(long long)b * tstride + k]);
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = (a[0][k] + a[1][k]) + (a[2][k] + a[3][k]);
}

// Scratch for grid reductions: partial[slot][block][N] and one ticket per slot.
struct RedScratch {
    double* partial;
    unsigned* ticket;
    int max_blocks;
};

// Finish a grid reduction of N values for `slot` (one slot per right-hand
// side).  Every block calls this with its block total in thread 0.  Returns
// true in thread 0 of the last block, with the grid total in `tot`.
template <int N>
__device__ __forceinline__ bool grid_sum(const double (&blk)[N], double (&tot)[N], RedScratch rs,
                                         int slot, int nblocks, int block, double* sh)
{
    __shared__ bool last;
    double* part = rs.partial + ((long long)slot * rs.max_blocks) * N;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) part[(long long)block * N + k] = blk[k];
        __threadfence();
        unsigned t = atomicAdd(&rs.ticket[slot], 1u);
        last = (t == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double v[N];
    sum_partials<N>(part, nblocks, v);
    block_sum<N>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) tot[k] = v[k];
        rs.ticket[slot] = 0;  // ready for the next launch
    }
    return threadIdx.x == 0;
}

}  // namespace wl
