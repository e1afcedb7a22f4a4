// BLAS-1 kernels and global reductions over internal fields (the "BLAS-like
// functions" of the BiCGStab solver, Sec. 5.3): complex dots and norms with
// FP64 accumulation above the thread level, precision conversion, zeroing
// and FP64 accumulation of a lower-precision correction.
//
// A vector is `nhalf` half fields per right-hand side stored back to back
// (nhalf = 1 for even-odd vectors, 2 for full-lattice ones); element j (one
// site) lives in half j / Vh at index j % Vh.  Each kernel
// runs one thread per site and right-hand side (grid.y = rhs).
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "internal.cuh"

namespace wl {

int resident_grid(const void* kernel, int block, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, long long>, int> cache;
    const auto key = std::make_pair(kernel, (long long)block * (1LL << 32) + (long long)smem);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0, dev = 0, sms = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess)
        per_sm = 1;
    cudaGetLastError();
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (per_sm > 0 ? per_sm : 1) * sms;
    cache[key] = grid;
    return grid;
}

__global__ void __launch_bounds__(256) finish_slots_kernel(const double* partial, long long stride,
                                                           int nblocks, double* out, int out_stride,
                                                           const int* active, int active_stride)
{
    const int slot = blockIdx.x;
    if (active && !active[(long long)slot * active_stride]) return;
    __shared__ double sh[3 * 32];
    double v[3];
    sum_partials<3>(partial + slot * stride, nblocks, v);
    block_sum<3>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[(long long)slot * out_stride + k] = v[k];
}

int launch_finish_slots(const double* partial, long long stride, int nblocks, int nslots,
                        double* out, int out_stride, const int* active, int active_stride,
                        cudaStream_t s)
{
    finish_slots_kernel<<<nslots, 256, 0, s>>>(partial, stride, nblocks, out, out_stride, active,
                                                active_stride);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

struct Vec {
    long long Vh;
    int nhalf;
    size_t hb;         // bytes of one half field
    long long rstride; // bytes between right-hand sides
};

__device__ __forceinline__ const char* at(const void* base, const Vec& v, int rhs, long long j,
                                          long long& i)
{
    const int h = j >= v.Vh ? 1 : 0;  // nhalf <= 2: a comparison, not a 64-bit division
    i = j - h * v.Vh;
    return (const char*)base + rhs * v.rstride + h * v.hb;
}

// (a, b) and ||b||^2 per right-hand side.  NORM: a is b, and only the norm
// is formed ((b, b) is that norm, with a zero imaginary part); for the FP64
// fields that is a third of the FP64 arithmetic.
template <int P, bool NORM>
__global__ void __launch_bounds__(256) cdot_kernel(const void* a, const void* b, Vec v, double* out,
                                                   int out_stride, const int* mask, RedScratch red)
{
    using T = typename Prec<P>::real;
    const int rhs = blockIdx.y;
    if (mask && !mask[rhs]) return;
    double part[3] = {0, 0, 0};  // per-site FP64 accumulation (off the hot path)
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < v.nhalf * v.Vh;
         j += (long long)gridDim.x * blockDim.x) {
        long long i;
        cx<T> x[12], y[12];
        load_spinor<P>(y, at(b, v, rhs, j, i), v.Vh, i);
        T cr = 0, ci = 0, nn = 0;
        if (NORM) {
#pragma unroll
            for (int c = 0; c < 12; ++c) nn = fma(y[c].re, y[c].re, fma(y[c].im, y[c].im, nn));
            cr = nn;
        } else {
            load_spinor<P>(x, at(a, v, rhs, j, i), v.Vh, i);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                cr = fma(x[c].re, y[c].re, fma(x[c].im, y[c].im, cr));
                ci = fma(x[c].re, y[c].im, fma(-x[c].im, y[c].re, ci));
                nn = fma(y[c].re, y[c].re, fma(y[c].im, y[c].im, nn));
            }
        }
        part[0] += (double)cr;
        part[1] += (double)ci;
        part[2] += (double)nn;
    }
    __shared__ double sh[3 * 32];
    block_sum<3>(part, sh);
    double tot[3];
    if (grid_sum<3>(part, tot, red, rhs, gridDim.x, blockIdx.x, sh)) {
        double* o = out + (long long)rhs * out_stride;
        o[0] = tot[0];
        o[1] = tot[1];
        o[2] = tot[2];
    }
}

template <int PD, int PS>
__global__ void convert_kernel(void* dst, Vec vd, const void* src, Vec vs, const int* mask)
{
    const int rhs = blockIdx.y;
    if (mask && !mask[rhs]) return;
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= vd.nhalf * vd.Vh) return;
    long long i;
    cx<typename Prec<PS>::real> x[12];
    load_spinor<PS>(x, at(src, vs, rhs, j, i), vs.Vh, i);
    cx<typename Prec<PD>::real> y[12];
#pragma unroll
    for (int c = 0; c < 12; ++c)
        y[c] = {(typename Prec<PD>::real)x[c].re, (typename Prec<PD>::real)x[c].im};
    store_spinor<PD>((void*)at(dst, vd, rhs, j, i), vd.Vh, i, y);
}

template <int P>
__global__ void zero_kernel(void* dst, Vec v, const int* mask)
{
    const int rhs = blockIdx.y;
    if (mask && !mask[rhs]) return;
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= v.nhalf * v.Vh) return;
    long long i;
    cx<typename Prec<P>::real> y[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) y[c] = {0, 0};
    store_spinor<P>((void*)at(dst, v, rhs, j, i), v.Vh, i, y);
}

// x_hi (FP64 or df64) += x_lo
template <int PH, int PL>
__global__ void accum_hi_kernel(void* xhi, Vec vh, const void* xlo, Vec vl, const int* mask)
{
    using TH = typename Prec<PH>::real;
    const int rhs = blockIdx.y;
    if (mask && !mask[rhs]) return;
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= vh.nhalf * vh.Vh) return;
    long long i;
    cx<typename Prec<PL>::real> x[12];
    load_spinor<PL>(x, at(xlo, vl, rhs, j, i), vl.Vh, i);
    cx<TH> y[12];
    char* ph = (char*)at(xhi, vh, rhs, j, i);
    load_spinor<PH>(y, ph, vh.Vh, i);
#pragma unroll
    for (int c = 0; c < 12; ++c) y[c] = {y[c].re + (TH)x[c].re, y[c].im + (TH)x[c].im};
    store_spinor<PH>(ph, vh.Vh, i, y);
}

static Vec make_vec(wl_gauge g, int prec, int nhalf, long long rs = 0)  // nhalf is 1 or 2
{
    Vec v;
    v.Vh = g->geo.Vh;
    v.nhalf = nhalf;
    v.hb = spinor_field_bytes(prec, g->geo.Vh);
    v.rstride = rs ? rs : (long long)(v.hb * nhalf);
    return v;
}

static const int kBlasBlock = 256;

static dim3 blas_grid(wl_gauge g, int nhalf, int nrhs)
{
    return dim3((unsigned)((nhalf * g->geo.Vh + kBlasBlock - 1) / kBlasBlock), (unsigned)nrhs);
}

int launch_cdot(wl_gauge g, int prec, const void* a, const void* b, int nhalf, int nrhs,
                double* out, int out_stride, const int* mask, cudaStream_t s, long long rs)
{
    dim3 grid = blas_grid(g, nhalf, nrhs);
    const bool norm = a == b;
    const void* kern = prec == WL_F64 ? (const void*)cdot_kernel<WL_F64, false>
                       : prec == WL_F32 ? (const void*)cdot_kernel<WL_F32, false>
                       : prec == WL_F16 ? (const void*)cdot_kernel<WL_F16, false>
                                        : (const void*)cdot_kernel<WL_DF64, false>;
    grid.x = std::min(grid.x, (unsigned)resident_grid(kern, kBlasBlock, 0));
    WL_TRY(ensure_red(g, nrhs, grid.x));
    const Vec v = make_vec(g, prec, nhalf, rs);
    auto go = [&](auto nt) {
        constexpr bool N = decltype(nt)::value;
        if (prec == WL_F64) cdot_kernel<WL_F64, N><<<grid, kBlasBlock, 0, s>>>(a, b, v, out, out_stride, mask, g->red);
        else if (prec == WL_F32) cdot_kernel<WL_F32, N><<<grid, kBlasBlock, 0, s>>>(a, b, v, out, out_stride, mask, g->red);
        else if (prec == WL_F16) cdot_kernel<WL_F16, N><<<grid, kBlasBlock, 0, s>>>(a, b, v, out, out_stride, mask, g->red);
        else cdot_kernel<WL_DF64, N><<<grid, kBlasBlock, 0, s>>>(a, b, v, out, out_stride, mask, g->red);
    };
    if (norm) go(std::true_type{});
    else go(std::false_type{});
    WL_CHECK_LAUNCH((norm ? 1.0 : 2.0) * v.hb * nhalf * nrhs);
    return WL_OK;
}

template <int PD>
static void convert_from(int psrc, void* dst, Vec vd, const void* src, Vec vs, dim3 grid,
                         const int* mask, cudaStream_t s)
{
    if (psrc == WL_F64) convert_kernel<PD, WL_F64><<<grid, kBlasBlock, 0, s>>>(dst, vd, src, vs, mask);
    else if (psrc == WL_F32) convert_kernel<PD, WL_F32><<<grid, kBlasBlock, 0, s>>>(dst, vd, src, vs, mask);
    else if (psrc == WL_F16) convert_kernel<PD, WL_F16><<<grid, kBlasBlock, 0, s>>>(dst, vd, src, vs, mask);
    else convert_kernel<PD, WL_DF64><<<grid, kBlasBlock, 0, s>>>(dst, vd, src, vs, mask);
}

int launch_convert(wl_gauge g, int pdst, void* dst, int psrc, const void* src, int nhalf, int nrhs,
                   const int* mask, cudaStream_t s, long long dst_rs, long long src_rs)
{
    const dim3 grid = blas_grid(g, nhalf, nrhs);
    const Vec vd = make_vec(g, pdst, nhalf, dst_rs), vs = make_vec(g, psrc, nhalf, src_rs);
    if (pdst == WL_F64) convert_from<WL_F64>(psrc, dst, vd, src, vs, grid, mask, s);
    else if (pdst == WL_F32) convert_from<WL_F32>(psrc, dst, vd, src, vs, grid, mask, s);
    else if (pdst == WL_F16) convert_from<WL_F16>(psrc, dst, vd, src, vs, grid, mask, s);
    else convert_from<WL_DF64>(psrc, dst, vd, src, vs, grid, mask, s);
    WL_CHECK_LAUNCH((double)(vd.hb + vs.hb) * nhalf * nrhs);
    return WL_OK;
}

int launch_zero(wl_gauge g, int prec, void* dst, int nhalf, int nrhs, const int* mask,
                cudaStream_t s)
{
    const dim3 grid = blas_grid(g, nhalf, nrhs);
    const Vec v = make_vec(g, prec, nhalf);
    if (prec == WL_F64) zero_kernel<WL_F64><<<grid, kBlasBlock, 0, s>>>(dst, v, mask);
    else if (prec == WL_F32) zero_kernel<WL_F32><<<grid, kBlasBlock, 0, s>>>(dst, v, mask);
    else if (prec == WL_F16) zero_kernel<WL_F16><<<grid, kBlasBlock, 0, s>>>(dst, v, mask);
    else zero_kernel<WL_DF64><<<grid, kBlasBlock, 0, s>>>(dst, v, mask);
    WL_CHECK_LAUNCH((double)v.hb * nhalf * nrhs);
    return WL_OK;
}

template <int PH>
static void accum_from(int plo, void* xhi, Vec vh, const void* xlo, Vec vl, dim3 grid,
                       const int* mask, cudaStream_t s)
{
    if (plo == WL_F64) accum_hi_kernel<PH, WL_F64><<<grid, kBlasBlock, 0, s>>>(xhi, vh, xlo, vl, mask);
    else if (plo == WL_F32) accum_hi_kernel<PH, WL_F32><<<grid, kBlasBlock, 0, s>>>(xhi, vh, xlo, vl, mask);
    else accum_hi_kernel<PH, WL_F16><<<grid, kBlasBlock, 0, s>>>(xhi, vh, xlo, vl, mask);
}

int launch_accum_hi(wl_gauge g, int phi, void* xhi, int plo, const void* xlo, int nhalf, int nrhs,
                    const int* mask, cudaStream_t s, long long hi_rs)
{
    const dim3 grid = blas_grid(g, nhalf, nrhs);
    const Vec vh = make_vec(g, phi, nhalf, hi_rs), vl = make_vec(g, plo, nhalf);
    if (phi == WL_DF64) accum_from<WL_DF64>(plo, xhi, vh, xlo, vl, grid, mask, s);
    else accum_from<WL_F64>(plo, xhi, vh, xlo, vl, grid, mask, s);
    WL_CHECK_LAUNCH((double)(2 * vh.hb + vl.hb) * nhalf * nrhs);
    return WL_OK;
}

}  // namespace wl

using namespace wl;

extern "C" int wl_cdot(wl_gauge g, double* out, const void* a, const void* b, wl_prec prec, int nrhs,
                       void* stream)
{
    WL_ENTRY();
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (!out || !a || !b) return set_error(WL_ERR_ARG, "NULL pointer");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    return launch_cdot(g, prec, a, b, 1, nrhs, out, 3, nullptr, (cudaStream_t)stream);
}
