// wl_cdot_noalloc: the per-right-hand-side dot products and norms of
// wl_cdot, for callers that cannot allocate device memory.
//
// Who needs it: code that runs inside another framework's memory pool and may
// not call cudaMalloc behind that allocator's back, latency-critical loops in
// which cudaMalloc/cudaFree would synchronise the device, and callers that
// hold only raw field pointers and no gauge object (wl_cdot keeps its
// reduction scratch in the gauge object's workspace, which is allocated).
//
// How: the per-block partial sums live in one file-scope __device__ array of
// fixed size, present on every GPU that loads the library until the process
// exits.  Two launches per call: every block writes its partials, then one
// block per right-hand side adds them in block order.  Every partial that is
// read was written by the same call, so nothing has to start at zero, no
// atomics are used, and the result is deterministic.  The array is shared by
// all calls: calls that overlap on the GPU (different streams, or different
// host threads on one device without ordering) race on it.
#include "internal.cuh"

namespace wl {

static constexpr int kNaBlocks = WL_NOALLOC_BLOCKS;  // reduction blocks per right-hand side
static constexpr int kNaMaxRhs = WL_NOALLOC_MAX_RHS;
static constexpr int kNaThreads = 256;

// partial[rhs][block][3]: 64 * 512 * 3 doubles = 768 KiB per device.
static __device__ __align__(256) double na_partial[kNaMaxRhs * kNaBlocks * 3];

template <int P>
__global__ void __launch_bounds__(kNaThreads) na_partial_kernel(const char* a, const char* b,
                                                                long long Vh, size_t fb,
                                                                double* partial)
{
    using T = typename Prec<P>::real;
    const int rhs = blockIdx.y;
    const char* pa = a + rhs * fb;
    const char* pb = b + rhs * fb;
    double part[3] = {0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)kNaThreads + threadIdx.x; i < Vh;
         i += (long long)gridDim.x * kNaThreads) {
        cx<T> x[12], y[12];
        load_spinor<P>(x, pa, Vh, i);
        load_spinor<P>(y, pb, Vh, i);
        T cr = 0, ci = 0, nn = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            cr = fma(x[c].re, y[c].re, fma(x[c].im, y[c].im, cr));
            ci = fma(x[c].re, y[c].im, fma(-x[c].im, y[c].re, ci));
            nn = fma(y[c].re, y[c].re, fma(y[c].im, y[c].im, nn));
        }
        part[0] += (double)cr;
        part[1] += (double)ci;
        part[2] += (double)nn;
    }
    __shared__ double sh[3 * 32];
    block_sum<3>(part, sh);
    if (threadIdx.x == 0) {
        double* o = partial + ((long long)rhs * kNaBlocks + blockIdx.x) * 3;
        o[0] = part[0];
        o[1] = part[1];
        o[2] = part[2];
    }
}

__global__ void __launch_bounds__(kNaThreads) na_finish_kernel(const double* partial, int nblocks,
                                                               double* out)
{
    const int rhs = blockIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kNaThreads)
        for (int k = 0; k < 3; ++k) v[k] += partial[((long long)rhs * kNaBlocks + b) * 3 + k];
    __shared__ double sh[3 * 32];
    block_sum<3>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out[3 * rhs + k] = v[k];
}

// Device address of na_partial in the current device's context.  The
// host-side symbol is only a stand-in for it, so the address is looked up on
// every call (a host-side query; cheap once the module is loaded): a context
// that was reset and re-created (cudaDeviceReset) gets the new address.
static int na_scratch(double** ptr)
{
    void* p = nullptr;
    WL_CUDA(cudaGetSymbolAddress(&p, na_partial));
    *ptr = (double*)p;
    return WL_OK;
}

}  // namespace wl

using namespace wl;

extern "C" int wl_cdot_noalloc(double* out, const void* a, const void* b, long long Vh,
                               wl_prec prec, int nrhs, void* stream)
{
    WL_ENTRY();
    if (!out || !a || !b) return set_error(WL_ERR_ARG, "NULL pointer");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (Vh < 1) return set_error(WL_ERR_ARG, "Vh must be >= 1");
    if (nrhs < 1 || nrhs > kNaMaxRhs)
        return set_error(WL_ERR_ARG, "nrhs must be in 1..WL_NOALLOC_MAX_RHS (64) for wl_cdot_noalloc");
    if (prec == WL_F16 && Vh % 4)  // 52 Vh bytes per field: 16-byte rows of the next field
        return set_error(WL_ERR_ARG, "FP16 fields need Vh divisible by 4");
    double* partial = nullptr;
    WL_TRY(na_scratch(&partial));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fb = spinor_field_bytes(prec, Vh);
    long long need = (Vh + kNaThreads - 1) / kNaThreads;
    const int nb = (int)(need < kNaBlocks ? need : kNaBlocks);
    const dim3 grid((unsigned)nb, (unsigned)nrhs);
    if (prec == WL_F64)
        na_partial_kernel<WL_F64><<<grid, kNaThreads, 0, s>>>((const char*)a, (const char*)b, Vh, fb, partial);
    else if (prec == WL_F32)
        na_partial_kernel<WL_F32><<<grid, kNaThreads, 0, s>>>((const char*)a, (const char*)b, Vh, fb, partial);
    else if (prec == WL_F16)
        na_partial_kernel<WL_F16><<<grid, kNaThreads, 0, s>>>((const char*)a, (const char*)b, Vh, fb, partial);
    else
        na_partial_kernel<WL_DF64><<<grid, kNaThreads, 0, s>>>((const char*)a, (const char*)b, Vh, fb, partial);
    WL_CHECK_LAUNCH(2.0 * fb * nrhs);
    na_finish_kernel<<<nrhs, kNaThreads, 0, s>>>(partial, nb, out);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}
