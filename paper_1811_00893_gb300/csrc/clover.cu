// Clover term (Sec. 2, Eq. 2): set-up of A = 1 + F and A^-1 per parity, and
// the site-diagonal multiply wl_clover_apply.
//
// The paper leaves the construction of F(x) out of its cost model; here F is
// an input field.  Set-up runs once per clover field: one thread per site and
// 6x6 block reads the block in FP64, checks that it is Hermitian, forms
// A = 1 + F, inverts it by Gauss-Jordan elimination with partial pivoting in
// FP64 (A^-1 of a Hermitian A is Hermitian, so its lower triangle and real
// diagonal are kept) and packs both into every precision the gauge object
// holds (layout in clover.cuh).  The hopping kernels apply A or A^-1 in their
// epilogue; wl_clover_apply is the stand-alone multiply.
#include <cmath>

#include "clover.cuh"
#include "internal.cuh"

namespace wl {

enum : int { kClovNotHermitian = 1, kClovSingular = 2, kClovF16Range = 4 };

template <int P>
__device__ __forceinline__ void store_clover_block(void* base, long long Vh, long long i, int b,
                                                   const double (&c)[36]);

template <>
__device__ __forceinline__ void store_clover_block<WL_F64>(void* base, long long Vh, long long i, int b,
                                                           const double (&c)[36])
{
    double2* p = (double2*)base + (long long)18 * b * Vh;
    for (int q = 0; q < 18; ++q) p[q * Vh + i] = make_double2(c[2 * q], c[2 * q + 1]);
}

template <>
__device__ __forceinline__ void store_clover_block<WL_F32>(void* base, long long Vh, long long i, int b,
                                                           const double (&c)[36])
{
    float4* p = (float4*)base + (long long)9 * b * Vh;
    for (int q = 0; q < 9; ++q)
        p[q * Vh + i] = make_float4((float)c[4 * q], (float)c[4 * q + 1], (float)c[4 * q + 2],
                                    (float)c[4 * q + 3]);
}

template <>
__device__ __forceinline__ void store_clover_block<WL_DF64>(void* base, long long Vh, long long i, int b,
                                                            const double (&c)[36])
{
    float4* p = (float4*)base + (long long)18 * b * Vh;
    for (int q = 0; q < 18; ++q) {
        const df64 a(c[2 * q]), d(c[2 * q + 1]);
        p[q * Vh + i] = make_float4(a.hi, a.lo, d.hi, d.lo);
    }
}

// FP16: block b occupies halves 36b .. 36b+35 of the site's 72; the two
// blocks share plane 4, so each thread writes its own 32-bit words.
template <>
__device__ __forceinline__ void store_clover_block<WL_F16>(void* base, long long Vh, long long i, int b,
                                                           const double (&c)[36])
{
    unsigned* p = (unsigned*)base;  // word w of plane q at (q * Vh + i) * 4 + w
    for (int k = 0; k < 18; ++k) {
        const int word = 18 * b + k;  // half2 word index within the site
        const int q = word / 4, w = word - 4 * q;
        p[(q * Vh + i) * 4 + w] = f2h((float)c[2 * k], (float)c[2 * k + 1]);
    }
}

struct CloverTargets {
    void* A[4];
    void* Ainv[4];
};

// One thread per (half site, block) of parity p.  F: canonical FP64
// [V][2][6][6] complex.
__global__ void build_clover_kernel(const double* __restrict__ F, Geom g, int p, CloverTargets t,
                                    int* flag)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= 2 * g.Vh) return;
    const long long i = idx >> 1;
    const int b = (int)(idx & 1);
    const long long s = site_of_half(g, p, i);
    const double* m = F + (s * 2 + b) * 72;  // 6x6 complex, row-major
    // Hermiticity: |M_rj - conj(M_jr)| against the largest entry
    double big = 0.0, dev = 0.0;
    for (int r = 0; r < 6; ++r)
        for (int j = 0; j < 6; ++j) {
            const double re = m[2 * (6 * r + j)], im = m[2 * (6 * r + j) + 1];
            const double tre = m[2 * (6 * j + r)], tim = m[2 * (6 * j + r) + 1];
            big = fmax(big, fmax(fabs(re), fabs(im)));
            dev = fmax(dev, fmax(fabs(re - tre), fabs(im + tim)));
        }
    int bad = 0;
    if (!(dev <= 1e-10 * fmax(big, 1e-300)) && big > 0.0) bad |= kClovNotHermitian;
    // A = 1 + F from the lower triangle and the real diagonal, as an
    // augmented [A | I] for Gauss-Jordan elimination
    double a[6][12][2];
    for (int r = 0; r < 6; ++r)
        for (int j = 0; j < 12; ++j) a[r][j][0] = a[r][j][1] = 0.0;
    for (int r = 0; r < 6; ++r) {
        a[r][r][0] = 1.0 + m[2 * (6 * r + r)];
        a[r][6 + r][0] = 1.0;
        for (int j = 0; j < r; ++j) {
            a[r][j][0] = m[2 * (6 * r + j)];
            a[r][j][1] = m[2 * (6 * r + j) + 1];
            a[j][r][0] = a[r][j][0];
            a[j][r][1] = -a[r][j][1];
        }
    }
    double c[36];
    for (int r = 0; r < 6; ++r) c[r] = a[r][r][0];
    {
        int k = 6;
        for (int r = 1; r < 6; ++r)
            for (int j = 0; j < r; ++j) {
                c[k++] = a[r][j][0];
                c[k++] = a[r][j][1];
            }
    }
    double anorm = 0.0;
    for (int r = 0; r < 6; ++r)
        for (int j = 0; j < 6; ++j) anorm = fmax(anorm, hypot(a[r][j][0], a[r][j][1]));
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        double best = hypot(a[col][col][0], a[col][col][1]);
        for (int r = col + 1; r < 6; ++r) {
            const double v = hypot(a[r][col][0], a[r][col][1]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > 1e-13 * anorm)) {
            bad |= kClovSingular;
            break;
        }
        if (piv != col)
            for (int j = 0; j < 12; ++j)
                for (int z = 0; z < 2; ++z) {
                    const double tmp = a[col][j][z];
                    a[col][j][z] = a[piv][j][z];
                    a[piv][j][z] = tmp;
                }
        // scale the pivot row by 1 / a_cc
        const double den = a[col][col][0] * a[col][col][0] + a[col][col][1] * a[col][col][1];
        const double ir = a[col][col][0] / den, ii = -a[col][col][1] / den;
        for (int j = 0; j < 12; ++j) {
            const double re = a[col][j][0] * ir - a[col][j][1] * ii;
            const double im = a[col][j][0] * ii + a[col][j][1] * ir;
            a[col][j][0] = re;
            a[col][j][1] = im;
        }
        // eliminate the column from every other row
        for (int r = 0; r < 6; ++r) {
            if (r == col) continue;
            const double fr = a[r][col][0], fi = a[r][col][1];
            for (int j = 0; j < 12; ++j) {
                a[r][j][0] -= fr * a[col][j][0] - fi * a[col][j][1];
                a[r][j][1] -= fr * a[col][j][1] + fi * a[col][j][0];
            }
        }
    }
    double ci[36];
    for (int r = 0; r < 6; ++r) ci[r] = a[r][6 + r][0];
    {
        int k = 6;
        for (int r = 1; r < 6; ++r)
            for (int j = 0; j < r; ++j) {
                ci[k++] = a[r][6 + j][0];
                ci[k++] = a[r][6 + j][1];
            }
    }
    for (int k = 0; k < 36; ++k)
        if (!(fabs(c[k]) < 6.0e4 && fabs(ci[k]) < 6.0e4)) bad |= kClovF16Range;
    if (bad) atomicOr(flag, bad);
    if (bad & (kClovNotHermitian | kClovSingular)) return;
    if (t.A[WL_F64]) {
        store_clover_block<WL_F64>(t.A[WL_F64], g.Vh, i, b, c);
        store_clover_block<WL_F64>(t.Ainv[WL_F64], g.Vh, i, b, ci);
    }
    if (t.A[WL_F32]) {
        store_clover_block<WL_F32>(t.A[WL_F32], g.Vh, i, b, c);
        store_clover_block<WL_F32>(t.Ainv[WL_F32], g.Vh, i, b, ci);
    }
    if (t.A[WL_DF64]) {
        store_clover_block<WL_DF64>(t.A[WL_DF64], g.Vh, i, b, c);
        store_clover_block<WL_DF64>(t.Ainv[WL_DF64], g.Vh, i, b, ci);
    }
    if (t.A[WL_F16] && !(bad & kClovF16Range)) {
        store_clover_block<WL_F16>(t.A[WL_F16], g.Vh, i, b, c);
        store_clover_block<WL_F16>(t.Ainv[WL_F16], g.Vh, i, b, ci);
    }
}

// out = C in on half fields, C = A or A^-1 of one parity.
template <int P>
__global__ void clover_apply_kernel(char* out, const char* in, const void* cl, long long Vh, size_t fb)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Vh) return;
    const int rhs = blockIdx.y;
    cx<typename Prec<P>::real> v[12];
    load_spinor<P>(v, in + rhs * fb, Vh, i);
    clover_mul<P>(v, cl, Vh, i);
    store_spinor<P>(out + rhs * fb, Vh, i, v);
}

void free_clover(wl_gauge g)
{
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 2; ++q)
            for (int k = 0; k < 2; ++k) {
                if (g->clov[p][q][k]) cudaFree(g->clov[p][q][k]);
                g->clov[p][q][k] = nullptr;
            }
    g->has_clover = false;
}

int launch_clover_apply(wl_gauge g, int prec, void* out, const void* in, int parity, int inverse,
                        int nrhs, cudaStream_t s, long long rs_out, long long rs_in)
{
    const void* cl = g->clov[prec][parity][inverse ? 1 : 0];
    if (!cl) return set_error(WL_ERR_STATE, "gauge object has no clover term in this precision");
    const long long Vh = g->geo.Vh;
    const size_t fb = spinor_field_bytes(prec, Vh);
    if (rs_out == 0) rs_out = (long long)fb;
    if (rs_in == 0) rs_in = (long long)fb;
    const int block = 128;
    for (int r0 = 0; r0 < nrhs; r0 += 65535) {
        const int n = nrhs - r0 < 65535 ? nrhs - r0 : 65535;
        const dim3 grid((unsigned)((Vh + block - 1) / block), (unsigned)n);
        char* o = (char*)out + (long long)r0 * rs_out;
        const char* x = (const char*)in + (long long)r0 * rs_in;
        if (rs_out != (long long)fb || rs_in != (long long)fb) {
            // strided right-hand sides: one launch each
            for (int r = 0; r < n; ++r) {
                WL_TRY(launch_clover_apply(g, prec, o + r * rs_out, x + r * rs_in, parity, inverse, 1, s, 0, 0));
            }
            continue;
        }
        switch (prec) {
            case WL_F64: clover_apply_kernel<WL_F64><<<grid, block, 0, s>>>(o, x, cl, Vh, fb); break;
            case WL_F32: clover_apply_kernel<WL_F32><<<grid, block, 0, s>>>(o, x, cl, Vh, fb); break;
            case WL_F16: clover_apply_kernel<WL_F16><<<grid, block, 0, s>>>(o, x, cl, Vh, fb); break;
            default: clover_apply_kernel<WL_DF64><<<grid, block, 0, s>>>(o, x, cl, Vh, fb); break;
        }
        WL_CHECK_LAUNCH((double)n * Vh * (2.0 * fb / Vh + clover_site_bytes(prec)));
    }
    return WL_OK;
}

}  // namespace wl

using namespace wl;

namespace wl {

// wl_clover_set without the entry checks (also attaches a block's term)
int clover_set(wl_gauge g, const double* F, cudaStream_t s)
{
    if (!F) {
        WL_CUDA(cudaStreamSynchronize(s));
        free_clover(g);
        return WL_OK;
    }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, F) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return set_error(WL_ERR_ARG, "clover field must be device memory");
    }
    const long long Vh = g->geo.Vh;
    CloverTargets t[2];
    for (int p = 0; p < 2; ++p)
        for (int prec = 0; prec < 4; ++prec) {
            t[p].A[prec] = t[p].Ainv[prec] = nullptr;
            if (!g->links[prec][0]) continue;
            for (int k = 0; k < 2; ++k)
                if (!g->clov[prec][p][k]) {
                    void* q = nullptr;
                    if (cudaMalloc(&q, clover_field_bytes(prec, Vh)) != cudaSuccess) {
                        cudaGetLastError();
                        free_clover(g);
                        return set_error(WL_ERR_CUDA, "cudaMalloc failed for the clover term");
                    }
                    g->clov[prec][p][k] = q;
                }
            t[p].A[prec] = g->clov[prec][p][0];
            t[p].Ainv[prec] = g->clov[prec][p][1];
        }
    int* flag = nullptr;
    WL_CUDA(cudaMalloc((void**)&flag, sizeof(int)));
    int hflag = 0;
    int rc = WL_OK;
    if (cudaMemsetAsync(flag, 0, sizeof(int), s) == cudaSuccess) {
        const int block = 128;
        const unsigned grid = (unsigned)((2 * Vh + block - 1) / block);
        for (int p = 0; p < 2 && rc == WL_OK; ++p) {
            build_clover_kernel<<<grid, block, 0, s>>>(F, g->geo, p, t[p], flag);
            if (cudaGetLastError() != cudaSuccess) rc = set_error(WL_ERR_CUDA, "clover set-up launch failed");
            count_launch(1, (double)Vh * (2 * 576.0));
        }
        if (rc == WL_OK &&
            (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaStreamSynchronize(s) != cudaSuccess))
            rc = set_error(WL_ERR_CUDA, "clover set-up failed on the device");
    } else {
        rc = set_error(WL_ERR_CUDA, "cudaMemsetAsync failed");
    }
    cudaFree(flag);
    if (rc != WL_OK) {
        cudaGetLastError();
        free_clover(g);
        return rc;
    }
    if (hflag & kClovNotHermitian) {
        free_clover(g);
        return set_error(WL_ERR_ARG, "clover field F is not Hermitian");
    }
    if (hflag & kClovSingular) {
        free_clover(g);
        return set_error(WL_ERR_ARG, "1 + F is singular at some site");
    }
    if ((hflag & kClovF16Range) && g->links[WL_F16][0]) {
        free_clover(g);
        return set_error(WL_ERR_ARG, "an entry of 1 + F or its inverse lies outside the FP16 range");
    }
    g->has_clover = true;
    return WL_OK;
}

}  // namespace wl

extern "C" int wl_clover_set(wl_gauge g, const double* F, void* stream)
{
    WL_ENTRY();
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (g->dd_part) return set_error(WL_ERR_STATE, "block of a domain decomposition: use the _dd calls");
    return clover_set(g, F, (cudaStream_t)stream);
}

extern "C" int wl_clover_apply(wl_gauge g, void* out, const void* in, int parity, int inverse,
                               wl_prec prec, int nrhs, void* stream)
{
    WL_ENTRY();
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (!out || !in) return set_error(WL_ERR_ARG, "NULL field pointer");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (parity != 0 && parity != 1) return set_error(WL_ERR_ARG, "parity must be 0 or 1");
    if (nrhs < 1) return set_error(WL_ERR_ARG, "nrhs must be >= 1");
    if (!g->has_clover) return set_error(WL_ERR_STATE, "gauge object has no clover term");
    return launch_clover_apply(g, prec, out, in, parity, inverse, nrhs, (cudaStream_t)stream, 0, 0);
}
