// wilson_solve on a decomposed lattice (dd.cuh): the BiCGStab of solver.cu
// (van der Vorst 1992; Sec. 2, the paragraph after Table 1) with FP64
// defect correction or reliable updates, run on every block in lockstep.
//
// Each block keeps its own copy of every right-hand side's scalars (Scal), as
// each process of a multi-GPU run would.  A reduction is formed per block and
// then summed over the blocks in block order (the allreduce); the sum is
// written into every block's copy, so the copies stay identical and every
// block takes the same decisions.  One iteration is
//   p update | v = M_ee p, (rhat, v) | s update | t = M_ee s, (s, t), ||t||^2 |
//   x, r update, (rhat, r), ||r||^2 -> allreduce -> advance the scalars,
// with two halo exchanges per M_ee.  The host reads block 0's copy after
// every chunk of iterations.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "dd.cuh"

namespace wl {

struct DDSolveWork {
    int inner = -1, nrhs = 0, xlo_prec = 0, outer = 0;
    size_t vb = 0;    // one inner half field
    size_t hb64 = 0;  // one FP64 (or df64) half field
    void *r[kMaxDomains] = {}, *rh[kMaxDomains] = {}, *p[kMaxDomains] = {}, *v[kMaxDomains] = {},
         *s[kMaxDomains] = {}, *t[kMaxDomains] = {}, *xlo[kMaxDomains] = {}, *tmp[kMaxDomains] = {};
    // b64, xhi, bout, x64: [even | odd] per rhs; bp, rhi: even; tmp64: odd
    double *b64[kMaxDomains] = {}, *bp[kMaxDomains] = {}, *xhi[kMaxDomains] = {}, *rhi[kMaxDomains] = {},
           *tmp64[kMaxDomains] = {}, *bout[kMaxDomains] = {}, *x64[kMaxDomains] = {};
    Scal* sc[kMaxDomains] = {};
    int* mask[kMaxDomains] = {};
    double* nrm[kMaxDomains] = {};
    double* part = nullptr;  // x/r update partials [dom][rhs][block][3]
    long long part_dom_stride = 0;
    int part_blocks = 0;
    Scal* sc_h = nullptr;     // pinned
    int* mask_h = nullptr;    // pinned
    double* nrm_h = nullptr;  // pinned
    std::vector<void*> owned;
};

}  // namespace wl

namespace wl {

void dd_free_solver(wl_dd dd)
{
    DDSolveWork* w = dd->sw;
    if (!w) return;
    for (void* q : w->owned) cudaFree(q);
    if (w->sc_h) cudaFreeHost(w->sc_h);
    if (w->mask_h) cudaFreeHost(w->mask_h);
    if (w->nrm_h) cudaFreeHost(w->nrm_h);
    delete w;
    dd->sw = nullptr;
}

static constexpr int kDDVec = 256;

// Per-block vectors of one update launch.
struct DDVecs {
    long long Vh;
    long long rs;  // bytes between right-hand sides (inner vectors)
    long long rsx; // of x_lo
    char* a[kMaxDomains];
    const char* b[kMaxDomains];
    const char* c[kMaxDomains];
    const char* d[kMaxDomains];
    const char* e[kMaxDomains];
    char* x[kMaxDomains];
    Scal* sc[kMaxDomains];
    double* part;
    long long part_dom_stride;
    int part_blocks;  // partial slots per right-hand side (allocated)
    int nparts;       // partials the x/r update leaves (its grid.x)
};

// p = r + beta (p - omega v):  a = p, b = r, c = v
template <int P>
__global__ void __launch_bounds__(kDDVec) dd_update_p_kernel(const DDVecs V)
{
    const int rhs = blockIdx.y, dom = blockIdx.z;
    const Scal& S = V.sc[dom][rhs];
    if (!S.active) return;
    __shared__ double coef[4];
    if (threadIdx.x == 0) {
        double c[4];
        beta_omega(S, c);
        for (int k = 0; k < 4; ++k) coef[k] = c[k];
    }
    __syncthreads();
    const long long i = blockIdx.x * (long long)kDDVec + threadIdx.x;
    if (i >= V.Vh) return;
    const long long o = rhs * V.rs;
    const double c[4] = {coef[0], coef[1], coef[2], coef[3]};
    p_update_site<P>(V.a[dom] + o, V.b[dom] + o, V.c[dom] + o, V.Vh, i, c);
}

// s = r - alpha v:  a = s, b = r, c = v
template <int P>
__global__ void __launch_bounds__(kDDVec) dd_update_s_kernel(const DDVecs V)
{
    const int rhs = blockIdx.y, dom = blockIdx.z;
    const Scal& S = V.sc[dom][rhs];
    if (!S.active) return;
    __shared__ double coef[2];
    if (threadIdx.x == 0) {
        const cx<double> al = safe_alpha(S);
        coef[0] = al.re;
        coef[1] = al.im;
    }
    __syncthreads();
    const long long i = blockIdx.x * (long long)kDDVec + threadIdx.x;
    if (i >= V.Vh) return;
    const long long o = rhs * V.rs;
    s_update_site<P>(V.a[dom] + o, V.b[dom] + o, V.c[dom] + o, V.Vh, i, {coef[0], coef[1]});
}

// x += alpha p + omega s; r = s - omega t; block partials of (rhat, r), ||r||^2:
// x = x_lo, a = r, b = p, c = s, d = t, e = rhat
template <int P, int PX>
__global__ void __launch_bounds__(kDDVec) dd_update_xr_kernel(const DDVecs V)
{
    const int rhs = blockIdx.y, dom = blockIdx.z;
    const Scal& S = V.sc[dom][rhs];
    if (!S.active) return;
    __shared__ double dcoef[4];
    __shared__ double sh[3 * 32];
    if (threadIdx.x == 0) {
        const cx<double> al = safe_alpha(S), om = safe_omega(S);
        dcoef[0] = al.re;
        dcoef[1] = al.im;
        dcoef[2] = om.re;
        dcoef[3] = om.im;
    }
    __syncthreads();
    using T = typename Prec<P>::real;
    const double dc[4] = {dcoef[0], dcoef[1], dcoef[2], dcoef[3]};
    T pt[3] = {0, 0, 0};  // a grid of resident blocks loops over the sites: few partials
    const long long o = rhs * V.rs;
    for (long long i = blockIdx.x * (long long)kDDVec + threadIdx.x; i < V.Vh; i += (long long)gridDim.x * kDDVec) {
        T q[3];
        xr_update_site<P, PX>(V.x[dom] + rhs * V.rsx, V.a[dom] + o, V.b[dom] + o, V.c[dom] + o, V.d[dom] + o,
                              V.e[dom] + o, V.Vh, i, dc, q);
        for (int k = 0; k < 3; ++k) pt[k] += q[k];
    }
    typename RedType<T>::type wp[3] = {(typename RedType<T>::type)pt[0], (typename RedType<T>::type)pt[1],
                                       (typename RedType<T>::type)pt[2]};
    warp_sum<3>(wp);
    double bp[3] = {(double)wp[0], (double)wp[1], (double)wp[2]};
    block_sum_warps<3>(bp, sh);
    if (threadIdx.x == 0) {
        double* q = V.part + dom * V.part_dom_stride + ((long long)rhs * V.part_blocks + blockIdx.x) * 3;
        q[0] = bp[0];
        q[1] = bp[1];
        q[2] = bp[2];
    }
}

// The allreduce of the x/r update: the total over all blocks' partials, then
// every block's copy of the scalars advances with it.  mode 0: both here;
// mode 1: this process's total to stage (summed over the processes next);
// mode 2: advance with the total in stage.
__global__ void __launch_bounds__(256) dd_advance_kernel(const DDVecs V, int ndom, int mode, double* stage)
{
    const int rhs = blockIdx.x;
    if (!V.sc[0][rhs].active) return;
    __shared__ double sh[3 * 32];
    double tot[3] = {0.0, 0.0, 0.0};
    if (mode == 2) {
        for (int k = 0; k < 3; ++k) tot[k] = stage[3 * rhs + k];
    } else {
        for (int d = 0; d < ndom; ++d) {
            double v[3];
            sum_partials<3>(V.part + d * V.part_dom_stride + (long long)rhs * V.part_blocks * 3, V.nparts, v);
            block_sum<3>(v, sh);
            if (threadIdx.x == 0)
                for (int k = 0; k < 3; ++k) tot[k] += v[k];
        }
    }
    if (threadIdx.x != 0) return;
    if (mode == 1) {
        for (int k = 0; k < 3; ++k) stage[3 * rhs + k] = tot[k];
        return;
    }
    for (int d = 0; d < ndom; ++d) {
        Scal& S = V.sc[d][rhs];
        const cx<double> al = safe_alpha(S), om = safe_omega(S);
        const double dc[4] = {al.re, al.im, om.re, om.im};
        advance_scalars(S, tot, dc);
    }
}

struct DDScal {
    Scal* sc[kMaxDomains];
    const int* mask[kMaxDomains];
};

// (Re)start the scalars of the masked right-hand sides of every block (rr
// holds (rhat, r), ||r||^2 from a preceding reduction).
__global__ void dd_init_scal_kernel(const DDScal A, int nrhs, int full)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x, dom = blockIdx.y;
    if (k >= nrhs || !A.mask[dom][k]) return;
    Scal& S = A.sc[dom][k];
    if (full) {
        S.rho_prev[0] = 1.0;
        S.rho_prev[1] = 0.0;
        S.alpha[0] = 1.0;
        S.alpha[1] = 0.0;
        S.omega[0] = 1.0;
        S.omega[1] = 0.0;
        S.rh2 = S.rr[2];
    }
    S.r2_max = S.rr[2];
    S.want_update = 0;
    S.active = S.rr[2] > S.target2 ? 1 : 0;
    if (!S.active) S.flags |= FLAG_CONVERGED;
}

struct DDMask {
    int* mask[kMaxDomains];
    unsigned word[256];  // 8192 right-hand sides per launch
};

// The host's mask as kernel parameters (see solver.cu set_mask_kernel: no
// race with a later rewrite of the host buffer).
__global__ void dd_set_mask_kernel(const DDMask M, int first, int n)
{
    const int dom = blockIdx.x;
    for (int k = threadIdx.x; k < n; k += blockDim.x) M.mask[dom][first + k] = (M.word[k >> 5] >> (k & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

template <typename F>
static int dd_dispatch(int prec, F&& f)
{
    switch (prec) {
        case WL_F64: return f(std::integral_constant<int, WL_F64>());
        case WL_F32: return f(std::integral_constant<int, WL_F32>());
        default: return f(std::integral_constant<int, WL_F16>());
    }
}

static int dd_alloc(DDSolveWork* w, void** p, size_t bytes)
{
    WL_CUDA(cudaMalloc(p, bytes));
    w->owned.push_back(*p);
    return WL_OK;
}

static int dd_ensure_ws(wl_dd dd, int inner, int nrhs)
{
    DDSolveWork* w = dd->sw;
    if (w && w->inner == inner && w->nrhs >= nrhs) return WL_OK;
    WL_CUDA(cudaDeviceSynchronize());
    dd_free_solver(dd);
    dd->sw = w = new DDSolveWork();
    w->inner = inner;
    w->nrhs = nrhs;
    w->xlo_prec = inner == WL_F64 ? WL_F64 : WL_F32;
    w->outer = inner == WL_F64 ? WL_F64 : WL_DF64;
    const long long Vh = dd->gloc.Vh;
    w->vb = spinor_field_bytes(inner, Vh);
    w->hb64 = spinor_field_bytes(WL_F64, Vh);
    const size_t n = (size_t)nrhs;
    for (int d = 0; d < dd->ndom; ++d) {
        void** iv[] = {&w->r[d], &w->rh[d], &w->p[d], &w->v[d], &w->s[d], &w->t[d], &w->tmp[d]};
        for (void** q : iv) WL_TRY(dd_alloc(w, q, w->vb * n));
        WL_TRY(dd_alloc(w, &w->xlo[d], spinor_field_bytes(w->xlo_prec, Vh) * n));
        WL_TRY(dd_alloc(w, (void**)&w->b64[d], 2 * w->hb64 * n));
        WL_TRY(dd_alloc(w, (void**)&w->bp[d], w->hb64 * n));
        WL_TRY(dd_alloc(w, (void**)&w->xhi[d], 2 * w->hb64 * n));
        WL_TRY(dd_alloc(w, (void**)&w->rhi[d], 2 * w->hb64 * n));  // both halves: the clover final check
        WL_TRY(dd_alloc(w, (void**)&w->tmp64[d], w->hb64 * n));
        if (w->outer == WL_F64) {
            w->bout[d] = w->b64[d];
            w->x64[d] = w->xhi[d];
        } else {
            WL_TRY(dd_alloc(w, (void**)&w->bout[d], 2 * w->hb64 * n));
            WL_TRY(dd_alloc(w, (void**)&w->x64[d], 2 * w->hb64 * n));
        }
        WL_TRY(dd_alloc(w, (void**)&w->sc[d], sizeof(Scal) * n));
        WL_CUDA(cudaMemset(w->sc[d], 0, sizeof(Scal) * n));
        WL_TRY(dd_alloc(w, (void**)&w->mask[d], sizeof(int) * n));
        WL_TRY(dd_alloc(w, (void**)&w->nrm[d], sizeof(double) * 3 * n));
    }
    w->part_blocks = (int)((Vh + kDDVec - 1) / kDDVec);
    w->part_dom_stride = (long long)nrhs * w->part_blocks * 3;
    WL_TRY(dd_alloc(w, (void**)&w->part, sizeof(double) * w->part_dom_stride * dd->ndom));
    WL_CUDA(cudaMallocHost((void**)&w->sc_h, sizeof(Scal) * n));
    WL_CUDA(cudaMallocHost((void**)&w->mask_h, sizeof(int) * n));
    WL_CUDA(cudaMallocHost((void**)&w->nrm_h, sizeof(double) * 3 * n));
    std::memset(w->sc_h, 0, sizeof(Scal) * n);
    return WL_OK;
}

static int dd_upload_mask(wl_dd dd, DDSolveWork* w, int nrhs, cudaStream_t s)
{
    for (int first = 0; first < nrhs; first += 8192) {
        const int n = std::min(8192, nrhs - first);
        DDMask M;
        std::memset(&M, 0, sizeof M);
        for (int d = 0; d < dd->ndom; ++d) M.mask[d] = w->mask[d];
        for (int k = 0; k < n; ++k)
            if (w->mask_h[first + k]) M.word[k >> 5] |= 1u << (k & 31);
        dd_set_mask_kernel<<<dd->ndom, 256, 0, s>>>(M, first, n);
        WL_CHECK_LAUNCH(0.0);
    }
    return WL_OK;
}

static int dd_push_scalars(wl_dd dd, DDSolveWork* w, int nrhs, cudaStream_t s)
{
    for (int d = 0; d < dd->ndom; ++d)
        WL_CUDA(cudaMemcpyAsync(w->sc[d], w->sc_h, sizeof(Scal) * nrhs, cudaMemcpyHostToDevice, s));
    return WL_OK;
}

static int dd_read_scalars(DDSolveWork* w, int nrhs, cudaStream_t s)
{
    WL_CUDA(cudaMemcpyAsync(w->sc_h, w->sc[0], sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, s));
    WL_CUDA(cudaStreamSynchronize(s));
    return WL_OK;
}

static int dd_read_norms(DDSolveWork* w, int nrhs, cudaStream_t s)
{
    WL_CUDA(cudaMemcpyAsync(w->nrm_h, w->nrm[0], sizeof(double) * 3 * nrhs, cudaMemcpyDeviceToHost, s));
    WL_CUDA(cudaStreamSynchronize(s));
    return WL_OK;
}

// Global (a, b), ||b||^2 of per-block half fields into out[d] + rhs * stride.
static int dd_dot(wl_dd dd, int prec, void* const* a, void* const* b, int nhalf, long long rs, int nrhs,
                  double* const* out, int out_stride, const int* const* mask, int mask_stride, cudaStream_t s)
{
    if (dd->loc_rhs < nrhs) {
        WL_CUDA(cudaDeviceSynchronize());
        if (dd->loc) cudaFree(dd->loc);
        dd->loc = nullptr;
        WL_CUDA(cudaMalloc((void**)&dd->loc, sizeof(double) * 3 * nrhs * dd->ndom));
        dd->loc_rhs = nrhs;
    }
    double* loc[kMaxDomains];
    for (int d = 0; d < dd->ndom; ++d) {
        loc[d] = dd->loc + (size_t)3 * nrhs * d;
        WL_TRY(launch_cdot(dd->dom[d], prec, a[d], b[d], nhalf, nrhs, loc[d], 3, mask ? mask[d] : nullptr, s, rs));
    }
    return dd_allreduce(dd, loc, out, out_stride, nrhs, mask, mask_stride, s);
}

// v = M_ee u (inner precision) with (w, v), ||v||^2 into every block's scalars.
static int dd_apply_A(wl_dd dd, DDSolveWork* w, void* const* out, void* const* in, void* const* wdot,
                      size_t scal_off, int nrhs, cudaStream_t s)
{
    const int P = w->inner;
    const size_t hb = w->vb;
    DDLaunch h1;
    h1.prec = P;
    h1.parity0 = 1;
    h1.nrhs = nrhs;
    for (int d = 0; d < dd->ndom; ++d) {
        h1.in[d][0] = in[d];
        h1.out[d][0] = w->tmp[d];
        h1.active[d] = &w->sc[d][0].active;
    }
    h1.rs_in = h1.rs_out = (long long)hb;
    h1.active_stride = kActiveStride;
    const bool clov = dd->dom[0]->has_clover;
    if (clov) h1.cl_mode = kClOut;  // tmp = A_oo^-1 H_oe in
    WL_TRY(dd_launch_hop(dd, h1, s));
    DDLaunch h2 = h1;
    h2.parity0 = 0;
    for (int d = 0; d < dd->ndom; ++d) {
        h2.in[d][0] = w->tmp[d];
        h2.out[d][0] = out[d];
        if (clov) h2.x2[d][0] = in[d];  // out = A_ee in - kappa^2 H_eo tmp
        else h2.x1[d][0] = in[d];
        h2.w[d][0] = wdot[d];
        h2.dot_out[d] = (double*)((char*)w->sc[d] + scal_off);
    }
    h2.rs_x1 = h2.rs_x2 = h2.rs_w = (long long)hb;
    if (clov) {
        h2.b1 = 1.0;
        h2.cl_mode = kClX2;
    } else {
        h2.cl_mode = kClNone;
    }
    h2.a = -dd->global.kappa * dd->global.kappa;
    h2.dot = true;
    h2.dot_stride = kScalStride;
    return dd_launch_hop(dd, h2, s);
}

static DDVecs dd_vecs(wl_dd dd, DDSolveWork* w)
{
    DDVecs V;
    std::memset(&V, 0, sizeof V);
    V.Vh = dd->gloc.Vh;
    V.rs = (long long)w->vb;
    V.rsx = (long long)spinor_field_bytes(w->xlo_prec, dd->gloc.Vh);
    for (int d = 0; d < dd->ndom; ++d) V.sc[d] = w->sc[d];
    V.part = w->part;
    V.part_dom_stride = w->part_dom_stride;
    V.part_blocks = w->part_blocks;
    V.nparts = std::max(1, std::min(w->part_blocks, 4 * dd->dom[0]->num_sms / std::max(1, dd->ndom)));
    return V;
}

static int dd_iteration(wl_dd dd, DDSolveWork* w, int nrhs, cudaStream_t s)
{
    const int P = w->inner;
    const dim3 grid((unsigned)w->part_blocks, (unsigned)nrhs, (unsigned)dd->ndom);
    const double vbytes = (double)w->vb * nrhs * dd->ndom;
    DDVecs V = dd_vecs(dd, w);
    for (int d = 0; d < dd->ndom; ++d) {
        V.a[d] = (char*)w->p[d];
        V.b[d] = (const char*)w->r[d];
        V.c[d] = (const char*)w->v[d];
    }
    WL_TRY(dd_dispatch(P, [&](auto pc) -> int {
        dd_update_p_kernel<decltype(pc)::value><<<grid, kDDVec, 0, s>>>(V);
        WL_CHECK_LAUNCH(4.0 * vbytes);
        return WL_OK;
    }));
    WL_TRY(dd_apply_A(dd, w, w->v, w->p, w->rh, offsetof(Scal, rv), nrhs, s));
    for (int d = 0; d < dd->ndom; ++d) {
        V.a[d] = (char*)w->s[d];
        V.b[d] = (const char*)w->r[d];
        V.c[d] = (const char*)w->v[d];
    }
    WL_TRY(dd_dispatch(P, [&](auto pc) -> int {
        dd_update_s_kernel<decltype(pc)::value><<<grid, kDDVec, 0, s>>>(V);
        WL_CHECK_LAUNCH(3.0 * vbytes);
        return WL_OK;
    }));
    WL_TRY(dd_apply_A(dd, w, w->t, w->s, w->s, offsetof(Scal, st), nrhs, s));
    for (int d = 0; d < dd->ndom; ++d) {
        V.x[d] = (char*)w->xlo[d];
        V.a[d] = (char*)w->r[d];
        V.b[d] = (const char*)w->p[d];
        V.c[d] = (const char*)w->s[d];
        V.d[d] = (const char*)w->t[d];
        V.e[d] = (const char*)w->rh[d];
    }
    WL_TRY(dd_dispatch(P, [&](auto pc) -> int {
        constexpr int PP = decltype(pc)::value;
        const dim3 rgrid((unsigned)V.nparts, grid.y, grid.z);
        if (w->xlo_prec == WL_F64) dd_update_xr_kernel<PP, WL_F64><<<rgrid, kDDVec, 0, s>>>(V);
        else dd_update_xr_kernel<PP, WL_F32><<<rgrid, kDDVec, 0, s>>>(V);
        WL_CHECK_LAUNCH((5.0 * w->vb + 2.0 * V.rsx) * nrhs * dd->ndom);
        return WL_OK;
    }));
    if (!dd->has_tr) {
        dd_advance_kernel<<<nrhs, 256, 0, s>>>(V, dd->ndom, 0, nullptr);
        WL_CHECK_LAUNCH(0.0);
        return WL_OK;
    }
    WL_TRY(dd_ensure_stage(dd, nrhs));
    dd_advance_kernel<<<nrhs, 256, 0, s>>>(V, dd->ndom, 1, dd->stage);
    WL_CHECK_LAUNCH(0.0);
    WL_TRY(dd_cross_sum(dd, nrhs, s));
    dd_advance_kernel<<<nrhs, 256, 0, s>>>(V, dd->ndom, 2, dd->stage);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

// r = b' - M_ee x in the outer precision for the masked right-hand sides,
// with the global ||r||^2 in nrm.
static int dd_residual(wl_dd dd, DDSolveWork* w, int nrhs, cudaStream_t s)
{
    const long long hb = (long long)w->hb64;
    DDLaunch h1;
    h1.prec = w->outer;
    h1.parity0 = 1;
    h1.nrhs = nrhs;
    for (int d = 0; d < dd->ndom; ++d) {
        h1.in[d][0] = w->xhi[d];
        h1.out[d][0] = w->tmp64[d];
        h1.active[d] = w->mask[d];
    }
    h1.rs_in = 2 * hb;
    h1.rs_out = hb;
    const bool clov = dd->dom[0]->has_clover;
    if (clov) h1.cl_mode = kClOut;  // tmp = A_oo^-1 H_oe x
    WL_TRY(dd_launch_hop(dd, h1, s));
    DDLaunch h2;
    h2.prec = w->outer;
    if (clov) h2.cl_mode = kClX2;  // r = b' - A_ee x + kappa^2 H_eo tmp
    h2.parity0 = 0;
    h2.nrhs = nrhs;
    for (int d = 0; d < dd->ndom; ++d) {
        h2.in[d][0] = w->tmp64[d];
        h2.out[d][0] = w->rhi[d];
        h2.x1[d][0] = w->bp[d];
        h2.x2[d][0] = w->xhi[d];
        h2.dot_out[d] = w->nrm[d];
        h2.active[d] = w->mask[d];
    }
    h2.rs_in = hb;
    h2.rs_out = hb;
    h2.rs_x1 = hb;
    h2.rs_x2 = 2 * hb;
    h2.b1 = -1.0;
    h2.a = dd->global.kappa * dd->global.kappa;
    h2.dot = true;
    return dd_launch_hop(dd, h2, s);
}

// Start an inner solve for the masked right-hand sides: r = r_hi, rhat = r,
// p = v = x_lo = 0, fresh scalars.
static int dd_inner_start(wl_dd dd, DDSolveWork* w, int nrhs, const std::vector<double>& target2, double delta2,
                          cudaStream_t s)
{
    const int P = w->inner;
    for (int k = 0; k < nrhs; ++k) {
        Scal& S = w->sc_h[k];
        S.active = 0;
        if (!w->mask_h[k]) continue;
        S.target2 = target2[k];
        S.delta2 = delta2;
        S.flags = 0;
        S.want_update = 0;
    }
    WL_TRY(dd_push_scalars(dd, w, nrhs, s));
    WL_TRY(dd_upload_mask(dd, w, nrhs, s));
    const int* masks[kMaxDomains];
    double* rr[kMaxDomains];
    for (int d = 0; d < dd->ndom; ++d) {
        wl_gauge g = dd->dom[d];
        WL_TRY(launch_convert(g, P, w->r[d], w->outer, w->rhi[d], 1, nrhs, w->mask[d], s));
        WL_TRY(launch_convert(g, P, w->rh[d], P, w->r[d], 1, nrhs, w->mask[d], s));
        WL_TRY(launch_zero(g, P, w->p[d], 1, nrhs, w->mask[d], s));
        WL_TRY(launch_zero(g, P, w->v[d], 1, nrhs, w->mask[d], s));
        WL_TRY(launch_zero(g, w->xlo_prec, w->xlo[d], 1, nrhs, w->mask[d], s));
        masks[d] = w->mask[d];
        rr[d] = w->sc[d][0].rr;
    }
    WL_TRY(dd_dot(dd, P, w->rh, w->r, 1, 0, nrhs, rr, kScalStride, masks, 1, s));
    DDScal A;
    for (int d = 0; d < dd->ndom; ++d) {
        A.sc[d] = w->sc[d];
        A.mask[d] = w->mask[d];
    }
    dd_init_scal_kernel<<<dim3((nrhs + 63) / 64, dd->ndom), 64, 0, s>>>(A, nrhs, 1);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

// Reliable update of the masked right-hand sides: x_hi += x_lo, r_hi = b' -
// M_ee x_hi, r = r_hi, rho = (rhat, r); the Krylov directions are kept.
static int dd_reliable_update(wl_dd dd, DDSolveWork* w, int nrhs, cudaStream_t s)
{
    const int P = w->inner;
    WL_TRY(dd_upload_mask(dd, w, nrhs, s));
    for (int d = 0; d < dd->ndom; ++d) {
        WL_TRY(launch_accum_hi(dd->dom[d], w->outer, w->xhi[d], w->xlo_prec, w->xlo[d], 1, nrhs, w->mask[d], s,
                               2 * (long long)w->hb64));
        WL_TRY(launch_zero(dd->dom[d], w->xlo_prec, w->xlo[d], 1, nrhs, w->mask[d], s));
    }
    WL_TRY(dd_residual(dd, w, nrhs, s));
    const int* masks[kMaxDomains];
    double* rr[kMaxDomains];
    for (int d = 0; d < dd->ndom; ++d) {
        WL_TRY(launch_convert(dd->dom[d], P, w->r[d], w->outer, w->rhi[d], 1, nrhs, w->mask[d], s));
        masks[d] = w->mask[d];
        rr[d] = w->sc[d][0].rr;
    }
    WL_TRY(dd_dot(dd, P, w->rh, w->r, 1, 0, nrhs, rr, kScalStride, masks, 1, s));
    DDScal A;
    for (int d = 0; d < dd->ndom; ++d) {
        A.sc[d] = w->sc[d];
        A.mask[d] = w->mask[d];
    }
    dd_init_scal_kernel<<<dim3((nrhs + 63) / 64, dd->ndom), 64, 0, s>>>(A, nrhs, 0);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

}  // namespace wl

using namespace wl;

extern "C" int wilson_solve_dd(wl_dd dd, double* const* x, const double* const* b, int nrhs,
                               const wl_solve_params* prm, wl_solve_info* info, void* stream)
{
    WL_ENTRY();
    const auto t0 = std::chrono::steady_clock::now();
    if (!dd) return set_error(WL_ERR_ARG, "NULL decomposition");
    if (!x || !b || !prm || !info) return set_error(WL_ERR_ARG, "NULL pointer");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    if (prm->inner < WL_F64 || prm->inner > WL_F16) return set_error(WL_ERR_ARG, "unknown inner precision");
    if (!(prm->tol > 0.0)) return set_error(WL_ERR_ARG, "tol must be > 0");
    if (prm->maxiter < 1) return set_error(WL_ERR_ARG, "maxiter must be >= 1");
    if (!prm->eo) return set_error(WL_ERR_ARG, "the decomposed solve takes even-odd systems (eo = 1)");
    for (int d = 0; d < dd->ndom; ++d) {
        if (!x[d] || !b[d]) return set_error(WL_ERR_ARG, "NULL block field");
        if (!dd->dom[d]->links[prm->inner][0])
            return set_error(WL_ERR_STATE, "decomposition was created without the inner precision");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int P = prm->inner;
    WL_TRY(dd_ensure_ws(dd, P, nrhs));
    DDSolveWork* w = dd->sw;
    const long long hb = (long long)w->hb64;
    const int nd = dd->ndom;
    const double kappa = dd->global.kappa;

    // b -> internal FP64 [even | odd]; ||b||^2; b in the outer precision
    for (int d = 0; d < nd; ++d) {
        wl_gauge g = dd->dom[d];
        WL_TRY(field_to_internal(g, w->b64[d], b[d], 0, WL_F64, nrhs, s, 2 * hb));
        WL_TRY(field_to_internal(g, (char*)w->b64[d] + hb, b[d], 1, WL_F64, nrhs, s, 2 * hb));
        if (w->bout[d] != w->b64[d])
            WL_TRY(launch_convert(g, w->outer, w->bout[d], WL_F64, w->b64[d], 2, nrhs, nullptr, s));
        WL_CUDA(cudaMemsetAsync(w->xhi[d], 0, 2 * hb * nrhs, s));
    }
    WL_TRY(dd_dot(dd, WL_F64, (void* const*)w->b64, (void* const*)w->b64, 2, 0, nrhs, w->nrm, 3, nullptr, 1, s));
    WL_TRY(dd_read_norms(w, nrhs, s));
    std::vector<double> bnorm2(nrhs), rnorm2(nrhs), target2(nrhs), true_resid(nrhs, 0.0);
    for (int k = 0; k < nrhs; ++k) bnorm2[k] = w->nrm_h[3 * k + 2];
    const bool clov = dd->dom[0]->has_clover;
    {  // b' = b_e + kappa H_eo b_o (outer precision; H_eo A_oo^-1 b_o with a clover term)
        DDLaunch h;
        h.prec = w->outer;
        h.parity0 = 0;
        h.nrhs = nrhs;
        for (int d = 0; d < nd; ++d) {
            h.in[d][0] = (const char*)w->bout[d] + hb;
            h.out[d][0] = w->bp[d];
            h.x1[d][0] = w->bout[d];
            if (clov) {
                WL_TRY(launch_clover_apply(dd->dom[d], w->outer, w->tmp64[d], (const char*)w->bout[d] + hb, 1, 1, nrhs,
                                           s, hb, 2 * hb));
                h.in[d][0] = w->tmp64[d];
            }
        }
        h.rs_in = clov ? hb : 2 * hb;
        h.rs_x1 = 2 * hb;
        h.rs_out = hb;
        h.a = kappa;
        WL_TRY(dd_launch_hop(dd, h, s));
    }
    std::vector<int> done(nrhs, 0), status(nrhs, WL_OK), outer(nrhs, 0), restarts(nrhs, 0), part(nrhs, 0),
        in_inner(nrhs, 0), poisoned(nrhs, 0), before(nrhs, 0);
    for (int k = 0; k < nrhs; ++k) {
        if (bnorm2[k] == 0.0) done[k] = 1;
        std::memset(&w->sc_h[k], 0, sizeof(Scal));
        w->mask_h[k] = done[k] ? 0 : 1;
    }
    WL_TRY(dd_push_scalars(dd, w, nrhs, s));
    WL_TRY(dd_upload_mask(dd, w, nrhs, s));
    {  // x = 0: r = b'
        const int* masks[kMaxDomains];
        for (int d = 0; d < nd; ++d) {
            WL_CUDA(cudaMemcpyAsync(w->rhi[d], w->bp[d], hb * nrhs, cudaMemcpyDeviceToDevice, s));
            masks[d] = w->mask[d];
        }
        WL_TRY(dd_dot(dd, w->outer, (void* const*)w->bp, (void* const*)w->bp, 1, 0, nrhs, w->nrm, 3, masks, 1, s));
        WL_TRY(dd_read_norms(w, nrhs, s));
        for (int k = 0; k < nrhs; ++k) rnorm2[k] = w->mask_h[k] ? w->nrm_h[3 * k + 2] : 0.0;
    }
    const double delta2 = prm->delta > 0.0 ? prm->delta * prm->delta : 0.0;
    const double inner_tol = prm->inner_tol > 0.0 ? prm->inner_tol : (P == WL_F64 ? 0.0 : P == WL_F32 ? 3e-6 : 1e-3);
    const int chunk = prm->graph_iters > 0 ? prm->graph_iters : prm->graph_iters < 0 ? -prm->graph_iters : 4;
    double safety = 0.5;
    int final_rounds = 0;

    for (;;) {
        for (;;) {  // outer rounds: FP64 residual -> inner solve -> x += e
            int any = 0;
            for (int k = 0; k < nrhs; ++k) {
                w->mask_h[k] = 0;
                if (done[k]) continue;
                const double goal2 = safety * safety * prm->tol * prm->tol * bnorm2[k];
                if (rnorm2[k] <= goal2) { done[k] = 1; continue; }
                if (!std::isfinite(rnorm2[k])) { done[k] = 1; status[k] = WL_ERR_NAN; continue; }
                if (w->sc_h[k].iters >= prm->maxiter) { done[k] = 1; status[k] = WL_ERR_NOT_CONVERGED; continue; }
                w->mask_h[k] = 1;
                any = 1;
                double t2 = inner_tol * inner_tol * rnorm2[k];
                if (delta2 > 0.0 || t2 < goal2) t2 = goal2;
                target2[k] = t2;
            }
            if (!any) break;
            for (int k = 0; k < nrhs; ++k) {
                before[k] = w->sc_h[k].iters;
                part[k] = in_inner[k] = w->mask_h[k];
                poisoned[k] = 0;
            }
            WL_TRY(dd_inner_start(dd, w, nrhs, target2, delta2, s));
            for (;;) {  // chunks of iterations
                int most = 0;
                for (int k = 0; k < nrhs; ++k)
                    if (in_inner[k]) most = std::max(most, w->sc_h[k].iters);
                const int kit = std::min(chunk, prm->maxiter - most);
                if (kit <= 0) break;
                for (int it = 0; it < kit; ++it) WL_TRY(dd_iteration(dd, w, nrhs, s));
                WL_TRY(dd_read_scalars(w, nrhs, s));
                int upd = 0, stopped = 0;
                for (int k = 0; k < nrhs; ++k) {
                    w->mask_h[k] = 0;
                    if (!in_inner[k]) continue;
                    Scal& S = w->sc_h[k];
                    if (S.active && S.iters >= prm->maxiter) {
                        S.active = 0;
                        S.flags |= FLAG_MAXITER;
                        stopped = 1;
                    }
                    if (S.active) {
                        if (S.want_update) { w->mask_h[k] = 1; upd = 1; }
                        continue;
                    }
                    in_inner[k] = 0;
                    if (S.flags & (FLAG_BREAKDOWN | FLAG_NAN)) {
                        if (S.flags & FLAG_NAN) poisoned[k] = 1;
                        if (++restarts[k] > 5) {
                            done[k] = 1;
                            status[k] = (S.flags & FLAG_NAN) ? WL_ERR_NAN : WL_ERR_BREAKDOWN;
                        }
                    }
                }
                if (stopped) WL_TRY(dd_push_scalars(dd, w, nrhs, s));
                if (upd) {
                    WL_TRY(dd_reliable_update(dd, w, nrhs, s));
                    for (int k = 0; k < nrhs; ++k)
                        if (w->mask_h[k]) outer[k]++;
                    WL_TRY(dd_read_scalars(w, nrhs, s));
                }
                bool alive = false;
                for (int k = 0; k < nrhs; ++k) alive |= in_inner[k] != 0;
                if (!alive) break;
            }
            // end of the round: x += x_lo (a NaN correction is dropped), FP64 residual
            int any_poison = 0;
            for (int k = 0; k < nrhs; ++k) {
                w->mask_h[k] = poisoned[k];
                any_poison |= poisoned[k];
                in_inner[k] = 0;
            }
            if (any_poison) {
                WL_TRY(dd_upload_mask(dd, w, nrhs, s));
                for (int d = 0; d < nd; ++d)
                    WL_TRY(launch_zero(dd->dom[d], w->xlo_prec, w->xlo[d], 1, nrhs, w->mask[d], s));
            }
            for (int k = 0; k < nrhs; ++k) w->mask_h[k] = part[k];
            WL_TRY(dd_upload_mask(dd, w, nrhs, s));
            for (int d = 0; d < nd; ++d)
                WL_TRY(launch_accum_hi(dd->dom[d], w->outer, w->xhi[d], w->xlo_prec, w->xlo[d], 1, nrhs, w->mask[d], s,
                                       2 * hb));
            WL_TRY(dd_residual(dd, w, nrhs, s));
            WL_TRY(dd_read_norms(w, nrhs, s));
            for (int k = 0; k < nrhs; ++k)
                if (part[k]) {
                    rnorm2[k] = w->nrm_h[3 * k + 2];
                    outer[k]++;
                    if (w->sc_h[k].iters == before[k]) done[k] = 1;  // the round could not move
                    if (outer[k] > kMaxOuter && !done[k]) {
                        done[k] = 1;
                        status[k] = WL_ERR_NOT_CONVERGED;
                    }
                }
        }
        // x in FP64, x_o = b_o + kappa H_oe x_e, and the true residual b_e - x_e +
        // kappa H_eo x_o (the odd half is zero by construction of x_o)
        for (int d = 0; d < nd; ++d)
            if (w->x64[d] != w->xhi[d])
                WL_TRY(launch_convert(dd->dom[d], WL_F64, w->x64[d], w->outer, w->xhi[d], 1, nrhs, nullptr, s, 2 * hb,
                                      2 * hb));
        {
            DDLaunch h;
            h.prec = WL_F64;
            h.parity0 = 1;
            h.nrhs = nrhs;
            for (int d = 0; d < nd; ++d) {
                h.in[d][0] = w->x64[d];
                h.out[d][0] = (char*)w->x64[d] + hb;
                h.x1[d][0] = (const char*)w->b64[d] + hb;
            }
            h.rs_in = h.rs_out = h.rs_x1 = 2 * hb;
            h.a = kappa;
            if (clov) h.cl_mode = kClOut;  // x_o = A_oo^-1 (b_o + kappa H_oe x_e)
            WL_TRY(dd_launch_hop(dd, h, s));
            // r_p = b_p - A_pp x_p + kappa H x_{1-p}: the even half (the odd one
            // is zero by construction of x_o); both with a clover term, whose
            // A_oo^-1 leaves a rounding-level odd residual
            DDLaunch r;
            r.prec = WL_F64;
            r.parity0 = 0;
            r.nparity = clov ? 2 : 1;
            r.nrhs = nrhs;
            for (int d = 0; d < nd; ++d) {
                r.in[d][0] = (const char*)w->x64[d] + hb;
                r.in[d][1] = w->x64[d];
                r.out[d][0] = w->rhi[d];
                r.out[d][1] = (char*)w->rhi[d] + hb;
                r.x1[d][0] = w->b64[d];
                r.x1[d][1] = (const char*)w->b64[d] + hb;
                r.x2[d][0] = w->x64[d];
                r.x2[d][1] = (const char*)w->x64[d] + hb;
                r.dot_out[d] = w->nrm[d];
            }
            r.rs_in = r.rs_x1 = r.rs_x2 = r.rs_out = 2 * hb;
            r.b1 = -1.0;
            r.a = kappa;
            r.dot = true;
            if (clov) r.cl_mode = kClX2;
            WL_TRY(dd_launch_hop(dd, r, s));
        }
        WL_TRY(dd_read_norms(w, nrhs, s));
        bool retry = false;
        for (int k = 0; k < nrhs; ++k) {
            const double tr = bnorm2[k] > 0 ? std::sqrt(w->nrm_h[3 * k + 2] / bnorm2[k]) : 0.0;
            true_resid[k] = tr;
            if (status[k] == WL_OK && !(tr <= prm->tol)) {
                if (final_rounds < 3 && w->sc_h[k].iters < prm->maxiter) {
                    done[k] = 0;
                    retry = true;
                } else {
                    status[k] = std::isfinite(tr) ? WL_ERR_NOT_CONVERGED : WL_ERR_NAN;
                }
            }
        }
        if (!retry) break;
        ++final_rounds;
        safety *= 0.1;  // the Schur residual met the goal but the full one did not: aim lower
        for (int k = 0; k < nrhs; ++k) w->mask_h[k] = done[k] ? 0 : 1;
        WL_TRY(dd_upload_mask(dd, w, nrhs, s));
        WL_TRY(dd_residual(dd, w, nrhs, s));
        WL_TRY(dd_read_norms(w, nrhs, s));
        for (int k = 0; k < nrhs; ++k)
            if (w->mask_h[k]) rnorm2[k] = w->nrm_h[3 * k + 2];
    }
    for (int d = 0; d < nd; ++d) {
        WL_TRY(field_to_canonical(dd->dom[d], x[d], w->x64[d], 0, WL_F64, nrhs, s, 2 * hb));
        WL_TRY(field_to_canonical(dd->dom[d], x[d], (const char*)w->x64[d] + hb, 1, WL_F64, nrhs, s, 2 * hb));
    }
    WL_CUDA(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int rc = WL_OK;
    for (int k = 0; k < nrhs; ++k) {
        info[k].iters = w->sc_h[k].iters;
        info[k].outer = outer[k];
        info[k].restarts = restarts[k];
        info[k].status = status[k];
        info[k].true_resid = true_resid[k];
        info[k].secs = secs;
        if (status[k] != WL_OK && rc == WL_OK) rc = status[k];
    }
    if (rc != WL_OK) set_error(rc, "at least one right-hand side did not reach tol");
    return rc;
}
