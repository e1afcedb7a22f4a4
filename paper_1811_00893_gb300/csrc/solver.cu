// BiCGStab for D x = b (Sec. 2: the Krylov solver for the non-Hermitian
// Wilson matrix) with a lower-precision inner iteration and FP64 correction
// (the "inner solver of a mixed precision solver" of the same paragraph).
//
// Iteration (van der Vorst 1992, shadow residual rhat = r0), one right-hand
// side per grid row, every scalar kept on the device:
//   K_b   beta = (rho/rho_prev)(alpha/omega);  p = r + beta (p - omega v)
//   A     v = A p                 (+ fused (rhat, v), ||v||^2)
//   K_c   alpha = rho / (rhat, v); s = r - alpha v
//   A     t = A s                 (+ fused (s, t), ||t||^2)
//   K_a   omega = (t, s)/(t, t);   x += alpha p + omega s;  r = s - omega t
//         (+ fused rho' = (rhat, r), ||r||^2; the last block advances the
//         scalars and decides convergence / breakdown / reliable update)
// A is M_ee = 1 - kappa^2 H_eo H_oe (two hopping launches) or the full D.
// Kernels read coefficients at block start; coefficients are written only by
// the last block of a reduction, after every other block of that launch has
// finished, so no launch sees a half-updated scalar.
//
// Outer loop (FP64): r = b' - A x in FP64, inner solve of A e = r in the
// inner precision, x += e in FP64.  With delta > 0 the inner Krylov space is
// kept and only the residual is replaced (reliable updates, Sleijpen & van
// der Vorst 1996); otherwise each inner solve restarts (defect correction).
// Convergence is always judged on the FP64 true residual of the full D.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace wl {

struct Scal {
    double rr[3];       // (rhat, r) re, im; ||r||^2
    double rho_prev[2];
    double alpha[2];
    double omega[2];
    double rv[3];       // (rhat, v); ||v||^2
    double st[3];       // (s, t); ||t||^2
    double target2;     // stop when ||r||^2 <= target2
    double r2_max;      // largest ||r||^2 since the last reliable update
    double delta2;      // reliable-update threshold delta^2 (0: off)
    double rh2;         // ||rhat||^2
    int active;
    int iters;
    int flags;
    int want_update;
};

enum { FLAG_CONVERGED = 1, FLAG_BREAKDOWN = 2, FLAG_NAN = 4, FLAG_MAXITER = 8 };

static const int kScalStride = sizeof(Scal) / sizeof(double);
static const int kMaxOuter = 500;  // FP64 corrections per solve
static const int kActiveStride = sizeof(Scal) / sizeof(int);

struct Workspace {
    int inner = -1, nrhs = 0, eo = -1, nhalf = 0, xlo_prec = 0;
    size_t vb = 0;    // bytes of one inner vector (nhalf halves)
    size_t vb64 = 0;  // bytes of one FP64 vector (nhalf halves)
    size_t hb64 = 0;  // bytes of one FP64 half field
    // inner-precision vectors (nrhs each)
    void *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
         *xlo = nullptr, *tmp = nullptr;
    // FP64 (nrhs each): b even/odd (or full b), b', x, r, odd temporary, odd x
    double *b64 = nullptr, *bp = nullptr, *xhi = nullptr, *rhi = nullptr, *tmp64 = nullptr,
           *xo = nullptr;
    Scal* sc = nullptr;
    Scal* sc_h = nullptr;  // pinned
    int* mask = nullptr;
    int* mask_h = nullptr;  // pinned
    double* nrm = nullptr;  // 3 doubles per rhs
    double* nrm_h = nullptr;  // pinned
    // staging of host buffers
    double* stage_b = nullptr;
    double* stage_x = nullptr;
    size_t stage_bytes = 0;
    // CUDA graph of k iterations
    cudaGraphExec_t graph = nullptr;
    int graph_k = 0;
    int graph_nrhs = 0;
    int graph_red_gen = -1;
    cudaStream_t cap_stream = nullptr;  // private stream for graph capture
    long long graph_kernels = 0;
    long long graph_bytes = 0;
};

static void free_ws(Workspace* w)
{
    if (!w) return;
    void* dev[] = {w->r, w->rh, w->p, w->v, w->s, w->t, w->xlo, w->tmp, w->b64, w->bp, w->xhi,
                   w->rhi, w->tmp64, w->xo, w->sc, w->mask, w->nrm, w->stage_b, w->stage_x};
    for (void* q : dev)
        if (q) cudaFree(q);
    if (w->sc_h) cudaFreeHost(w->sc_h);
    if (w->mask_h) cudaFreeHost(w->mask_h);
    if (w->nrm_h) cudaFreeHost(w->nrm_h);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
}

}  // namespace wl

void free_workspace(wl_gauge g)
{
    if (g->ws) {
        wl::free_ws(g->ws);
        delete g->ws;
        g->ws = nullptr;
    }
}

namespace wl {

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------

struct Vec2 {
    long long Vh;
    int nhalf;
    size_t hb;
    long long rstride;
};

__device__ __forceinline__ long long split_index(const Vec2& v, long long j, long long& off)
{
    const int h = (int)(j / v.Vh);
    off = h * (long long)v.hb;
    return j - h * v.Vh;
}

__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// beta = (rho / rho_prev)(alpha / omega);  p = r + beta (p - omega v)
template <int P>
__global__ void __launch_bounds__(256) update_p_kernel(char* p, const char* r, const char* v,
                                                       Vec2 vec, const Scal* sc)
{
    using T = typename Prec<P>::real;
    const int rhs = blockIdx.y;
    const Scal& S = sc[rhs];
    if (!S.active) return;
    __shared__ T coef[4];
    if (threadIdx.x == 0) {
        const cx<double> rho = {S.rr[0], S.rr[1]}, rp = {S.rho_prev[0], S.rho_prev[1]};
        const cx<double> al = {S.alpha[0], S.alpha[1]}, om = {S.omega[0], S.omega[1]};
        const cx<double> beta = cdiv(rho, rp) * cdiv(al, om);
        coef[0] = (T)beta.re;
        coef[1] = (T)beta.im;
        coef[2] = (T)om.re;
        coef[3] = (T)om.im;
    }
    __syncthreads();
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= vec.nhalf * vec.Vh) return;
    long long off;
    const long long i = split_index(vec, j, off);
    off += rhs * vec.rstride;
    const cx<T> beta = {coef[0], coef[1]}, om = {coef[2], coef[3]};
    cx<T> pp[12], rr[12], vv[12];
    load_spinor<P>(pp, p + off, vec.Vh, i);
    load_spinor<P>(rr, r + off, vec.Vh, i);
    load_spinor<P>(vv, v + off, vec.Vh, i);
#pragma unroll
    for (int c = 0; c < 12; ++c) pp[c] = rr[c] + beta * (pp[c] - om * vv[c]);
    store_spinor<P>(p + off, vec.Vh, i, pp);
}

__device__ __forceinline__ cx<double> safe_alpha(const Scal& S)
{
    const double rv2 = S.rv[0] * S.rv[0] + S.rv[1] * S.rv[1];
    if (!(rv2 > 1e-60 * S.rh2 * S.rv[2])) return {0.0, 0.0};  // breakdown: no step
    return cdiv({S.rr[0], S.rr[1]}, {S.rv[0], S.rv[1]});
}

__device__ __forceinline__ cx<double> safe_omega(const Scal& S)
{
    if (!(S.st[2] > 0.0)) return {0.0, 0.0};
    return {S.st[0] / S.st[2], -S.st[1] / S.st[2]};  // (t, s)/(t, t) = conj((s, t))/||t||^2
}

// alpha = rho / (rhat, v);  s = r - alpha v
template <int P>
__global__ void __launch_bounds__(256) update_s_kernel(char* s, const char* r, const char* v,
                                                       Vec2 vec, const Scal* sc)
{
    using T = typename Prec<P>::real;
    const int rhs = blockIdx.y;
    const Scal& S = sc[rhs];
    if (!S.active) return;
    __shared__ T coef[2];
    if (threadIdx.x == 0) {
        const cx<double> al = safe_alpha(S);
        coef[0] = (T)al.re;
        coef[1] = (T)al.im;
    }
    __syncthreads();
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= vec.nhalf * vec.Vh) return;
    long long off;
    const long long i = split_index(vec, j, off);
    off += rhs * vec.rstride;
    const cx<T> al = {coef[0], coef[1]};
    cx<T> rr[12], vv[12];
    load_spinor<P>(rr, r + off, vec.Vh, i);
    load_spinor<P>(vv, v + off, vec.Vh, i);
#pragma unroll
    for (int c = 0; c < 12; ++c) rr[c] = rr[c] - al * vv[c];
    store_spinor<P>(s + off, vec.Vh, i, rr);
}

// omega = (t, s)/(t, t);  x += alpha p + omega s;  r = s - omega t;
// fused rho' = (rhat, r), ||r||^2; the last block advances the scalars.
template <int P, int PX>
__global__ void __launch_bounds__(256) update_xr_kernel(char* x, Vec2 vx, char* r, const char* p,
                                                        const char* s, const char* t,
                                                        const char* rh, Vec2 vec, Scal* sc,
                                                        RedScratch red)
{
    using T = typename Prec<P>::real;
    using TX = typename Prec<PX>::real;
    const int rhs = blockIdx.y;
    Scal& S = sc[rhs];
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
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double part[3] = {0, 0, 0};
    if (j < vec.nhalf * vec.Vh) {
        long long off, offx;
        const long long i = split_index(vec, j, off);
        split_index(vx, j, offx);
        off += rhs * vec.rstride;
        offx += rhs * vx.rstride;
        const cx<T> al = {(T)dcoef[0], (T)dcoef[1]}, om = {(T)dcoef[2], (T)dcoef[3]};
        cx<T> pp[12], ss[12];
        load_spinor<P>(pp, p + off, vec.Vh, i);
        load_spinor<P>(ss, s + off, vec.Vh, i);
        {
            cx<TX> xx[12];
            load_spinor<PX>(xx, x + offx, vec.Vh, i);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const cx<T> d = al * pp[c] + om * ss[c];
                xx[c] = {xx[c].re + (TX)d.re, xx[c].im + (TX)d.im};
            }
            store_spinor<PX>(x + offx, vec.Vh, i, xx);
        }
        cx<T> tt[12];
        load_spinor<P>(tt, t + off, vec.Vh, i);
#pragma unroll
        for (int c = 0; c < 12; ++c) ss[c] = ss[c] - om * tt[c];
        store_spinor<P>(r + off, vec.Vh, i, ss);
        // reduce on the stored (rounded) residual so rho matches what K_b reads
        cx<T> rn[12], hh[12];
        load_spinor<P>(rn, r + off, vec.Vh, i);
        load_spinor<P>(hh, rh + off, vec.Vh, i);
        T cr = 0, ci = 0, nn = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            cr = fma(hh[c].re, rn[c].re, fma(hh[c].im, rn[c].im, cr));
            ci = fma(hh[c].re, rn[c].im, fma(-hh[c].im, rn[c].re, ci));
            nn = fma(rn[c].re, rn[c].re, fma(rn[c].im, rn[c].im, nn));
        }
        part[0] = cr;
        part[1] = ci;
        part[2] = nn;
    }
    block_sum<3>(part, sh);
    double tot[3];
    if (grid_sum<3>(part, tot, red, rhs, gridDim.x, blockIdx.x, sh)) {
        S.rho_prev[0] = S.rr[0];
        S.rho_prev[1] = S.rr[1];
        S.alpha[0] = dcoef[0];
        S.alpha[1] = dcoef[1];
        S.omega[0] = dcoef[2];
        S.omega[1] = dcoef[3];
        S.rr[0] = tot[0];
        S.rr[1] = tot[1];
        S.rr[2] = tot[2];
        S.iters += 1;
        const bool stepped = (dcoef[0] != 0.0 || dcoef[1] != 0.0);
        const bool omega0 = (dcoef[2] == 0.0 && dcoef[3] == 0.0);
        if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
            S.flags |= FLAG_NAN;
            S.active = 0;
        } else if (tot[2] <= S.target2) {
            S.flags |= FLAG_CONVERGED;
            S.active = 0;
        } else if (!stepped || omega0) {
            S.flags |= FLAG_BREAKDOWN;
            S.active = 0;
        } else if (S.delta2 > 0.0) {
            if (tot[2] > S.r2_max) S.r2_max = tot[2];
            if (tot[2] < S.delta2 * S.r2_max) S.want_update = 1;
        }
    }
}

// Start (or restart) the scalars of the masked right-hand sides; rr holds
// (rhat, r) and ||r||^2 from a preceding cdot.
__global__ void init_scal_kernel(Scal* sc, const int* mask, int nrhs, int full)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs || !mask[k]) return;
    Scal& S = sc[k];
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

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

static Vec2 vec_of(wl_gauge g, int prec, int nhalf)
{
    Vec2 v;
    v.Vh = g->geo.Vh;
    v.nhalf = nhalf;
    v.hb = spinor_field_bytes(prec, g->geo.Vh);
    v.rstride = (long long)(v.hb * nhalf);
    return v;
}

static const int kBlock = 256;

template <typename F>
static int dispatch_prec(int prec, F&& f)
{
    switch (prec) {
        case WL_F64: return f(std::integral_constant<int, WL_F64>());
        case WL_F32: return f(std::integral_constant<int, WL_F32>());
        default: return f(std::integral_constant<int, WL_F16>());
    }
}


static int ws_alloc(void** p, size_t bytes)
{
    WL_CUDA(cudaMalloc(p, bytes));
    return WL_OK;
}

static int ensure_ws(wl_gauge g, int inner, int nrhs, int eo)
{
    Workspace* w = g->ws;
    if (w && w->inner == inner && w->nrhs >= nrhs && w->eo == eo) return WL_OK;
    WL_CUDA(cudaDeviceSynchronize());
    free_workspace(g);
    g->ws = new Workspace();
    w = g->ws;
    w->inner = inner;
    w->nrhs = nrhs;
    w->eo = eo;
    w->nhalf = eo ? 1 : 2;
    w->xlo_prec = inner == WL_F64 ? WL_F64 : WL_F32;
    const long long Vh = g->geo.Vh;
    w->vb = spinor_field_bytes(inner, Vh) * w->nhalf;
    w->hb64 = spinor_field_bytes(WL_F64, Vh);
    w->vb64 = w->hb64 * w->nhalf;
    const size_t n = (size_t)nrhs;
    void** inner_vecs[] = {&w->r, &w->rh, &w->p, &w->v, &w->s, &w->t};
    for (void** q : inner_vecs) WL_TRY(ws_alloc(q, w->vb * n));
    WL_TRY(ws_alloc(&w->xlo, spinor_field_bytes(w->xlo_prec, Vh) * w->nhalf * n));
    if (eo) WL_TRY(ws_alloc(&w->tmp, spinor_field_bytes(inner, Vh) * n));
    WL_TRY(ws_alloc((void**)&w->b64, 2 * w->hb64 * n));  // even | odd per rhs
    WL_TRY(ws_alloc((void**)&w->bp, w->vb64 * n));
    WL_TRY(ws_alloc((void**)&w->xhi, 2 * w->hb64 * n));  // full x (even | odd) per rhs
    WL_TRY(ws_alloc((void**)&w->rhi, 2 * w->hb64 * n));
    WL_TRY(ws_alloc((void**)&w->tmp64, w->hb64 * n));
    WL_TRY(ws_alloc((void**)&w->sc, sizeof(Scal) * n));
    WL_TRY(ws_alloc((void**)&w->mask, sizeof(int) * n));
    WL_TRY(ws_alloc((void**)&w->nrm, sizeof(double) * 3 * n));
    WL_CUDA(cudaMallocHost((void**)&w->sc_h, sizeof(Scal) * n));
    WL_CUDA(cudaMallocHost((void**)&w->mask_h, sizeof(int) * n));
    WL_CUDA(cudaMallocHost((void**)&w->nrm_h, sizeof(double) * 3 * n));
    WL_CUDA(cudaMemset(w->sc, 0, sizeof(Scal) * n));
    std::memset(w->sc_h, 0, sizeof(Scal) * n);
    // reduction scratch for every kernel the solve launches (no growth later,
    // so graph capture never needs to allocate)
    const long long hop_blocks = 2 * ((Vh + 127) / 128);
    const long long blas_blocks = (2 * Vh + kBlock - 1) / kBlock;
    WL_TRY(ensure_red(g, nrhs, hop_blocks > blas_blocks ? hop_blocks : blas_blocks));
    return WL_OK;
}

// stride between right-hand sides of the FP64 full fields (even | odd)
static long long full_rs(const Workspace* w) { return (long long)(2 * w->hb64); }

// A v (inner precision) with fused (w, out) and ||out||^2 into dot_out.
static int apply_A(wl_gauge g, Workspace* w, int prec, void* out, const void* in, const void* wdot,
                   double* dot_out, const int* active, int nrhs, cudaStream_t s)
{
    const size_t hb = spinor_field_bytes(prec, g->geo.Vh);
    if (w->eo) {
        HopLaunch h1;
        h1.prec = prec;
        h1.parity0 = 1;
        h1.nrhs = nrhs;
        h1.in[0] = in;
        h1.out[0] = w->tmp;
        h1.rs_in = h1.rs_out = (long long)hb;
        h1.active = active;
        h1.active_stride = kActiveStride;
        WL_TRY(launch_hop(g, h1, s));
        HopLaunch h2 = h1;
        h2.parity0 = 0;
        h2.in[0] = w->tmp;
        h2.out[0] = out;
        h2.x1[0] = in;
        h2.rs_x1 = (long long)hb;
        h2.a = -g->kappa * g->kappa;
        h2.w[0] = wdot;
        h2.rs_w = (long long)hb;
        h2.dot = true;
        h2.dot_out = dot_out;
        h2.dot_stride = kScalStride;
        return launch_hop(g, h2, s);
    }
    HopLaunch h;
    h.prec = prec;
    h.parity0 = 0;
    h.nparity = 2;
    h.nrhs = nrhs;
    h.in[0] = (const char*)in + hb;
    h.in[1] = in;
    h.out[0] = out;
    h.out[1] = (char*)out + hb;
    h.x1[0] = in;
    h.x1[1] = (const char*)in + hb;
    h.w[0] = wdot;
    h.w[1] = (const char*)wdot + hb;
    h.rs_in = h.rs_out = h.rs_x1 = h.rs_w = (long long)(2 * hb);
    h.a = -g->kappa;
    h.dot = true;
    h.dot_out = dot_out;
    h.dot_stride = kScalStride;
    h.active = active;
    h.active_stride = kActiveStride;
    return launch_hop(g, h, s);
}

static int enqueue_iteration(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s)
{
    const int P = w->inner;
    const Vec2 v = vec_of(g, P, w->nhalf);
    const Vec2 vx = vec_of(g, w->xlo_prec, w->nhalf);
    const dim3 grid((unsigned)((w->nhalf * g->geo.Vh + kBlock - 1) / kBlock), (unsigned)nrhs);
    const int* active = &w->sc[0].active;
    WL_TRY(dispatch_prec(P, [&](auto pc) -> int {
        constexpr int PP = decltype(pc)::value;
        update_p_kernel<PP><<<grid, kBlock, 0, s>>>((char*)w->p, (const char*)w->r,
                                                    (const char*)w->v, v, w->sc);
        WL_CHECK_LAUNCH(4.0 * w->vb * nrhs);
        return WL_OK;
    }));
    WL_TRY(apply_A(g, w, P, w->v, w->p, w->rh, w->sc[0].rv, active, nrhs, s));
    WL_TRY(dispatch_prec(P, [&](auto pc) -> int {
        constexpr int PP = decltype(pc)::value;
        update_s_kernel<PP><<<grid, kBlock, 0, s>>>((char*)w->s, (const char*)w->r,
                                                    (const char*)w->v, v, w->sc);
        WL_CHECK_LAUNCH(3.0 * w->vb * nrhs);
        return WL_OK;
    }));
    WL_TRY(apply_A(g, w, P, w->t, w->s, w->s, w->sc[0].st, active, nrhs, s));
    return dispatch_prec(P, [&](auto pc) -> int {
        constexpr int PP = decltype(pc)::value;
        if (w->xlo_prec == WL_F64)
            update_xr_kernel<PP, WL_F64><<<grid, kBlock, 0, s>>>(
                (char*)w->xlo, vx, (char*)w->r, (const char*)w->p, (const char*)w->s,
                (const char*)w->t, (const char*)w->rh, v, w->sc, g->red);
        else
            update_xr_kernel<PP, WL_F32><<<grid, kBlock, 0, s>>>(
                (char*)w->xlo, vx, (char*)w->r, (const char*)w->p, (const char*)w->s,
                (const char*)w->t, (const char*)w->rh, v, w->sc, g->red);
        // reads p, s, t, rhat and x; writes x and r
        WL_CHECK_LAUNCH((5.0 * w->vb + 2.0 * (double)vx.hb * w->nhalf) * nrhs);
        return WL_OK;
    });
}

// Run k iterations: a CUDA-graph replay when graph_k > 0, else eager launches.
static int run_chunk(wl_gauge g, Workspace* w, int nrhs, int k, bool use_graph, cudaStream_t s)
{
    if (!use_graph) {
        for (int it = 0; it < k; ++it) WL_TRY(enqueue_iteration(g, w, nrhs, s));
        return WL_OK;
    }
    if (!w->graph || w->graph_k != k || w->graph_nrhs != nrhs || w->graph_red_gen != g->red_gen) {
        if (w->graph) cudaGraphExecDestroy(w->graph);
        w->graph = nullptr;
        // capture on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the caller's stream
        if (!w->cap_stream) WL_CUDA(cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking));
        const long long c0 = g_launches.load(), b0 = g_bytes.load();
        WL_CUDA(cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = WL_OK;
        for (int it = 0; it < k && rc == WL_OK; ++it) rc = enqueue_iteration(g, w, nrhs, w->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(w->cap_stream, &graph);
        if (rc != WL_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return set_error(WL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        w->graph_kernels = g_launches.load() - c0;
        w->graph_bytes = g_bytes.load() - b0;
        g_launches.fetch_sub(w->graph_kernels);  // captured, not yet run
        g_bytes.fetch_sub(w->graph_bytes);
        e = cudaGraphInstantiate(&w->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return set_error(WL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        w->graph_k = k;
        w->graph_nrhs = nrhs;
        w->graph_red_gen = g->red_gen;
    }
    WL_CUDA(cudaGraphLaunch(w->graph, s));
    count_launch(w->graph_kernels, (double)w->graph_bytes);
    return WL_OK;
}

// r = b' - A x in FP64 for masked rhs, with ||r||^2 into w->nrm.
static int residual64(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s)
{
    const size_t hb = w->hb64;
    if (w->eo) {
        HopLaunch h1;
        h1.prec = WL_F64;
        h1.parity0 = 1;
        h1.nrhs = nrhs;
        h1.in[0] = w->xhi;
        h1.out[0] = w->tmp64;
        h1.rs_in = full_rs(w);
        h1.rs_out = (long long)hb;
        h1.active = w->mask;
        WL_TRY(launch_hop(g, h1, s));
        HopLaunch h2;
        h2.prec = WL_F64;
        h2.parity0 = 0;
        h2.nrhs = nrhs;
        h2.in[0] = w->tmp64;
        h2.out[0] = w->rhi;
        h2.x1[0] = w->bp;
        h2.x2[0] = w->xhi;
        h2.rs_in = (long long)hb;
        h2.rs_out = (long long)w->vb64;
        h2.rs_x1 = (long long)hb;
        h2.rs_x2 = full_rs(w);
        h2.b1 = -1.0;
        h2.a = g->kappa * g->kappa;
        h2.dot = true;
        h2.dot_out = w->nrm;
        h2.active = w->mask;
        return launch_hop(g, h2, s);
    }
    // full: r_p = b_p - x_p + kappa H x_{1-p}
    HopLaunch h;
    h.prec = WL_F64;
    h.parity0 = 0;
    h.nparity = 2;
    h.nrhs = nrhs;
    h.in[0] = (const char*)w->xhi + hb;
    h.in[1] = w->xhi;
    h.out[0] = w->rhi;
    h.out[1] = (char*)w->rhi + hb;
    h.x1[0] = w->bp;
    h.x1[1] = (const char*)w->bp + hb;
    h.x2[0] = w->xhi;
    h.x2[1] = (const char*)w->xhi + hb;
    h.rs_in = h.rs_out = h.rs_x1 = h.rs_x2 = full_rs(w);
    h.b1 = -1.0;
    h.a = g->kappa;
    h.dot = true;
    h.dot_out = w->nrm;
    h.active = w->mask;
    return launch_hop(g, h, s);
}

// r_full = b - D x on the full lattice (FP64) with ||r||^2 into w->nrm.
static int true_residual64(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s)
{
    const size_t hb = w->hb64;
    HopLaunch h;
    h.prec = WL_F64;
    h.parity0 = 0;
    h.nparity = 2;
    h.nrhs = nrhs;
    h.in[0] = (const char*)w->xhi + hb;
    h.in[1] = w->xhi;
    h.out[0] = w->rhi;
    h.out[1] = (char*)w->rhi + hb;
    h.x1[0] = w->b64;
    h.x1[1] = (const char*)w->b64 + hb;
    h.x2[0] = w->xhi;
    h.x2[1] = (const char*)w->xhi + hb;
    h.rs_in = h.rs_out = h.rs_x1 = h.rs_x2 = full_rs(w);
    h.b1 = -1.0;
    h.a = g->kappa;
    h.dot = true;
    h.dot_out = w->nrm;
    return launch_hop(g, h, s);
}

static int upload_mask(Workspace* w, int nrhs, cudaStream_t s)
{
    WL_CUDA(cudaMemcpyAsync(w->mask, w->mask_h, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
    return WL_OK;
}

static int read_norms(Workspace* w, int nrhs, cudaStream_t s)
{
    WL_CUDA(cudaMemcpyAsync(w->nrm_h, w->nrm, sizeof(double) * 3 * nrhs, cudaMemcpyDeviceToHost, s));
    WL_CUDA(cudaStreamSynchronize(s));
    return WL_OK;
}

// Begin an inner solve for the masked rhs: r = r_hi (converted), rhat = r,
// p = v = x_lo = 0, fresh scalars with the given targets.
static int inner_start(wl_gauge g, Workspace* w, int nrhs, const double* target2,
                       double delta2, cudaStream_t s)
{
    const int P = w->inner;
    for (int k = 0; k < nrhs; ++k) {
        Scal& S = w->sc_h[k];
        if (!w->mask_h[k]) {
            S.active = 0;
            continue;
        }
        S.target2 = target2[k];
        S.delta2 = delta2;
        S.flags = 0;
        S.want_update = 0;
        S.active = 0;
    }
    // push host-side fields of all rhs (device-side fields of unmasked rhs
    // are not touched by the masked kernels below, and the host copy of
    // them is current after the last read-back)
    WL_CUDA(cudaMemcpyAsync(w->sc, w->sc_h, sizeof(Scal) * nrhs, cudaMemcpyHostToDevice, s));
    WL_TRY(upload_mask(w, nrhs, s));
    WL_TRY(launch_convert(g, P, w->r, WL_F64, w->rhi, w->nhalf, nrhs, w->mask, s));
    WL_TRY(launch_convert(g, P, w->rh, P, w->r, w->nhalf, nrhs, w->mask, s));
    WL_TRY(launch_zero(g, P, w->p, w->nhalf, nrhs, w->mask, s));
    WL_TRY(launch_zero(g, P, w->v, w->nhalf, nrhs, w->mask, s));
    WL_TRY(launch_zero(g, w->xlo_prec, w->xlo, w->nhalf, nrhs, w->mask, s));
    WL_TRY(launch_cdot(g, P, w->rh, w->r, w->nhalf, nrhs, w->sc[0].rr, kScalStride, w->mask, s));
    init_scal_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(w->sc, w->mask, nrhs, 1);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

// Reliable update for the masked rhs: x_hi += x_lo, x_lo = 0, r_hi = b' - A x_hi,
// r = r_hi; the Krylov directions and rhat are kept.
static int reliable_update(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s)
{
    const int P = w->inner;
    WL_TRY(upload_mask(w, nrhs, s));
    WL_TRY(launch_accum_hi(g, w->xhi, w->xlo_prec, w->xlo, w->nhalf, nrhs, w->mask, s, full_rs(w)));
    WL_TRY(launch_zero(g, w->xlo_prec, w->xlo, w->nhalf, nrhs, w->mask, s));
    WL_TRY(residual64(g, w, nrhs, s));
    WL_TRY(launch_convert(g, P, w->r, WL_F64, w->rhi, w->nhalf, nrhs, w->mask, s));
    WL_TRY(launch_cdot(g, P, w->rh, w->r, w->nhalf, nrhs, w->sc[0].rr, kScalStride, w->mask, s));
    init_scal_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(w->sc, w->mask, nrhs, 0);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

}  // namespace wl

using namespace wl;

static bool is_host_pointer(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

extern "C" int wilson_solve(wl_gauge g, double* x, const double* b, int nrhs,
                            const wl_solve_params* prm, wl_solve_info* info, void* stream)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (!x || !b || !prm || !info) return set_error(WL_ERR_ARG, "NULL pointer");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    if (prm->inner < WL_F64 || prm->inner > WL_F16) return set_error(WL_ERR_ARG, "unknown inner precision");
    if (!(prm->tol > 0.0)) return set_error(WL_ERR_ARG, "tol must be > 0");
    if (prm->maxiter < 1) return set_error(WL_ERR_ARG, "maxiter must be >= 1");
    if (!g->links[prm->inner][0])
        return set_error(WL_ERR_STATE, "gauge object was created without the inner precision");
    cudaStream_t s = (cudaStream_t)stream;
    const int eo = prm->eo ? 1 : 0;
    const int P = prm->inner;
    WL_TRY(ensure_ws(g, P, nrhs, eo));
    Workspace* w = g->ws;
    const long long V = 2 * g->geo.Vh;
    const size_t canon = (size_t)V * 24 * sizeof(double) * nrhs;

    // host buffers are staged through the workspace
    const bool host_b = is_host_pointer(b), host_x = is_host_pointer(x);
    const double* bd = b;
    double* xd = x;
    if (host_b || host_x) {
        if (w->stage_bytes < canon) {
            if (w->stage_b) cudaFree(w->stage_b);
            if (w->stage_x) cudaFree(w->stage_x);
            w->stage_b = w->stage_x = nullptr;
            w->stage_bytes = 0;
            WL_CUDA(cudaMalloc((void**)&w->stage_b, canon));
            WL_CUDA(cudaMalloc((void**)&w->stage_x, canon));
            w->stage_bytes = canon;
        }
        if (host_b) {
            WL_CUDA(cudaMemcpyAsync(w->stage_b, b, canon, cudaMemcpyHostToDevice, s));
            bd = w->stage_b;
        }
        if (host_x) {
            if (prm->use_x0) WL_CUDA(cudaMemcpyAsync(w->stage_x, x, canon, cudaMemcpyHostToDevice, s));
            xd = w->stage_x;
        }
    }

    const size_t hb64 = w->hb64;
    const int nh = w->nhalf;
    // b -> internal FP64 (even | odd per rhs); the conversion writes with the
    // rhs stride of one half field, so convert each rhs separately
    for (int r = 0; r < nrhs; ++r) {
        char* dst = (char*)w->b64 + r * 2 * hb64;
        const double* src = bd + (size_t)r * V * 24;
        WL_TRY(wl_field_to_internal(g, dst, src, 0, WL_F64, 1, s));
        WL_TRY(wl_field_to_internal(g, dst + hb64, src, 1, WL_F64, 1, s));
        if (prm->use_x0) {
            char* xdst = (char*)w->xhi + r * 2 * hb64;
            const double* xs = xd + (size_t)r * V * 24;
            WL_TRY(wl_field_to_internal(g, xdst, xs, 0, WL_F64, 1, s));
            WL_TRY(wl_field_to_internal(g, xdst + hb64, xs, 1, WL_F64, 1, s));
        }
    }
    if (!prm->use_x0) WL_CUDA(cudaMemsetAsync(w->xhi, 0, 2 * hb64 * nrhs, s));
    // ||b||^2 over the full lattice
    for (int k = 0; k < nrhs; ++k) w->mask_h[k] = 1;
    WL_TRY(upload_mask(w, nrhs, s));
    WL_TRY(launch_cdot(g, WL_F64, w->b64, w->b64, 2, nrhs, w->nrm, 3, nullptr, s));
    WL_TRY(read_norms(w, nrhs, s));
    std::vector<double> bnorm2(nrhs), rnorm2(nrhs), target2(nrhs);
    for (int k = 0; k < nrhs; ++k) bnorm2[k] = w->nrm_h[3 * k + 2];
    // b' = b_e + kappa H_eo b_o (even-odd) or b (full)
    if (eo) {
        HopLaunch h;
        h.prec = WL_F64;
        h.parity0 = 0;
        h.nrhs = nrhs;
        h.in[0] = (const char*)w->b64 + hb64;
        h.out[0] = w->bp;
        h.x1[0] = w->b64;
        h.rs_in = h.rs_x1 = full_rs(w);
        h.rs_out = (long long)hb64;
        h.a = g->kappa;
        WL_TRY(launch_hop(g, h, s));
    } else {
        WL_CUDA(cudaMemcpyAsync(w->bp, w->b64, 2 * hb64 * nrhs, cudaMemcpyDeviceToDevice, s));
    }
    // state per rhs
    std::vector<int> done(nrhs, 0), status(nrhs, WL_OK), outer(nrhs, 0), restarts(nrhs, 0);
    for (int k = 0; k < nrhs; ++k) {
        if (bnorm2[k] == 0.0) done[k] = 1;  // x = 0 solves b = 0 exactly
        w->sc_h[k] = Scal();
        std::memset(&w->sc_h[k], 0, sizeof(Scal));
    }
    WL_CUDA(cudaMemcpyAsync(w->sc, w->sc_h, sizeof(Scal) * nrhs, cudaMemcpyHostToDevice, s));
    for (int k = 0; k < nrhs; ++k) w->mask_h[k] = done[k] ? 0 : 1;
    WL_TRY(upload_mask(w, nrhs, s));
    if (prm->use_x0) {
        WL_TRY(residual64(g, w, nrhs, s));
    } else {  // x = 0: r = b' exactly, no FP64 matrix apply needed
        WL_CUDA(cudaMemcpy2DAsync(w->rhi, w->vb64, w->bp, w->vb64, w->vb64, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
        WL_TRY(launch_cdot(g, WL_F64, w->bp, w->bp, w->nhalf, nrhs, w->nrm, 3, w->mask, s));
    }
    WL_TRY(read_norms(w, nrhs, s));
    for (int k = 0; k < nrhs; ++k) rnorm2[k] = w->mask_h[k] ? w->nrm_h[3 * k + 2] : 0.0;

    const double delta2 = prm->delta > 0.0 ? prm->delta * prm->delta : 0.0;
    const double inner_tol =
        prm->inner_tol > 0.0 ? prm->inner_tol : (P == WL_F64 ? 0.0 : P == WL_F32 ? 1e-5 : 1e-3);
    const int chunk = prm->graph_iters > 0 ? prm->graph_iters
                      : prm->graph_iters < 0 ? -prm->graph_iters : 4;
    const bool use_graph = prm->graph_iters > 0;
    double safety = 0.5;  // aim below tol on the Schur residual; tightened if the true residual misses
    int final_rounds = 0;

    for (;;) {
        // ---------------- outer loop: FP64 residual -> inner solve -> FP64 update
        for (;;) {
            int any = 0;
            for (int k = 0; k < nrhs; ++k) {
                if (done[k]) { w->mask_h[k] = 0; continue; }
                const double goal2 = safety * safety * prm->tol * prm->tol * bnorm2[k];
                if (rnorm2[k] <= goal2) { done[k] = 1; w->mask_h[k] = 0; continue; }
                if (!std::isfinite(rnorm2[k])) { done[k] = 1; status[k] = WL_ERR_NAN; w->mask_h[k] = 0; continue; }
                if (w->sc_h[k].iters >= prm->maxiter) { done[k] = 1; status[k] = WL_ERR_NOT_CONVERGED; w->mask_h[k] = 0; continue; }
                w->mask_h[k] = 1;
                any = 1;
                double t2 = inner_tol * inner_tol * rnorm2[k];
                if (delta2 > 0.0 || t2 < goal2) t2 = goal2;
                target2[k] = t2;
            }
            if (!any) break;
            std::vector<int> iters_before(nrhs);
            for (int k = 0; k < nrhs; ++k) iters_before[k] = w->sc_h[k].iters;
            WL_TRY(inner_start(g, w, nrhs, target2.data(), delta2, s));
            std::vector<int> part(w->mask_h, w->mask_h + nrhs);  // took part in this round
            std::vector<int> in_inner(part), poisoned(nrhs, 0);
            for (;;) {
                int most = 0;  // iterations done by the furthest-along active rhs
                for (int k = 0; k < nrhs; ++k)
                    if (in_inner[k] && w->sc_h[k].iters > most) most = w->sc_h[k].iters;
                const int k_run = chunk < prm->maxiter - most ? chunk : prm->maxiter - most;
                if (k_run <= 0) break;
                WL_TRY(run_chunk(g, w, nrhs, k_run, use_graph && k_run == chunk, s));
                WL_CUDA(cudaMemcpyAsync(w->sc_h, w->sc, sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, s));
                WL_CUDA(cudaStreamSynchronize(s));
                int upd = 0, stopped = 0;
                for (int k = 0; k < nrhs; ++k) {
                    w->mask_h[k] = 0;
                    if (!in_inner[k]) continue;
                    Scal& S = w->sc_h[k];
                    if (S.active && S.iters >= prm->maxiter) {
                        S.active = 0;  // pushed to the device below
                        S.flags |= FLAG_MAXITER;
                        stopped = 1;
                    }
                    if (S.active) {
                        if (S.want_update) { w->mask_h[k] = 1; upd = 1; }
                        continue;
                    }
                    in_inner[k] = 0;  // converged, out of iterations, or broke down
                    if (S.flags & (FLAG_BREAKDOWN | FLAG_NAN)) {
                        if (S.flags & FLAG_NAN) poisoned[k] = 1;
                        if (++restarts[k] > 5) {
                            done[k] = 1;
                            status[k] = (S.flags & FLAG_NAN) ? WL_ERR_NAN : WL_ERR_BREAKDOWN;
                        }
                    }
                }
                if (stopped)
                    WL_CUDA(cudaMemcpyAsync(w->sc, w->sc_h, sizeof(Scal) * nrhs, cudaMemcpyHostToDevice, s));
                if (upd) {
                    WL_TRY(reliable_update(g, w, nrhs, s));
                    for (int k = 0; k < nrhs; ++k) if (w->mask_h[k]) outer[k]++;
                    // refresh the host copy so later pushes keep the new scalars
                    WL_CUDA(cudaMemcpyAsync(w->sc_h, w->sc, sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, s));
                    WL_CUDA(cudaStreamSynchronize(s));
                }
                bool alive = false;
                for (int k = 0; k < nrhs; ++k) alive |= in_inner[k] != 0;
                if (!alive) break;
            }
            // x_hi += x_lo; r_hi = b' - A x_hi for every rhs that took part
            int any_poison = 0;
            for (int k = 0; k < nrhs; ++k) {
                w->mask_h[k] = poisoned[k];
                any_poison |= poisoned[k];
            }
            if (any_poison) {  // a NaN correction is dropped, not accumulated
                WL_TRY(upload_mask(w, nrhs, s));
                WL_TRY(launch_zero(g, w->xlo_prec, w->xlo, nh, nrhs, w->mask, s));
            }
            for (int k = 0; k < nrhs; ++k) w->mask_h[k] = part[k];
            WL_TRY(upload_mask(w, nrhs, s));
            WL_TRY(launch_accum_hi(g, w->xhi, w->xlo_prec, w->xlo, nh, nrhs, w->mask, s, full_rs(w)));
            WL_TRY(residual64(g, w, nrhs, s));
            WL_TRY(read_norms(w, nrhs, s));
            for (int k = 0; k < nrhs; ++k)
                if (part[k]) {
                    rnorm2[k] = w->nrm_h[3 * k + 2];
                    outer[k]++;
                    // an inner solve that could not move (its start already met the
                    // inner target) ends the outer loop; the true residual decides
                    if (w->sc_h[k].iters == iters_before[k] && !done[k]) done[k] = 1;
                    if (outer[k] > kMaxOuter && !done[k]) {
                        done[k] = 1;
                        status[k] = WL_ERR_NOT_CONVERGED;
                    }
                }
        }
        // ---------------- reconstruct the odd half and check the true residual
        if (eo) {
            HopLaunch h;
            h.prec = WL_F64;
            h.parity0 = 1;
            h.nrhs = nrhs;
            h.in[0] = w->xhi;
            h.out[0] = (char*)w->xhi + hb64;
            h.x1[0] = (const char*)w->b64 + hb64;
            h.rs_in = h.rs_out = h.rs_x1 = full_rs(w);
            h.a = g->kappa;
            WL_TRY(launch_hop(g, h, s));
        }
        WL_TRY(true_residual64(g, w, nrhs, s));
        WL_TRY(read_norms(w, nrhs, s));
        bool retry = false;
        for (int k = 0; k < nrhs; ++k) {
            const double tr = bnorm2[k] > 0 ? std::sqrt(w->nrm_h[3 * k + 2] / bnorm2[k]) : 0.0;
            info[k].true_resid = tr;
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
        // the Schur residual met the goal but the full one did not: aim lower
        ++final_rounds;
        safety *= 0.1;
        for (int k = 0; k < nrhs; ++k) w->mask_h[k] = done[k] ? 0 : 1;
        WL_TRY(upload_mask(w, nrhs, s));
        WL_TRY(residual64(g, w, nrhs, s));
        WL_TRY(read_norms(w, nrhs, s));
        for (int k = 0; k < nrhs; ++k) if (w->mask_h[k]) rnorm2[k] = w->nrm_h[3 * k + 2];
    }
    // x -> canonical
    for (int r = 0; r < nrhs; ++r) {
        const char* src = (const char*)w->xhi + r * 2 * hb64;
        double* dst = xd + (size_t)r * V * 24;
        WL_TRY(wl_field_to_canonical(g, dst, src, 0, WL_F64, 1, s));
        WL_TRY(wl_field_to_canonical(g, dst, src + hb64, 1, WL_F64, 1, s));
    }
    if (host_x) WL_CUDA(cudaMemcpyAsync(x, xd, canon, cudaMemcpyDeviceToHost, s));
    WL_CUDA(cudaStreamSynchronize(s));
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int rc = WL_OK;
    for (int k = 0; k < nrhs; ++k) {
        info[k].iters = w->sc_h[k].iters;
        info[k].outer = outer[k];
        info[k].restarts = restarts[k];
        info[k].status = status[k];
        info[k].secs = secs;
        if (status[k] != WL_OK && rc == WL_OK) rc = status[k];
    }
    if (rc != WL_OK) set_error(rc, "at least one right-hand side did not reach tol");
    return rc;
}

extern "C" int wilson_solve_batch(int nlat, const wl_gauge* gs, double* const* x,
                                  const double* const* b, const int* nrhs,
                                  const wl_solve_params* p, wl_solve_info* info, void* stream)
{
    if (nlat < 1 || !gs || !x || !b || !nrhs || !p || !info)
        return set_error(WL_ERR_ARG, "bad batch arguments");
    int rc = WL_OK, off = 0;
    for (int l = 0; l < nlat; ++l) {
        const int r = wilson_solve(gs[l], x[l], b[l], nrhs[l], p, info + off, stream);
        if (r != WL_OK && rc == WL_OK) rc = r;
        if (r == WL_ERR_ARG || r == WL_ERR_CUDA || r == WL_ERR_STATE) return r;
        off += nrhs[l];
    }
    return rc;
}
