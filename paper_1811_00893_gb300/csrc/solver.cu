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
// Convergence is always decided on the FP64 true residual of the full D.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "hop.cuh"
#include "solver.cuh"

namespace wl {

// Per-round log of the outer loop on stderr when WL_SOLVE_VERBOSE is set
// (diagnostics only; one line per event and right-hand side).
static bool solve_verbose()
{
    static const bool on = getenv("WL_SOLVE_VERBOSE") != nullptr;
    return on;
}


static void free_ws(Workspace* w)
{
    if (!w) return;
    void* dev[] = {w->r, w->rh, w->p, w->v, w->s, w->t, w->xlo, w->tmp, w->b64, w->bp, w->xhi,
                   w->rhi, w->tmp64, w->sc, w->mask, w->nrm, w->stage_b, w->stage_x,
                   w->bout == w->b64 ? nullptr : w->bout, w->x64 == w->xhi ? nullptr : w->x64};
    for (void* q : dev)
        if (q) cudaFree(q);
    if (w->sc_h) cudaFreeHost(w->sc_h);
    if (w->mask_h) cudaFreeHost(w->mask_h);
    if (w->nrm_h) cudaFreeHost(w->nrm_h);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
    if (w->aux) cudaStreamDestroy(w->aux);
    if (w->ev_x) cudaEventDestroy(w->ev_x);
    if (w->ev_sent) cudaEventDestroy(w->ev_sent);
    if (w->lane) cudaStreamDestroy(w->lane);
    if (w->ev_lane) cudaEventDestroy(w->ev_lane);
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
// device kernels (single lattice; one right-hand side per grid row)
// ---------------------------------------------------------------------------

struct Vec2 {
    long long Vh;
    int nhalf;
    size_t hb;
    long long rstride;
};

// Half and site of element j.  A vector has one half (even-odd) or two (full
// lattice), so the half is a comparison, not a 64-bit division.
__device__ __forceinline__ long long split_index(const Vec2& v, long long j, long long& off)
{
    const int h = j >= v.Vh ? 1 : 0;
    off = h * (long long)v.hb;
    return j - h * v.Vh;
}

template <int P>
__global__ void __launch_bounds__(256) update_p_kernel(char* p, const char* r, const char* v,
                                                       Vec2 vec, const Scal* sc)
{
    const int rhs = blockIdx.y;
    const Scal& S = sc[rhs];
    if (!S.active) return;
    __shared__ double coef[4];
    if (threadIdx.x == 0) {
        double c[4];
        beta_omega(S, c);
        for (int k = 0; k < 4; ++k) coef[k] = c[k];
    }
    __syncthreads();
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= vec.nhalf * vec.Vh) return;
    long long off;
    const long long i = split_index(vec, j, off);
    off += rhs * vec.rstride;
    const double c[4] = {coef[0], coef[1], coef[2], coef[3]};
    p_update_site<P>(p + off, r + off, v + off, vec.Vh, i, c);
}

template <int P>
__global__ void __launch_bounds__(256) update_s_kernel(char* s, const char* r, const char* v,
                                                       Vec2 vec, const Scal* sc)
{
    const int rhs = blockIdx.y;
    const Scal& S = sc[rhs];
    if (!S.active) return;
    __shared__ double coef[2];
    if (threadIdx.x == 0) {
        const cx<double> al = safe_alpha(S);
        coef[0] = al.re;
        coef[1] = al.im;
    }
    __syncthreads();
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= vec.nhalf * vec.Vh) return;
    long long off;
    const long long i = split_index(vec, j, off);
    off += rhs * vec.rstride;
    s_update_site<P>(s + off, r + off, v + off, vec.Vh, i, {coef[0], coef[1]});
}

template <int P, int PX>
__global__ void __launch_bounds__(256) update_xr_kernel(char* x, Vec2 vx, char* r, const char* p,
                                                        const char* s, const char* t,
                                                        const char* rh, Vec2 vec, Scal* sc,
                                                        RedScratch red)
{
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
    using T = typename Prec<P>::real;
    const double dc[4] = {dcoef[0], dcoef[1], dcoef[2], dcoef[3]};
    T tpart[3] = {0, 0, 0};  // this thread's sites in the kernel's arithmetic
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < vec.nhalf * vec.Vh;
         j += (long long)gridDim.x * blockDim.x) {
        long long off, offx;
        const long long i = split_index(vec, j, off);
        split_index(vx, j, offx);
        off += rhs * vec.rstride;
        offx += rhs * vx.rstride;
        T pt[3];
        xr_update_site<P, PX>(x + offx, r + off, p + off, s + off, t + off, rh + off, vec.Vh, i,
                              dc, pt);
        for (int k = 0; k < 3; ++k) tpart[k] += pt[k];
    }
    typename RedType<T>::type wp[3] = {(typename RedType<T>::type)tpart[0],
                                       (typename RedType<T>::type)tpart[1],
                                       (typename RedType<T>::type)tpart[2]};
    warp_sum<3>(wp);  // warp totals in the arithmetic type, FP64 from there
    double part[3] = {(double)wp[0], (double)wp[1], (double)wp[2]};
    block_sum_warps<3>(part, sh);
    double tot[3];
    if (grid_sum<3>(part, tot, red, rhs, gridDim.x, blockIdx.x, sh)) advance_scalars(S, tot, dc);
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

static Vec2 vec_of(wl_gauge g, int prec, int nhalf)  // nhalf is 1 or 2
{
    Vec2 v;
    v.Vh = g->geo.Vh;
    v.nhalf = nhalf;
    v.hb = spinor_field_bytes(prec, g->geo.Vh);
    v.rstride = (long long)(v.hb * nhalf);
    return v;
}

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

int ensure_ws(wl_gauge g, int inner, int nrhs, int eo)
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
    // outer residual corrections of mixed-precision solves in df64 (FP32-rate
    // arithmetic, ~2^-44 rounding); the plain FP64 solve stays in FP64
    w->outer = inner == WL_F64 ? WL_F64 : WL_DF64;
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
    if (w->outer == WL_F64) {
        w->bout = w->b64;
        w->x64 = w->xhi;
    } else {
        WL_TRY(ws_alloc((void**)&w->bout, 2 * w->hb64 * n));
        WL_TRY(ws_alloc((void**)&w->x64, 2 * w->hb64 * n));
    }
    WL_TRY(ws_alloc((void**)&w->sc, sizeof(Scal) * n));
    WL_TRY(ws_alloc((void**)&w->mask, sizeof(int) * n));
    WL_TRY(ws_alloc((void**)&w->nrm, sizeof(double) * 6 * n));
    WL_CUDA(cudaMallocHost((void**)&w->sc_h, sizeof(Scal) * n));
    WL_CUDA(cudaMallocHost((void**)&w->mask_h, sizeof(int) * n));
    WL_CUDA(cudaMallocHost((void**)&w->nrm_h, sizeof(double) * 6 * n));
    WL_CUDA(cudaMemset(w->sc, 0, sizeof(Scal) * n));
    std::memset(w->sc_h, 0, sizeof(Scal) * n);
    // reduction scratch for every kernel the solve launches (no growth later,
    // so graph capture never needs to allocate)
    const long long hop_blocks = 2 * ((Vh + 31) / 32);  // smallest hop tile: 32 sites
    const long long blas_blocks = (2 * Vh + kBlock - 1) / kBlock;
    WL_TRY(ensure_red(g, nrhs, hop_blocks > blas_blocks ? hop_blocks : blas_blocks));
    return WL_OK;
}


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
        if (g->has_clover) {  // tmp = A_oo^-1 H_oe in
            h1.cl_mode = kClOut;
            h1.clov[0] = g->clov[prec][1][1];
        }
        WL_TRY(launch_hop(g, h1, s));
        HopLaunch h2 = h1;
        h2.parity0 = 0;
        h2.in[0] = w->tmp;
        h2.out[0] = out;
        h2.a = -g->kappa * g->kappa;
        if (g->has_clover) {  // out = A_ee in - kappa^2 H_eo tmp
            h2.x2[0] = in;
            h2.rs_x2 = (long long)hb;
            h2.b1 = 1.0;
            h2.cl_mode = kClX2;
            h2.clov[0] = g->clov[prec][0][0];
        } else {
            h2.x1[0] = in;
            h2.rs_x1 = (long long)hb;
            h2.cl_mode = kClNone;
        }
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
    h.w[0] = wdot;
    h.w[1] = (const char*)wdot + hb;
    h.rs_in = h.rs_out = h.rs_w = (long long)(2 * hb);
    h.a = -g->kappa;
    if (g->has_clover) {  // out_p = A_pp in_p - kappa H in_{1-p}
        h.x2[0] = in;
        h.x2[1] = (const char*)in + hb;
        h.rs_x2 = (long long)(2 * hb);
        h.b1 = 1.0;
        h.cl_mode = kClX2;
        h.clov[0] = g->clov[prec][0][0];
        h.clov[1] = g->clov[prec][1][0];
    } else {
        h.x1[0] = in;
        h.x1[1] = (const char*)in + hb;
        h.rs_x1 = (long long)(2 * hb);
    }
    h.dot = true;
    h.dot_out = dot_out;
    h.dot_stride = kScalStride;
    h.active = active;
    h.active_stride = kActiveStride;
    return launch_hop(g, h, s);
}

// Threads per block of the per-iteration vector kernels over n elements: 256,
// or fewer on small lattices, so that the grid still reaches every SM (an 8^4
// FP64 solve's updates are bound by the FP64 pipes of the SMs they run on).
static int vec_block(long long n, int sms)
{
    int b = kBlock;
    while (b > 32 && (n + b - 1) / b < 2LL * sms) b >>= 1;
    return b;
}

static int enqueue_iteration(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s)
{
    const int P = w->inner;
    const Vec2 v = vec_of(g, P, w->nhalf);
    const Vec2 vx = vec_of(g, w->xlo_prec, w->nhalf);
    const int vb = vec_block(w->nhalf * g->geo.Vh, g->num_sms);
    const dim3 grid((unsigned)((w->nhalf * g->geo.Vh + vb - 1) / vb), (unsigned)nrhs);
    const int* active = &w->sc[0].active;
    WL_TRY(dispatch_prec(P, [&](auto pc) -> int {
        constexpr int PP = decltype(pc)::value;
        update_p_kernel<PP><<<grid, vb, 0, s>>>((char*)w->p, (const char*)w->r,
                                                    (const char*)w->v, v, w->sc);
        WL_CHECK_LAUNCH(4.0 * w->vb * nrhs);
        return WL_OK;
    }));
    WL_TRY(apply_A(g, w, P, w->v, w->p, w->rh, w->sc[0].rv, active, nrhs, s));
    WL_TRY(dispatch_prec(P, [&](auto pc) -> int {
        constexpr int PP = decltype(pc)::value;
        update_s_kernel<PP><<<grid, vb, 0, s>>>((char*)w->s, (const char*)w->r,
                                                    (const char*)w->v, v, w->sc);
        WL_CHECK_LAUNCH(3.0 * w->vb * nrhs);
        return WL_OK;
    }));
    WL_TRY(apply_A(g, w, P, w->t, w->s, w->s, w->sc[0].st, active, nrhs, s));
    return dispatch_prec(P, [&](auto pc) -> int {
        constexpr int PP = decltype(pc)::value;
        // grid of resident blocks: the fused reduction leaves few partials
        dim3 rgrid = grid;
        rgrid.x = std::min(grid.x, (unsigned)resident_grid(
                                       w->xlo_prec == WL_F64 ? (const void*)update_xr_kernel<PP, WL_F64>
                                                             : (const void*)update_xr_kernel<PP, WL_F32>,
                                       vb, 0));
        if (w->xlo_prec == WL_F64)
            update_xr_kernel<PP, WL_F64><<<rgrid, vb, 0, s>>>(
                (char*)w->xlo, vx, (char*)w->r, (const char*)w->p, (const char*)w->s,
                (const char*)w->t, (const char*)w->rh, v, w->sc, g->red);
        else
            update_xr_kernel<PP, WL_F32><<<rgrid, vb, 0, s>>>(
                (char*)w->xlo, vx, (char*)w->r, (const char*)w->p, (const char*)w->s,
                (const char*)w->t, (const char*)w->rh, v, w->sc, g->red);
        // reads p, s, t, rhat and x; writes x and r
        WL_CHECK_LAUNCH((5.0 * w->vb + 2.0 * (double)vx.hb * w->nhalf) * nrhs);
        return WL_OK;
    });
}

// Run k iterations: a CUDA-graph replay when graph_k > 0, else eager launches.
static int run_chunk_impl(wl_gauge g, Workspace* w, int nrhs, int k, bool use_graph, cudaStream_t s);

// Run k iterations and remember what they were charged (see discount_chunk).
// The autotuner cannot time launches inside a stream capture, so before the
// first captured chunk for this many right-hand sides v = M p is applied once
// outside it, which times the iteration's hopping launches.  At a chunk
// boundary v = M p already holds (p = v = 0 at a round's start), and the
// per-site results do not depend on the launch shape, so v keeps its value;
// tmp and the dot product are recomputed before they are read.  The launches
// are tuning, not solve work: they leave the counters and timing records as
// they were.  (Eager chunks tune their launches themselves.)
static int tune_iteration(wl_gauge g, Workspace* w, int nrhs, bool use_graph, cudaStream_t s)
{
    if (w->tuned_nrhs == nrhs) return WL_OK;
    if (use_graph) {
        const long long c0 = g_launches.load(), b0 = g_bytes.load();
        const bool timed = g->timing.on;
        g->timing.on = false;
        const int rc = apply_A(g, w, w->inner, w->v, w->p, w->rh, w->sc[0].rv, nullptr, nrhs, s);
        g->timing.on = timed;
        g_launches.fetch_sub(g_launches.load() - c0);
        g_bytes.fetch_sub(g_bytes.load() - b0);
        WL_TRY(rc);
    }
    w->tuned_nrhs = nrhs;
    return WL_OK;
}

int run_chunk(wl_gauge g, Workspace* w, int nrhs, int k, bool use_graph, cudaStream_t s)
{
    WL_TRY(tune_iteration(g, w, nrhs, use_graph, s));
    const long long b0 = g_bytes.load();
    w->chunk_slot0 = g->timing.used;
    const int rc = run_chunk_impl(g, w, nrhs, k, use_graph, s);
    w->chunk_k = rc == WL_OK ? k : 0;
    w->chunk_bytes = g_bytes.load() - b0;
    w->chunk_slot1 = g->timing.used;
    return rc;
}

// The last `skipped` iterations of the last chunk ran after every right-hand
// side had stopped: their launches exited at once.  Take them out of the
// algorithmic-byte counter and out of the per-launch timing records, so that
// both describe the work done.
void discount_chunk(wl_gauge g, Workspace* w, int skipped)
{
    if (skipped <= 0 || w->chunk_k <= 0) return;
    if (skipped > w->chunk_k) skipped = w->chunk_k;
    g_bytes.fetch_sub(w->chunk_bytes / w->chunk_k * skipped);
    const size_t slots = w->chunk_slot1 - w->chunk_slot0;  // this chunk's timed launches
    if (slots % (size_t)w->chunk_k == 0) {
        const size_t per_iter = slots / (size_t)w->chunk_k;
        for (size_t q = w->chunk_slot1 - per_iter * skipped; q < w->chunk_slot1; ++q)
            g->timing.bytes[q] = -1.0;  // excluded by wl_timing_read
    }
    w->chunk_k = 0;
}

static int run_chunk_impl(wl_gauge g, Workspace* w, int nrhs, int k, bool use_graph, cudaStream_t s)
{
    if (!use_graph) {
        for (int it = 0; it < k; ++it) WL_TRY(enqueue_iteration(g, w, nrhs, s));
        return WL_OK;
    }
    const bool timed = g->timing.on;
    if (!w->graph || w->graph_k != k || w->graph_nrhs != nrhs || w->graph_red_gen != g->red_gen ||
        w->graph_timed != timed) {
        if (w->graph) cudaGraphExecDestroy(w->graph);
        w->graph = nullptr;
        // capture on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the caller's stream
        if (!w->cap_stream) WL_CUDA(cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking));
        const long long c0 = g_launches.load(), b0 = g_bytes.load();
        timing_capture_begin(g);
        WL_CUDA(cudaStreamBeginCapture(w->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = WL_OK;
        for (int it = 0; it < k && rc == WL_OK; ++it) rc = enqueue_iteration(g, w, nrhs, w->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(w->cap_stream, &graph);
        w->graph_tslots = timing_capture_end(g);
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
        w->graph_timed = timed;
    }
    WL_TRY(timing_harvest(g));  // the previous replay's times, before this one records them again
    WL_CUDA(cudaGraphLaunch(w->graph, s));
    count_launch(w->graph_kernels, (double)w->graph_bytes);
    if (w->graph_timed) timing_replayed(g, w->graph_tslots);
    return WL_OK;
}

// r = b' - A x in FP64 for masked rhs, with ||r||^2 into w->nrm.
int residual64(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s)
{
    const size_t hb = w->hb64;
    if (w->eo) {
        HopLaunch h1;
        h1.prec = w->outer;
        h1.parity0 = 1;
        h1.nrhs = nrhs;
        h1.in[0] = w->xhi;
        h1.out[0] = w->tmp64;
        h1.rs_in = full_rs(w);
        h1.rs_out = (long long)hb;
        h1.active = w->mask;
        if (g->has_clover) {  // tmp = A_oo^-1 H_oe x
            h1.cl_mode = kClOut;
            h1.clov[0] = g->clov[w->outer][1][1];
        }
        WL_TRY(launch_hop(g, h1, s));
        HopLaunch h2;
        h2.prec = w->outer;
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
        if (g->has_clover) {  // r = b' - A_ee x + kappa^2 H_eo tmp
            h2.cl_mode = kClX2;
            h2.clov[0] = g->clov[w->outer][0][0];
        }
        return launch_hop(g, h2, s);
    }
    // full: r_p = b_p - x_p + kappa H x_{1-p}
    HopLaunch h;
    h.prec = w->outer;
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
    if (g->has_clover) {  // r_p = b_p - A_pp x_p + kappa H x_{1-p}
        h.cl_mode = kClX2;
        h.clov[0] = g->clov[w->outer][0][0];
        h.clov[1] = g->clov[w->outer][1][0];
    }
    return launch_hop(g, h, s);
}

// r_full = b - D x on the full lattice (FP64) with ||r||^2 into w->nrm.
// r = b - D x in FP64 with ||r||^2 into w->nrm.  Full solves evaluate both
// parities.  Even-odd Wilson solves evaluate the even half only: the odd
// half, b_o - x_o + kappa H_oe x_e, is zero by construction because x_o was
// just formed as b_o + kappa H_oe x_e by the same FP64 operations.  With a
// clover term x_o = A_oo^-1 (...) leaves a rounding-level odd residual, so
// both halves are evaluated.
int true_residual64(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s, double* dot_out)
{
    const size_t hb = w->hb64;
    HopLaunch h;
    h.prec = WL_F64;  // IEEE FP64 on the FP64 copies of b and x
    h.parity0 = 0;
    h.nparity = w->eo && !g->has_clover ? 1 : 2;
    if (g->has_clover) {  // r_p = b_p - A_pp x_p + kappa H x_{1-p}
        h.cl_mode = kClX2;
        h.clov[0] = g->clov[WL_F64][0][0];
        h.clov[1] = g->clov[WL_F64][1][0];
    }
    h.nrhs = nrhs;
    h.in[0] = (const char*)w->x64 + hb;
    h.in[1] = w->x64;
    h.out[0] = w->rhi;
    h.out[1] = (char*)w->rhi + hb;
    h.x1[0] = w->b64;
    h.x1[1] = (const char*)w->b64 + hb;
    h.x2[0] = w->x64;
    h.x2[1] = (const char*)w->x64 + hb;
    h.rs_in = h.rs_out = h.rs_x1 = h.rs_x2 = full_rs(w);
    h.b1 = -1.0;
    h.a = g->kappa;
    h.dot = true;
    h.dot_out = dot_out ? dot_out : w->nrm;
    return launch_hop(g, h, s);
}

// The host mask travels as kernel parameters (bit-packed), which the launch
// copies when it is issued: the host may rewrite mask_h right after, as the
// outer loop does, without racing an asynchronous copy from pinned memory.
struct MaskBits {
    unsigned word[256];  // 8192 right-hand sides per launch
};

__global__ void set_mask_kernel(int* mask, int first, int n, const MaskBits bits)
{
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        mask[first + k] = (bits.word[k >> 5] >> (k & 31)) & 1u;
}

int upload_mask(Workspace* w, int nrhs, cudaStream_t s)
{
    for (int first = 0; first < nrhs; first += 8192) {
        const int n = nrhs - first < 8192 ? nrhs - first : 8192;
        MaskBits bits;
        std::memset(&bits, 0, sizeof bits);
        for (int k = 0; k < n; ++k)
            if (w->mask_h[first + k]) bits.word[k >> 5] |= 1u << (k & 31);
        set_mask_kernel<<<1, 256, 0, s>>>(w->mask, first, n, bits);
        WL_CHECK_LAUNCH(0.0);
    }
    return WL_OK;
}

int read_norms(Workspace* w, int nrhs, cudaStream_t s)
{
    WL_CUDA(cudaMemcpyAsync(w->nrm_h, w->nrm, sizeof(double) * 3 * nrhs, cudaMemcpyDeviceToHost, s));
    WL_CUDA(cudaStreamSynchronize(s));
    return WL_OK;
}

// Begin an inner solve for the masked rhs: r = r_hi (converted), rhat = r,
// p = v = x_lo = 0, fresh scalars with the given targets.
int inner_start(wl_gauge g, Workspace* w, int nrhs, const double* target2,
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
    WL_TRY(launch_convert(g, P, w->r, w->outer, w->rhi, w->nhalf, nrhs, w->mask, s));
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
int reliable_update(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s)
{
    const int P = w->inner;
    WL_TRY(upload_mask(w, nrhs, s));
    WL_TRY(launch_accum_hi(g, w->outer, w->xhi, w->xlo_prec, w->xlo, w->nhalf, nrhs, w->mask, s,
                           full_rs(w)));
    WL_TRY(launch_zero(g, w->xlo_prec, w->xlo, w->nhalf, nrhs, w->mask, s));
    WL_TRY(residual64(g, w, nrhs, s));
    WL_TRY(launch_convert(g, P, w->r, w->outer, w->rhi, w->nhalf, nrhs, w->mask, s));
    WL_TRY(launch_cdot(g, P, w->rh, w->r, w->nhalf, nrhs, w->sc[0].rr, kScalStride, w->mask, s));
    init_scal_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(w->sc, w->mask, nrhs, 0);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

}  // namespace wl

namespace wl {

static bool is_host_pointer(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

static int check_params(wl_gauge g, const void* x, const void* b, int nrhs,
                        const wl_solve_params* prm)
{
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (g->dd_part) return set_error(WL_ERR_STATE, "block of a domain decomposition: use the _dd calls");
    if (!x || !b || !prm) return set_error(WL_ERR_ARG, "NULL pointer");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    if (prm->inner < WL_F64 || prm->inner > WL_F16) return set_error(WL_ERR_ARG, "unknown inner precision");
    if (!(prm->tol > 0.0)) return set_error(WL_ERR_ARG, "tol must be > 0");
    if (prm->maxiter < 1) return set_error(WL_ERR_ARG, "maxiter must be >= 1");
    if (!g->links[prm->inner][0])
        return set_error(WL_ERR_STATE, "gauge object was created without the inner precision");
    return WL_OK;
}

int stream_join(cudaStream_t into, cudaStream_t from, cudaEvent_t ev)
{
    WL_CUDA(cudaEventRecord(ev, from));
    WL_CUDA(cudaStreamWaitEvent(into, ev, 0));
    return WL_OK;
}

int SolveState::begin(wl_gauge g_, double* x, const double* b, int nrhs_, const wl_solve_params* p,
                      cudaStream_t s_)
{
    WL_TRY(begin_issue(g_, x, b, nrhs_, p, s_, false));
    WL_CUDA(cudaStreamSynchronize(s));
    begin_collect();
    return WL_OK;
}

int SolveState::begin_issue(wl_gauge g_, double* x, const double* b, int nrhs_, const wl_solve_params* p,
                            cudaStream_t s_, bool lane)
{
    t0 = std::chrono::steady_clock::now();
    WL_TRY(check_params(g_, x, b, nrhs_, p));
    g = g_;
    prm = p;
    nrhs = nrhs_;
    s = s_;
    eo = p->eo ? 1 : 0;
    P = p->inner;
    x_user = x;
    WL_TRY(ensure_ws(g, P, nrhs, eo));
    w = g->ws;
    w->chunk_k = 0;
    if (lane) {  // the workspace's own stream, after the caller's work on s
        if (!w->lane) {
            WL_CUDA(cudaStreamCreateWithFlags(&w->lane, cudaStreamNonBlocking));
            WL_CUDA(cudaEventCreateWithFlags(&w->ev_lane, cudaEventDisableTiming));
        }
        WL_TRY(stream_join(w->lane, s_, w->ev_lane));
        s = w->lane;
        own_stream = true;
    }
    const long long V = 2 * g->geo.Vh;
    canon = (size_t)V * 24 * sizeof(double) * nrhs;

    // host buffers are staged through the workspace
    const bool host_b = is_host_pointer(b);
    host_x = is_host_pointer(x);
    const double* bd = b;
    xd = x;
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
    // b -> internal FP64 (even | odd per rhs): one conversion per parity for all rhs
    WL_TRY(field_to_internal(g, w->b64, bd, 0, WL_F64, nrhs, s, 2 * (long long)hb64));
    WL_TRY(field_to_internal(g, (char*)w->b64 + hb64, bd, 1, WL_F64, nrhs, s, 2 * (long long)hb64));
    if (prm->use_x0) {
        WL_TRY(field_to_internal(g, w->xhi, xd, 0, w->outer, nrhs, s, 2 * (long long)hb64));
        WL_TRY(field_to_internal(g, (char*)w->xhi + hb64, xd, 1, w->outer, nrhs, s, 2 * (long long)hb64));
    }
    if (!prm->use_x0) WL_CUDA(cudaMemsetAsync(w->xhi, 0, 2 * hb64 * nrhs, s));
    // ||b||^2 over the full lattice, into the second set of norm slots
    WL_TRY(launch_cdot(g, WL_F64, w->b64, w->b64, 2, nrhs, w->nrm + 3 * nrhs, 3, nullptr, s));
    if (w->bout != w->b64)  // b in the outer precision
        WL_TRY(launch_convert(g, w->outer, w->bout, WL_F64, w->b64, 2, nrhs, nullptr, s));
    // b' = b_e + kappa H_eo b_o (even-odd) or b (full)
    if (eo) {
        HopLaunch h;
        h.prec = w->outer;
        h.parity0 = 0;
        h.nrhs = nrhs;
        h.in[0] = (const char*)w->bout + hb64;
        h.out[0] = w->bp;
        h.x1[0] = w->bout;
        h.rs_in = h.rs_x1 = full_rs(w);
        h.rs_out = (long long)hb64;
        h.a = g->kappa;
        if (g->has_clover) {  // b' = b_e + kappa H_eo A_oo^-1 b_o
            WL_TRY(launch_clover_apply(g, w->outer, w->tmp64, (const char*)w->bout + hb64, 1, 1, nrhs, s,
                                       (long long)hb64, full_rs(w)));
            h.in[0] = w->tmp64;
            h.rs_in = (long long)hb64;
        }
        WL_TRY(launch_hop(g, h, s));
    } else {
        WL_CUDA(cudaMemcpyAsync(w->bp, w->bout, 2 * hb64 * nrhs, cudaMemcpyDeviceToDevice, s));
    }
    for (int k = 0; k < nrhs; ++k) std::memset(&w->sc_h[k], 0, sizeof(Scal));
    WL_CUDA(cudaMemcpyAsync(w->sc, w->sc_h, sizeof(Scal) * nrhs, cudaMemcpyHostToDevice, s));
    // the first residual of every right-hand side (a zero b is found by the
    // host afterwards and never iterated)
    for (int k = 0; k < nrhs; ++k) w->mask_h[k] = 1;
    if (prm->use_x0) {
        WL_TRY(upload_mask(w, nrhs, s));
        WL_TRY(residual64(g, w, nrhs, s));
    } else {  // x = 0: r = b' exactly, no FP64 matrix apply needed
        WL_CUDA(cudaMemcpyAsync(w->rhi, w->bp, w->vb64 * nrhs, cudaMemcpyDeviceToDevice, s));
        WL_TRY(launch_cdot(g, w->outer, w->bp, w->bp, w->nhalf, nrhs, w->nrm, 3, nullptr, s));
    }
    WL_CUDA(cudaMemcpyAsync(w->nrm_h, w->nrm, sizeof(double) * 6 * nrhs, cudaMemcpyDeviceToHost, s));
    return WL_OK;
}

void SolveState::begin_collect()
{
    bnorm2.assign(nrhs, 0.0);
    rnorm2.assign(nrhs, 0.0);
    target2.assign(nrhs, 0.0);
    done.assign(nrhs, 0);
    final_target.assign(nrhs, 0);
    shortcut.assign(nrhs, 0);
    status.assign(nrhs, WL_OK);
    outer.assign(nrhs, 0);
    restarts.assign(nrhs, 0);
    part.assign(nrhs, 0);
    in_inner.assign(nrhs, 0);
    poisoned.assign(nrhs, 0);
    iters_before.assign(nrhs, 0);
    for (int k = 0; k < nrhs; ++k) {
        bnorm2[k] = w->nrm_h[3 * nrhs + 3 * k + 2];
        if (bnorm2[k] == 0.0) done[k] = 1;  // x = 0 solves b = 0 exactly
        rnorm2[k] = done[k] ? 0.0 : w->nrm_h[3 * k + 2];
    }
    delta2 = prm->delta > 0.0 ? prm->delta * prm->delta : 0.0;
    // default inner reduction per round: FP32 to 3e-6 (a sweep over 1e-4 .. 3e-7
    // on the 32^3 x 64, 12-RHS and clover workloads found it fastest), FP16 to 1e-3
    inner_tol = prm->inner_tol > 0.0 ? prm->inner_tol : (P == WL_F64 ? 0.0 : P == WL_F32 ? 3e-6 : 1e-3);
    // iterations per host check; replayed as a CUDA graph unless graph_iters < 0
    chunk = prm->graph_iters > 0 ? prm->graph_iters : prm->graph_iters < 0 ? -prm->graph_iters : 4;
    use_graph = prm->graph_iters >= 0;
    safety = 0.5;  // aim below tol on the Schur residual; tightened if the true residual misses
    final_rounds = 0;
}

int SolveState::plan(bool* any_out)
{
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
        final_target[k] = t2 == goal2;
        if (solve_verbose())
            fprintf(stderr, "[wl solve] Vh=%lld rhs %d: round from iters %d, |r|/|b| %.3e, target %.3e%s\n",
                    g->geo.Vh, k, w->sc_h[k].iters, std::sqrt(rnorm2[k] / bnorm2[k]),
                    std::sqrt(t2 / bnorm2[k]), final_target[k] ? " (final)" : "");
    }
    *any_out = any != 0;
    if (!any) return WL_OK;
    hist_rr.assign(nrhs, 0.0);
    hist_it.assign(nrhs, 0);
    next_k = 0;
    for (int k = 0; k < nrhs; ++k) {
        iters_before[k] = w->sc_h[k].iters;
        part[k] = in_inner[k] = w->mask_h[k];
        poisoned[k] = 0;
        hist_rr[k] = rnorm2[k];
        hist_it[k] = iters_before[k];
    }
    return inner_start(g, w, nrhs, target2.data(), delta2, s);
}

int SolveState::cap() const
{
    int most = 0;  // iterations done by the furthest-along right-hand side of the round
    for (int k = 0; k < nrhs; ++k)
        if (in_inner[k] && w->sc_h[k].iters > most) most = w->sc_h[k].iters;
    return chunk < prm->maxiter - most ? chunk : prm->maxiter - most;
}

int SolveState::want() const { return next_k > 0 && next_k < chunk ? next_k : chunk; }

int SolveState::budget() const { return std::min(cap(), want()); }

// Length of the next chunk: the iterations each active right-hand side still
// needs to reach its inner target (or its next reliable update), extrapolated
// from the residual's decay over the last chunk; the longest of them, at most
// one chunk.  Launching past convergence costs empty launches, stopping short
// one more host round trip.
void SolveState::predict_next()
{
    int most = 0;
    bool any = false;
    for (int k = 0; k < nrhs; ++k) {
        if (!in_inner[k]) continue;
        const Scal& S = w->sc_h[k];
        const double rr = S.rr[2];
        const int dit = S.iters - hist_it[k];
        if (S.active) {
            any = true;
            int n = chunk;
            if (dit > 0 && rr > 0.0 && hist_rr[k] > rr) {
                const double rate = std::log(rr / hist_rr[k]) / dit;  // per iteration, < 0
                double est = std::log(S.target2 / rr) / rate;
                if (S.delta2 > 0.0 && S.r2_max > 0.0)
                    est = std::min(est, std::log(S.delta2 * S.r2_max / rr) / rate);
                n = est <= 1.0 ? 1 : (int)std::ceil(std::min(est, (double)chunk));
            }
            most = std::max(most, n);
        }
        hist_rr[k] = rr;
        hist_it[k] = S.iters;
    }
    next_k = any ? most : 0;
}

int SolveState::read_scalars()
{
    WL_CUDA(cudaMemcpyAsync(w->sc_h, w->sc, sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, s));
    WL_CUDA(cudaStreamSynchronize(s));
    return WL_OK;
}

int SolveState::after_chunk(bool* alive)
{
    int upd = 0, stopped = 0;
    {  // iterations of the chunk that ran after every right-hand side had stopped
        int did = 0;
        for (int k = 0; k < nrhs; ++k)
            if (in_inner[k]) did = std::max(did, w->sc_h[k].iters - hist_it[k]);
        discount_chunk(g, w, w->chunk_k - did);
    }
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
        if (solve_verbose())
            for (int k = 0; k < nrhs; ++k)
                if (w->mask_h[k])
                    fprintf(stderr, "[wl solve] Vh=%lld rhs %d: reliable update at iters %d\n", g->geo.Vh, k,
                            w->sc_h[k].iters);
        WL_TRY(read_scalars());  // keep the host copy current for later pushes
    }
    bool a = false;
    for (int k = 0; k < nrhs; ++k) a |= in_inner[k] != 0;
    *alive = a;
    if (a) predict_next();
    return WL_OK;
}

int SolveState::finish_round()
{
    bool pending = false;
    WL_TRY(finish_round_issue(&pending));
    if (!pending) return WL_OK;
    WL_CUDA(cudaStreamSynchronize(s));
    finish_round_collect();
    return WL_OK;
}

int SolveState::finish_round_issue(bool* pending)
{
    *pending = false;
    const int nh = w->nhalf;
    int any_poison = 0;
    for (int k = 0; k < nrhs; ++k) {
        w->mask_h[k] = poisoned[k];
        any_poison |= poisoned[k];
        in_inner[k] = 0;
    }
    if (any_poison) {  // a NaN correction is dropped, not accumulated
        WL_TRY(upload_mask(w, nrhs, s));
        WL_TRY(launch_zero(g, w->xlo_prec, w->xlo, nh, nrhs, w->mask, s));
    }
    for (int k = 0; k < nrhs; ++k) w->mask_h[k] = part[k];
    WL_TRY(upload_mask(w, nrhs, s));
    WL_TRY(launch_accum_hi(g, w->outer, w->xhi, w->xlo_prec, w->xlo, nh, nrhs, w->mask, s,
                           full_rs(w)));
    // a right-hand side whose inner solve just reached the final goal goes
    // straight to the true-residual check; the others need the FP64 residual
    int need = 0;
    for (int k = 0; k < nrhs; ++k) {
        const bool reached = part[k] && final_target[k] && !poisoned[k] &&
                             (w->sc_h[k].flags & FLAG_CONVERGED) && w->sc_h[k].iters > iters_before[k];
        if (reached) {
            done[k] = 1;
            shortcut[k] = 1;
            outer[k]++;
            part[k] = 0;
        }
        if (solve_verbose() && (reached || part[k]))
            fprintf(stderr, "[wl solve] Vh=%lld rhs %d: round ends at iters %d, flags %d%s\n", g->geo.Vh, k,
                    w->sc_h[k].iters, w->sc_h[k].flags, reached ? ", final goal reached: true residual next" : "");
        w->mask_h[k] = part[k];
        need |= part[k];
    }
    if (!need) return WL_OK;
    WL_TRY(upload_mask(w, nrhs, s));
    WL_TRY(residual64(g, w, nrhs, s));
    WL_CUDA(cudaMemcpyAsync(w->nrm_h, w->nrm, sizeof(double) * 3 * nrhs, cudaMemcpyDeviceToHost, s));
    *pending = true;
    return WL_OK;
}

void SolveState::finish_round_collect()
{
    for (int k = 0; k < nrhs; ++k)
        if (part[k]) {
            rnorm2[k] = w->nrm_h[3 * k + 2];
            outer[k]++;
            if (solve_verbose())
                fprintf(stderr, "[wl solve] Vh=%lld rhs %d: outer residual %.3e\n", g->geo.Vh, k,
                        std::sqrt(rnorm2[k] / bnorm2[k]));
            // an inner solve that could not move (its start already met the
            // inner target) ends the outer loop; the true residual decides
            if (w->sc_h[k].iters == iters_before[k] && !done[k]) done[k] = 1;
            if (outer[k] > kMaxOuter && !done[k]) {
                done[k] = 1;
                status[k] = WL_ERR_NOT_CONVERGED;
            }
        }
}

int SolveState::finalize(bool* retry_out)
{
    WL_TRY(finalize_issue());
    WL_CUDA(cudaStreamSynchronize(s));
    return finalize_collect(retry_out);
}

int SolveState::finalize_issue()
{
    const size_t hb64 = w->hb64;
    if (w->x64 != w->xhi)  // the solution in FP64 (the even half for even-odd solves)
        WL_TRY(launch_convert(g, WL_F64, w->x64, w->outer, w->xhi, w->nhalf, nrhs, nullptr, s,
                              full_rs(w), full_rs(w)));
    if (eo) {  // x_o = b_o + kappa H_oe x_e in FP64
        HopLaunch h;
        h.prec = WL_F64;
        h.parity0 = 1;
        h.nrhs = nrhs;
        h.in[0] = w->x64;
        h.out[0] = (char*)w->x64 + hb64;
        h.x1[0] = (const char*)w->b64 + hb64;
        h.rs_in = h.rs_out = h.rs_x1 = full_rs(w);
        h.a = g->kappa;
        if (g->has_clover) {  // x_o = A_oo^-1 (b_o + kappa H_oe x_e)
            h.cl_mode = kClOut;
            h.clov[0] = g->clov[WL_F64][1][1];
        }
        WL_TRY(launch_hop(g, h, s));
    }
    WL_TRY(send_x());  // the caller's x is written while the check below runs
    // the norms go straight to the pinned host buffer: a copy-engine read-back
    // would queue behind the copy of x
    double* nrm_dev = nullptr;
    WL_CUDA(cudaHostGetDevicePointer((void**)&nrm_dev, w->nrm_h, 0));
    return true_residual64(g, w, nrhs, s, nrm_dev);
}

int SolveState::finalize_collect(bool* retry_out)
{
    bool retry = false, tighten = false;
    for (int k = 0; k < nrhs; ++k) {
        const double tr = bnorm2[k] > 0 ? std::sqrt(w->nrm_h[3 * k + 2] / bnorm2[k]) : 0.0;
        rnorm2[k] = tr;  // kept for end(); overwritten below on retry
        if (solve_verbose())
            fprintf(stderr, "[wl solve] Vh=%lld rhs %d: true residual %.3e at iters %d (shortcut %d)\n",
                    g->geo.Vh, k, tr, w->sc_h[k].iters, shortcut[k]);
        if (status[k] == WL_OK && !(tr <= prm->tol)) {
            if (shortcut[k]) {
                // only the iterated residual had met the goal: run another round
                // from the FP64 residual at the same goal
                shortcut[k] = 0;
                done[k] = 0;
                retry = true;
            } else if (final_rounds < 3 && w->sc_h[k].iters < prm->maxiter) {
                done[k] = 0;
                retry = tighten = true;
            } else {
                status[k] = std::isfinite(tr) ? WL_ERR_NOT_CONVERGED : WL_ERR_NAN;
            }
        } else {
            shortcut[k] = 0;
        }
    }
    true_resid.assign(rnorm2.begin(), rnorm2.end());
    *retry_out = retry;
    if (!retry) return WL_OK;
    // the next rounds rewrite x: only after the side stream has read it
    WL_CUDA(cudaStreamWaitEvent(s, w->ev_sent, 0));
    x_sent = false;
    if (tighten) {  // the FP64 Schur residual met the goal but the full one did not: aim lower
        ++final_rounds;
        safety *= 0.1;
    }
    for (int k = 0; k < nrhs; ++k) w->mask_h[k] = done[k] ? 0 : 1;
    WL_TRY(upload_mask(w, nrhs, s));
    WL_TRY(residual64(g, w, nrhs, s));
    WL_TRY(read_norms(w, nrhs, s));
    for (int k = 0; k < nrhs; ++k) if (w->mask_h[k]) rnorm2[k] = w->nrm_h[3 * k + 2];
    return WL_OK;
}

int SolveState::send_x()
{
    if (!w->aux) {
        WL_CUDA(cudaStreamCreateWithFlags(&w->aux, cudaStreamNonBlocking));
        WL_CUDA(cudaEventCreateWithFlags(&w->ev_x, cudaEventDisableTiming));
        WL_CUDA(cudaEventCreateWithFlags(&w->ev_sent, cudaEventDisableTiming));
    }
    // the conversion runs on the solver's stream (the check that follows is a
    // grid of resident blocks, which would hold it off the SMs); only the copy
    // to the host, on the copy engine, runs beside the check
    const size_t hb64 = w->hb64;
    WL_TRY(field_to_canonical(g, xd, w->x64, 0, WL_F64, nrhs, s, 2 * (long long)hb64));
    WL_TRY(field_to_canonical(g, xd, (const char*)w->x64 + hb64, 1, WL_F64, nrhs, s, 2 * (long long)hb64));
    WL_CUDA(cudaEventRecord(w->ev_x, s));
    WL_CUDA(cudaStreamWaitEvent(w->aux, w->ev_x, 0));
    x_sent = true;  // from here on the side stream is waited for on every exit
    if (host_x) WL_CUDA(cudaMemcpyAsync(x_user, xd, canon, cudaMemcpyDeviceToHost, w->aux));
    WL_CUDA(cudaEventRecord(w->ev_sent, w->aux));
    return WL_OK;
}

SolveState::~SolveState()
{
    // an early return must not leave a copy into the caller's buffer in flight
    // (nor, on a lane stream, work that reads or writes the caller's buffers)
    if (w && x_sent && w->aux) cudaStreamSynchronize(w->aux);
    if (own_stream && s) cudaStreamSynchronize(s);
}

int SolveState::end(wl_solve_info* info)
{
    if (!x_sent) WL_TRY(send_x());
    WL_CUDA(cudaStreamSynchronize(w->aux));
    WL_CUDA(cudaStreamSynchronize(s));
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int rc = WL_OK;
    for (int k = 0; k < nrhs; ++k) {
        info[k].iters = w->sc_h[k].iters;
        info[k].outer = outer[k];
        info[k].restarts = restarts[k];
        info[k].status = status[k];
        info[k].true_resid = true_resid.empty() ? 0.0 : true_resid[k];
        info[k].secs = secs;
        if (status[k] != WL_OK && rc == WL_OK) rc = status[k];
    }
    if (rc != WL_OK) set_error(rc, "at least one right-hand side did not reach tol");
    return rc;
}

}  // namespace wl

using namespace wl;

extern "C" int wilson_solve(wl_gauge g, double* x, const double* b, int nrhs,
                            const wl_solve_params* prm, wl_solve_info* info, void* stream)
{
    WL_ENTRY();
    if (!info) return set_error(WL_ERR_ARG, "NULL pointer");
    SolveState st;
    WL_TRY(st.begin(g, x, b, nrhs, prm, (cudaStream_t)stream));
    for (;;) {
        for (;;) {  // outer loop: FP64 residual -> inner solve -> FP64 update
            bool any = false;
            WL_TRY(st.plan(&any));
            if (!any) break;
            for (;;) {
                const int k = st.budget();
                if (k <= 0) break;
                WL_TRY(run_chunk(g, st.w, nrhs, k, st.use_graph && k == st.chunk, st.s));
                WL_TRY(st.read_scalars());
                bool alive = false;
                WL_TRY(st.after_chunk(&alive));
                if (!alive) break;
            }
            WL_TRY(st.finish_round());
        }
        bool retry = false;
        WL_TRY(st.finalize(&retry));
        if (!retry) break;
    }
    return st.end(info);
}
