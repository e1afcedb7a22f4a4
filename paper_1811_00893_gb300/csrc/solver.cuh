// Solver internals shared by the single-lattice solve (solver.cu) and the
// multi-lattice batch (batch.cu): the per-right-hand-side device scalars,
// the workspace, the per-site BiCGStab updates and the host-side state of
// one lattice's solve.
#pragma once

#include <chrono>
#include <vector>

#include "internal.cuh"

namespace wl {

// Device scalars of one right-hand side's BiCGStab.
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
static const int kActiveStride = sizeof(Scal) / sizeof(int);
static const int kMaxOuter = 500;  // FP64 corrections per solve
static const int kBlock = 256;     // vector-kernel block size

struct Workspace {
    int inner = -1, nrhs = 0, eo = -1, nhalf = 0, xlo_prec = 0, outer = 0;
    // the last chunk: iterations enqueued, bytes charged, timing slots used
    int chunk_k = 0;
    long long chunk_bytes = 0;
    size_t chunk_slot0 = 0, chunk_slot1 = 0;
    size_t vb = 0;    // bytes of one inner vector (nhalf halves)
    size_t vb64 = 0;  // bytes of one FP64 vector (nhalf halves)
    size_t hb64 = 0;  // bytes of one FP64 half field
    // inner-precision vectors (nrhs each)
    void *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
         *xlo = nullptr, *tmp = nullptr;
    // outer-precision vectors (nrhs each): b', x (even | odd), residual, odd temporary;
    // b64 and x64 are the IEEE FP64 b and x (even | odd) of the final check, bout
    // is b in the outer precision (aliases b64 and xhi when the outer is FP64)
    double *b64 = nullptr, *bp = nullptr, *xhi = nullptr, *rhi = nullptr, *tmp64 = nullptr;
    double *bout = nullptr, *x64 = nullptr;
    Scal* sc = nullptr;
    Scal* sc_h = nullptr;  // pinned
    int* mask = nullptr;
    int* mask_h = nullptr;  // pinned
    double* nrm = nullptr;  // 6 doubles per rhs: two sets of 3 (dot, norm)
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
    long long graph_kernels = 0;
    long long graph_bytes = 0;
    bool graph_timed = false;   // captured while per-launch timing was on
    size_t graph_tslots = 0;    // its timed launches (capture slots)
    cudaStream_t cap_stream = nullptr;  // private stream for graph capture
    int tuned_nrhs = 0;  // the iteration's hopping launches were timed for this many rhs
    // the solution's canonical copy (and host copy) while the final check runs
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_x = nullptr, ev_sent = nullptr;
    // this gauge object's own stream, for its share of a batch's per-lattice work
    cudaStream_t lane = nullptr;
    cudaEvent_t ev_lane = nullptr;
};

// Make `into` wait for the work already enqueued on `from` (ev: a scratch event).
int stream_join(cudaStream_t into, cudaStream_t from, cudaEvent_t ev);

// ---------------------------------------------------------------------------
// per-site BiCGStab updates (device), used by single and batched kernels
// ---------------------------------------------------------------------------

__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// beta = (rho / rho_prev)(alpha / omega) and omega, as {beta.re, beta.im, om.re, om.im}
__device__ __forceinline__ void beta_omega(const Scal& S, double (&c)[4])
{
    const cx<double> rho = {S.rr[0], S.rr[1]}, rp = {S.rho_prev[0], S.rho_prev[1]};
    const cx<double> al = {S.alpha[0], S.alpha[1]}, om = {S.omega[0], S.omega[1]};
    const cx<double> beta = cdiv(rho, rp) * cdiv(al, om);
    c[0] = beta.re;
    c[1] = beta.im;
    c[2] = om.re;
    c[3] = om.im;
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

// p = r + beta (p - omega v)
template <int P>
__device__ __forceinline__ void p_update_site(char* p, const char* r, const char* v, long long Vh,
                                              long long i, const double (&c)[4])
{
    using T = typename Prec<P>::real;
    const cx<T> beta = {(T)c[0], (T)c[1]}, om = {(T)c[2], (T)c[3]};
    cx<T> pp[12], rr[12], vv[12];
    load_spinor<P>(pp, p, Vh, i);
    load_spinor<P>(rr, r, Vh, i);
    load_spinor<P>(vv, v, Vh, i);
#pragma unroll
    for (int c2 = 0; c2 < 12; ++c2) pp[c2] = rr[c2] + beta * (pp[c2] - om * vv[c2]);
    store_spinor<P>(p, Vh, i, pp);
}

// s = r - alpha v
template <int P>
__device__ __forceinline__ void s_update_site(char* s, const char* r, const char* v, long long Vh,
                                              long long i, cx<double> al_)
{
    using T = typename Prec<P>::real;
    const cx<T> al = {(T)al_.re, (T)al_.im};
    cx<T> rr[12], vv[12];
    load_spinor<P>(rr, r, Vh, i);
    load_spinor<P>(vv, v, Vh, i);
#pragma unroll
    for (int c = 0; c < 12; ++c) rr[c] = rr[c] - al * vv[c];
    store_spinor<P>(s, Vh, i, rr);
}

// x += alpha p + omega s;  r = s - omega t;  part = (rhat, r), ||r||^2 of the
// stored (rounded) r, so rho matches what the next p update reads
template <int P, int PX>
__device__ __forceinline__ void xr_update_site(char* x, char* r, const char* p, const char* s,
                                               const char* t, const char* rh, long long Vh,
                                               long long i, const double (&dc)[4],
                                               typename Prec<P>::real (&part)[3])
{
    using T = typename Prec<P>::real;
    using TX = typename Prec<PX>::real;
    const cx<T> al = {(T)dc[0], (T)dc[1]}, om = {(T)dc[2], (T)dc[3]};
    cx<T> pp[12], ss[12];
    load_spinor<P>(pp, p, Vh, i);
    load_spinor<P>(ss, s, Vh, i);
    {
        cx<TX> xx[12];
        load_spinor<PX>(xx, x, Vh, i);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const cx<T> d = al * pp[c] + om * ss[c];
            xx[c] = {xx[c].re + (TX)d.re, xx[c].im + (TX)d.im};
        }
        store_spinor<PX>(x, Vh, i, xx);
    }
    cx<T> tt[12];
    load_spinor<P>(tt, t, Vh, i);
#pragma unroll
    for (int c = 0; c < 12; ++c) ss[c] = ss[c] - om * tt[c];
    store_spinor<P>(r, Vh, i, ss);
    cx<T> rn[12], hh[12];
    load_spinor<P>(rn, r, Vh, i);
    load_spinor<P>(hh, rh, Vh, i);
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

// The last block of the x/r update advances one right-hand side's scalars and
// decides convergence, breakdown or a reliable update.
__device__ __forceinline__ void advance_scalars(Scal& S, const double (&tot)[3],
                                                const double (&dc)[4])
{
    S.rho_prev[0] = S.rr[0];
    S.rho_prev[1] = S.rr[1];
    S.alpha[0] = dc[0];
    S.alpha[1] = dc[1];
    S.omega[0] = dc[2];
    S.omega[1] = dc[3];
    S.rr[0] = tot[0];
    S.rr[1] = tot[1];
    S.rr[2] = tot[2];
    S.iters += 1;
    const bool stepped = (dc[0] != 0.0 || dc[1] != 0.0);
    const bool omega0 = (dc[2] == 0.0 && dc[3] == 0.0);
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int ensure_ws(wl_gauge g, int inner, int nrhs, int eo);
int upload_mask(Workspace* w, int nrhs, cudaStream_t s);
int run_chunk(wl_gauge g, Workspace* w, int nrhs, int k, bool use_graph, cudaStream_t s);
void discount_chunk(wl_gauge g, Workspace* w, int skipped);
int read_norms(Workspace* w, int nrhs, cudaStream_t s);
int residual64(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s);
// dot_out: where the norms go (default w->nrm; finalize passes the pinned
// host buffer's device alias, so that no copy-engine transfer is needed)
int true_residual64(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s, double* dot_out = nullptr);
int inner_start(wl_gauge g, Workspace* w, int nrhs, const double* target2, double delta2,
                cudaStream_t s);
int reliable_update(wl_gauge g, Workspace* w, int nrhs, cudaStream_t s);
inline long long full_rs(const Workspace* w) { return (long long)(2 * w->hb64); }

// One lattice's solve, advanced step by step by a driver (wilson_solve runs
// one; wilson_solve_batch runs several and replaces the inner iterations by
// batched launches).  Between rounds every right-hand side is inactive on
// the device, so batched kernels skip this lattice.
struct SolveState {
    wl_gauge g = nullptr;
    Workspace* w = nullptr;
    const wl_solve_params* prm = nullptr;
    int nrhs = 0, eo = 0, P = 0;
    cudaStream_t s = nullptr;
    bool own_stream = false;  // s is the workspace's lane stream (batched solves)
    double* x_user = nullptr;
    double* xd = nullptr;
    bool host_x = false;
    size_t canon = 0;
    std::vector<double> bnorm2, rnorm2, target2, true_resid;
    std::vector<int> done, status, outer, restarts, part, in_inner, poisoned, iters_before;
    std::vector<int> final_target;  // this round's inner target is the final goal
    std::vector<int> shortcut;      // went to the final check on the iterated residual
    double delta2 = 0.0, inner_tol = 0.0, safety = 0.5;
    int final_rounds = 0, chunk = 4;
    // residual history at the last chunk boundary, for the length of the next chunk
    std::vector<double> hist_rr;
    std::vector<int> hist_it;
    int next_k = 0;  // predicted iterations to the next stop (0: none yet)
    bool use_graph = false;
    std::chrono::steady_clock::time_point t0;

    // The steps that need host values computed on the device come in two
    // halves: *_issue enqueues the work and the read-back, *_collect uses the
    // values once the caller has synchronised s.  A batch issues every
    // lattice's half on its own stream before it waits for any of them.

    // set up: stage host buffers, convert b (and x0), b', ||b||^2, r = b' - A x0
    // and ||r||^2.  With lane, the work runs on the workspace's own stream,
    // after the work already on s.
    int begin(wl_gauge g, double* x, const double* b, int nrhs, const wl_solve_params* p,
              cudaStream_t s);
    int begin_issue(wl_gauge g, double* x, const double* b, int nrhs, const wl_solve_params* p,
                    cudaStream_t s, bool lane);
    void begin_collect();
    // choose the right-hand sides of the next inner round and start it; *any
    // is false when no right-hand side needs one
    int plan(bool* any);
    // iterations the next chunk may run (0: the round must end): the smaller
    // of cap() (one chunk, within maxiter) and want() (the prediction)
    int budget() const;
    int cap() const;
    int want() const;
    // extrapolate the iterations to the next stop from the residual history
    void predict_next();
    // copy the device scalars to the host (the stream is synchronised)
    int read_scalars();
    // after a chunk: reliable updates, breakdowns, iteration limits; *alive is
    // false once every right-hand side of the round has stopped
    int after_chunk(bool* alive);
    // end a round: x += x_lo in FP64 and the FP64 residual (*pending: a
    // read-back was issued and collect must follow the synchronisation)
    int finish_round();
    int finish_round_issue(bool* pending);
    void finish_round_collect();
    // reconstruct the odd half, the true residual of the full D; *retry asks
    // for more rounds with a tighter goal
    int finalize(bool* retry);
    int finalize_issue();
    int finalize_collect(bool* retry);
    // write x to the caller's buffer on the side stream (x_sent): the canonical
    // conversion and, for host x, the copy overlap the final check
    int send_x();
    bool x_sent = false;
    ~SolveState();
    // x back to the caller's layout, per-rhs info; returns the first failure
    int end(wl_solve_info* info);
};

}  // namespace wl
