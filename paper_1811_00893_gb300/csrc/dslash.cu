// Host side of the hopping term: launch shapes, the autotuner, right-hand-side
// chunking and the C entry points wilson_dslash / wilson_mult.  The kernels
// are in hop_kernels.cuh.  The epilogue optionally forms
// out = x1 + b1*x2 + a*H in (with the clover term of Eq. 2 folded in) and
// accumulates the complex dot (w, out) and ||out||^2 into a deterministic
// grid reduction, so the solver's matrix applies carry their reductions for
// free.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "hop_kernels.cuh"

namespace wl {

// the other variants are instantiated in their own translation units:
// clover modes in dslash_clover_x2.cu / dslash_clover_out.cu, compressed links
// (LF = 1) in dslash_r12.cu / dslash_r12_clover.cu
extern template struct HopKernels<kClX2, 0>;
extern template struct HopKernels<kClOut, 0>;
extern template struct HopKernels<kClNone, 1>;
extern template struct HopKernels<kClX2, 1>;
extern template struct HopKernels<kClOut, 1>;
extern template struct HopKernels<kClNone, 2>;  // dslash_r8.cu

// The kernel family of a launch: clover mode and link format.
template <typename F>
static void with_variant(const HopLaunch& h, int lf, F&& f)
{
    if (lf == 2) {  // eight-real links: Wilson launches only
        f(HopKernels<kClNone, 2>());
    } else if (lf) {
        switch (h.cl_mode) {
            case kClX2: f(HopKernels<kClX2, 1>()); break;
            case kClOut: f(HopKernels<kClOut, 1>()); break;
            default: f(HopKernels<kClNone, 1>()); break;
        }
    } else {
        switch (h.cl_mode) {
            case kClX2: f(HopKernels<kClX2, 0>()); break;
            case kClOut: f(HopKernels<kClOut, 0>()); break;
            default: f(HopKernels<kClNone, 0>()); break;
        }
    }
}

// Bytes of the links of one site (all eight hops) in the launch's format.
static size_t link_site_bytes(int prec, int lf)
{
    if (lf == 2) return 256;
    if (lf) return prec == WL_F32 ? 384 : 192;
    return link_field_bytes(prec, 1);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static const int kHopBlock = 128;

static void launch_single(const HopLaunch& h, int lf, const HopArgs& A, dim3 grid, int block,
                          cudaStream_t s)
{
    with_variant(h, lf, [&](auto K) { K.single(h.prec, h.dagger, h.dot, A, grid, block, s); });
}

static void launch_multi(const HopLaunch& h, int lf, const HopArgs& A, int nrhs, dim3 grid, dim3 block,
                         size_t smem, cudaStream_t s)
{
    with_variant(h, lf, [&](auto K) { K.multi(h.prec, h.dagger, h.dot, A, nrhs, grid, block, smem, s); });
}

static void launch_pipe(const HopLaunch& h, int lf, const HopArgs& A, int nrhs, int ntiles, dim3 grid,
                        dim3 block, size_t smem, cudaStream_t s)
{
    with_variant(h, lf, [&](auto K) { K.pipe(h.prec, h.dagger, h.dot, A, nrhs, ntiles, grid, block, smem, s); });
}

static const void* pipe_kernel(const HopLaunch& h, int lf)
{
    const void* k = nullptr;
    with_variant(h, lf, [&](auto K) { k = K.pipe_kernel(h.prec, h.dagger, h.dot); });
    return k;
}

// Multi-RHS launch shapes: 1..8 = right-hand-side lanes (warps) of
// hop_mrhs_kernel; kPipeShape + lanes = the pipelined persistent kernel.
static const int kPipeShape = 16;
// Single-RHS reducing launches: block size (grid of resident blocks), or
// kFullGrid + block size (full grid and a finishing launch).
static const int kFullGrid = 1000;
// Single-RHS FP64 Wilson launches: three threads per site (hop_rows_kernel).
static const int kRowsShape = 2000;
// Multi-RHS launches of the wide types: kPerRhs + block size = the single-RHS
// kernel with one grid row per right-hand side (grid.y), links read once per
// right-hand side (these launches are bound by arithmetic, not by bytes);
// reducing launches use the full grid and a finishing launch.
static const int kPerRhs = 3000;

static bool rows_allowed(const HopLaunch& h, int lf)
{
    return h.prec == WL_F64 && h.cl_mode == kClNone && lf == 0;
}

// Resident-block grid of the reducing single-RHS hop kernel.
static int single_grid_cap(const HopLaunch& h, int lf, int block)
{
    const void* k = nullptr;
    with_variant(h, lf, [&](auto K) { k = K.reducing(h.prec, h.dagger); });
    return resident_grid(k, block, 0);
}

// Launch one chunk of right-hand sides with launch shape `shape`: threads per
// block for the single-RHS kernel, right-hand-side lanes (warps) per block for
// the multi-RHS kernel.
static int launch_shape(const HopLaunch& h, int lf, HopArgs& A, int nrhs, int shape, cudaStream_t s)
{
    const bool multi = nrhs > 1;
    const int tile = multi ? kTile : shape;
    const long long bpp = (A.g.Vh + tile - 1) / tile;
    A.blocks_per_parity = (int)bpp;
    A.nparity = h.nparity;
    unsigned gx = (unsigned)(bpp * h.nparity);
    if (!multi && shape == kRowsShape) {
        A.blocks_per_parity = (int)((A.g.Vh + kRowSites - 1) / kRowSites);
        A.partials_only = h.dot ? 1 : 0;
        gx = (unsigned)((long long)A.blocks_per_parity * h.nparity);
        HopKernels<kClNone, 0>::rows(h.dagger != 0, h.dot, A, dim3(gx, 1), s);
        if (h.dot)
            return launch_finish_slots(A.red.partial, (long long)A.red.max_blocks * 3, (int)gx, 1, A.dot_out,
                                       A.dot_stride, A.active, A.active_stride, s);
    } else if (!multi) {
        // shapes above kFullGrid: the reducing kernel over the full grid, one
        // site per thread, with a finishing launch for the partial sums
        const bool full = shape > kFullGrid;
        const int block = full ? shape - kFullGrid : shape;
        A.partials_only = h.dot && full ? 1 : 0;
        A.blocks_per_parity = (int)((A.g.Vh + block - 1) / block);
        gx = (unsigned)((long long)A.blocks_per_parity * h.nparity);
        if (h.dot && !full) gx = std::min(gx, (unsigned)single_grid_cap(h, lf, block));
        launch_single(h, lf, A, dim3(gx, 1), block, s);
        if (A.partials_only)
            return launch_finish_slots(A.red.partial, (long long)A.red.max_blocks * 3, (int)gx, 1,
                                       A.dot_out, A.dot_stride, A.active, A.active_stride, s);
    } else if (shape > kPerRhs) {
        const int block = shape - kPerRhs;
        A.blocks_per_parity = (int)((A.g.Vh + block - 1) / block);
        gx = (unsigned)((long long)A.blocks_per_parity * h.nparity);
        A.partials_only = h.dot ? 1 : 0;
        launch_single(h, lf, A, dim3(gx, (unsigned)nrhs), block, s);
        if (h.dot)
            return launch_finish_slots(A.red.partial, (long long)A.red.max_blocks * 3, (int)gx, nrhs,
                                       A.dot_out, A.dot_stride, A.active, A.active_stride, s);
    } else if (shape > kPipeShape) {
        const dim3 block(kTile, shape - kPipeShape);
        const size_t smem = 2 * link_site_bytes(h.prec, lf) * kTile + sizeof(double) * 3 * nrhs;
        const int ntiles = (int)gx;
        const int grid = std::min(ntiles, resident_grid(pipe_kernel(h, lf), kTile * (shape - kPipeShape), smem));
        launch_pipe(h, lf, A, nrhs, ntiles, dim3((unsigned)grid), block, smem, s);
        if (h.dot)  // per-tile partials, added in tile order
            return launch_finish_slots(A.red.partial, (long long)A.red.max_blocks * 3, ntiles, nrhs,
                                       A.dot_out, A.dot_stride, A.active, A.active_stride, s);
    } else {
        const dim3 block(kTile, shape);
        const size_t smem = link_site_bytes(h.prec, lf) * kTile + sizeof(double) * 3 * nrhs;
        launch_multi(h, lf, A, nrhs, dim3(gx), block, smem, s);
        if (h.dot)  // add the per-block partials of each right-hand side
            return launch_finish_slots(A.red.partial, (long long)A.red.max_blocks * 3, (int)gx, nrhs,
                                       A.dot_out, A.dot_stride, A.active, A.active_stride, s);
    }
    return WL_OK;
}

static bool autotune_enabled()
{
    static const bool on = [] {
        const char* e = getenv("WL_AUTOTUNE");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Pick the launch shape for this kernel configuration: the cached choice, or
// (first use, outside stream capture) the fastest candidate timed with CUDA
// events on the launching stream.  Re-running a hopping launch is harmless:
// it is out of place and its reductions are recomputed from scratch.
static int tuned_shape(wl_gauge g, const HopLaunch& h, int lf, HopArgs& A, int nrhs, cudaStream_t s,
                       int* shape)
{
    const bool multi = nrhs > 1;
    const int dflt = multi ? (nrhs < 8 ? nrhs : 8) : kHopBlock;
    char key[96];
    snprintf(key, sizeof key, "hop p%d d%d dot%d np%d r%d x%d%d w%d c%d l%d", h.prec, h.dagger, (int)h.dot,
             h.nparity, nrhs, h.x1[0] != nullptr, h.x2[0] != nullptr, h.w[0] != nullptr, h.cl_mode, lf);
    auto it = g->tuned.find(key);
    if (it != g->tuned.end()) {
        *shape = it->second.block;
        return WL_OK;
    }
    *shape = dflt;
    if (!multi) {  // explicit override of the single-RHS shape (for sweeps and tests)
        const char* fb = getenv("WL_HOP_BLOCK");
        const int v = fb ? atoi(fb) : 0;
        const int b = v > kFullGrid ? v - kFullGrid : v;
        if (((b == 32 || b == 64 || b == 128 || b == 256) && (v < kFullGrid || h.dot)) ||
            (v == kRowsShape && rows_allowed(h, lf))) {
            *shape = v;
            return WL_OK;
        }
    } else {  // explicit override of the multi-RHS shape (for sweeps and tests)
        const char* fs = getenv("WL_MRHS_SHAPE");
        const int v = fs ? atoi(fs) : 0;
        const bool narrow = h.prec == WL_F32 || h.prec == WL_F16;
        const int pb = v - kPerRhs;
        if ((v >= 1 && v <= 8 && v <= nrhs) ||
            (narrow && v > kPipeShape && v <= kPipeShape + 8 && v - kPipeShape <= nrhs) ||
            pb == 64 || pb == 128 || pb == 256) {
            *shape = v;
            return WL_OK;
        }
    }
    if (!autotune_enabled() || is_capturing(s)) return WL_OK;
    std::vector<int> cand;
    if (multi) {
        for (int l : {1, 2, 4, 8})
            if (l <= nrhs) cand.push_back(l);
        if (h.prec == WL_F32 || h.prec == WL_F16) {
            for (int l : {2, 4, 8})
                if (l <= nrhs) cand.push_back(kPipeShape + l);
        } else {
            for (int b : {64, 128, 256}) cand.push_back(kPerRhs + b);
        }
    } else {
        // 32-thread blocks too on small launches, whose grids would otherwise
        // reach only some of the SMs
        const bool small = g->geo.Vh * h.nparity <= 65536;
        cand = {64, 128, 256};
        if (small) cand.push_back(32);
        if (h.dot) {
            for (int b : {64, 128, 256}) cand.push_back(kFullGrid + b);
            if (small) cand.push_back(kFullGrid + 32);
        }
        if (rows_allowed(h, lf)) cand.push_back(kRowsShape);
    }
    // the timings must not share the GPU with work on other streams (a
    // batch's lattices run their own steps side by side)
    WL_CUDA(cudaDeviceSynchronize());
    cudaEvent_t e0, e1;
    WL_CUDA(cudaEventCreate(&e0));
    WL_CUDA(cudaEventCreate(&e1));
    for (int c : cand) {  // warm every candidate once
        WL_TRY(launch_shape(h, lf, A, nrhs, c, s));
        WL_CHECK_LAUNCH(0.0);
    }
    // interleaved rounds so that a drifting clock or cache state affects every
    // candidate alike; each keeps its fastest round
    std::vector<float> best_t(cand.size(), 1e30f);
    for (int round = 0; round < 4; ++round)
        for (size_t ci = 0; ci < cand.size(); ++ci) {
            cudaEventRecord(e0, s);
            WL_TRY(launch_shape(h, lf, A, nrhs, cand[ci], s));
            cudaEventRecord(e1, s);
            WL_CHECK_LAUNCH(0.0);
            WL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_t[ci] = std::min(best_t[ci], ms);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    size_t bi = 0;
    for (size_t ci = 1; ci < cand.size(); ++ci)
        if (best_t[ci] < best_t[bi]) bi = ci;
    const int best_shape = cand[bi];
    if (getenv("WL_AUTOTUNE_VERBOSE")) {
        fprintf(stderr, "[wl autotune] %s Vh=%lld:", key, g->geo.Vh);
        for (size_t ci = 0; ci < cand.size(); ++ci) fprintf(stderr, " %d:%.1fus", cand[ci], best_t[ci] * 1e3f);
        fprintf(stderr, " -> %d\n", best_shape);
    }
    Tuned tv;
    tv.block = best_shape;
    g->tuned[key] = tv;
    *shape = best_shape;
    return WL_OK;
}

static int launch_hop_chunk(wl_gauge g, const HopLaunch& h, int lf, HopArgs A, int nrhs, cudaStream_t s)
{
    const bool multi = nrhs > 1;
    if (h.dot) {  // sized for the smallest tile any candidate shape uses
        const long long most = ((g->geo.Vh + 31) / 32) * h.nparity;
        WL_TRY(ensure_red(g, nrhs, most));
    }
    A.red = g->red;
    int shape = 0;
    WL_TRY(tuned_shape(g, h, lf, A, nrhs, s, &shape));
    (void)multi;
    // algorithmic bytes: links once for all rhs; in, out and epilogue fields per rhs
    // (and the clover matrix once, like the links)
    const int extra = (h.x1[0] ? 1 : 0) + (h.x2[0] ? 1 : 0) + (h.w[0] ? 1 : 0);
    const double bytes = (double)g->geo.Vh * h.nparity *
                         (link_site_bytes(h.prec, lf) + (h.cl_mode ? clover_site_bytes(h.prec) : 0) +
                          (double)nrhs * (2 + extra) * spinor_field_bytes(h.prec, 1));
    int slot = -1;
    timing_begin(g, s, bytes, h.prec, &slot);
    WL_TRY(launch_shape(h, lf, A, nrhs, shape, s));
    WL_CHECK_LAUNCH(bytes);
    timing_end(g, s, slot);
    return WL_OK;
}

int launch_hop(wl_gauge g, const HopLaunch& h, cudaStream_t s)
{
    if (!g->links[h.prec][0])
        return set_error(WL_ERR_STATE, "gauge object has no links in the requested precision");
    // compressed links when the gauge object holds them (WL_NO_R12 turns them
    // off, for comparisons)
    static const bool r12_off = getenv("WL_NO_R12") != nullptr;
    int lf = (h.prec == WL_F32 || h.prec == WL_F16) && g->links_r12[h.prec][0] && !r12_off ? 1 : 0;
    // eight-real links: FP32 single-RHS Wilson launches
    if (h.prec == WL_F32 && g->links_r8[WL_F32][0] && h.nrhs == 1 && h.cl_mode == kClNone && !r12_off) lf = 2;
    HopArgs A;
    A.g = g->geo;
    A.partials_only = 0;
    for (int k = 0; k < 2; ++k) {
        const int p = h.parity0 + (k < h.nparity ? k : 0);
        A.links[k] = lf == 2 ? g->links_r8[h.prec][p] : lf ? g->links_r12[h.prec][p] : g->links[h.prec][p];
        A.cl[k] = h.clov[k];
    }
    for (int mu = 0; mu < 4; ++mu) A.ph[mu] = {(float)g->bc_re[mu], (float)g->bc_im[mu]};
    if (h.cl_mode && (!h.clov[0] || (h.nparity == 2 && !h.clov[1])))
        return set_error(WL_ERR_STATE, "gauge object has no clover term in the requested precision");
    A.rs_in = h.rs_in;
    A.rs_out = h.rs_out;
    A.rs_x1 = h.rs_x1;
    A.rs_x2 = h.rs_x2;
    A.rs_w = h.rs_w;
    A.a = h.a;
    A.b1 = h.b1;
    A.parity0 = h.parity0;
    A.dot_stride = h.dot_stride;
    A.active_stride = h.active_stride;
    // right-hand sides go in chunks of at most kMaxRhsLaunch per launch
    for (int r0 = 0; r0 < h.nrhs; r0 += kMaxRhsLaunch) {
        const int n = h.nrhs - r0 < kMaxRhsLaunch ? h.nrhs - r0 : kMaxRhsLaunch;
        auto off = [&](const void* q, long long rs) -> const char* {
            return q ? (const char*)q + r0 * rs : nullptr;
        };
        for (int k = 0; k < 2; ++k) {
            A.in[k] = off(h.in[k], h.rs_in);
            A.out[k] = (char*)off(h.out[k], h.rs_out);
            A.x1[k] = off(h.x1[k], h.rs_x1);
            A.x2[k] = off(h.x2[k], h.rs_x2);
            A.w[k] = off(h.w[k], h.rs_w);
        }
        A.dot_out = h.dot_out ? h.dot_out + (long long)r0 * h.dot_stride : nullptr;
        A.active = h.active ? h.active + (long long)r0 * h.active_stride : nullptr;
        WL_TRY(launch_hop_chunk(g, h, lf, A, n, s));
    }
    return WL_OK;
}

}  // namespace wl

using namespace wl;

static int check_common(wl_gauge g, const void* out, const void* in, wl_prec prec, int nrhs)
{
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (g->dd_part) return set_error(WL_ERR_STATE, "block of a domain decomposition: use the _dd calls");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (nrhs < 1) return set_error(WL_ERR_ARG, "nrhs must be >= 1");
    if (nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be <= 65535");
    if (!out || !in) return set_error(WL_ERR_ARG, "NULL field pointer");
    if (!g->links[prec][0])
        return set_error(WL_ERR_STATE, "gauge object was created without this precision");
    const size_t fb = spinor_field_bytes(prec, g->geo.Vh);
    const char *o = (const char*)out, *i = (const char*)in;
    if (o < i + fb * nrhs && i < o + fb * nrhs) return set_error(WL_ERR_ARG, "out and in overlap");
    return WL_OK;
}

extern "C" int wilson_dslash(wl_gauge g, void* out, const void* in, int out_parity, int dagger,
                             wl_prec prec, int nrhs, void* stream)
{
    WL_ENTRY();
    WL_TRY(check_common(g, out, in, prec, nrhs));
    if (out_parity != 0 && out_parity != 1) return set_error(WL_ERR_ARG, "out_parity must be 0 or 1");
    const size_t fb = spinor_field_bytes(prec, g->geo.Vh);
    HopLaunch h;
    h.prec = prec;
    h.dagger = dagger ? 1 : 0;
    h.parity0 = out_parity;
    h.nparity = 1;
    h.nrhs = nrhs;
    h.in[0] = in;
    h.out[0] = out;
    h.rs_in = h.rs_out = (long long)fb;
    h.a = 1.0;
    return launch_hop(g, h, (cudaStream_t)stream);
}

extern "C" int wilson_mult(wl_gauge g, void* out, const void* in, int eo, int dagger, wl_prec prec,
                           int nrhs, void* stream)
{
    WL_ENTRY();
    WL_TRY(check_common(g, out, in, prec, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fb = spinor_field_bytes(prec, g->geo.Vh);
    const double kappa = g->kappa;
    if (!eo) {
        // full D on [even | odd] halves: out_p = in_p - kappa H in_{1-p}
        if ((const char*)out < (const char*)in + 2 * fb * nrhs &&
            (const char*)in < (const char*)out + 2 * fb * nrhs)
            return set_error(WL_ERR_ARG, "out and in overlap");
        HopLaunch h;
        h.prec = prec;
        h.dagger = dagger ? 1 : 0;
        h.parity0 = 0;
        h.nparity = 2;
        h.nrhs = nrhs;
        h.in[0] = (const char*)in + fb;   // even outputs read odd inputs
        h.in[1] = (const char*)in;
        h.out[0] = out;
        h.out[1] = (char*)out + fb;
        h.rs_in = h.rs_out = (long long)(2 * fb);
        h.a = -kappa;
        if (g->has_clover) {  // out_p = A_pp in_p - kappa H in_{1-p}
            h.x2[0] = in;
            h.x2[1] = (const char*)in + fb;
            h.rs_x2 = (long long)(2 * fb);
            h.b1 = 1.0;
            h.cl_mode = kClX2;
            h.clov[0] = g->clov[prec][0][0];
            h.clov[1] = g->clov[prec][1][0];
        } else {
            h.x1[0] = in;
            h.x1[1] = (const char*)in + fb;
            h.rs_x1 = (long long)(2 * fb);
        }
        return launch_hop(g, h, s);
    }
    // M_ee = 1 - kappa^2 H_eo H_oe on even half fields (A_ee - kappa^2 H_eo A_oo^-1 H_oe
    // with a clover term)
    WL_TRY(ensure_tmp(g, prec, fb * nrhs));
    HopLaunch h1;
    h1.prec = prec;
    h1.dagger = dagger ? 1 : 0;
    h1.parity0 = 1;
    h1.nrhs = nrhs;
    h1.in[0] = in;
    h1.out[0] = g->tmp[prec];
    h1.rs_in = h1.rs_out = (long long)fb;
    h1.a = 1.0;
    if (g->has_clover) {  // tmp = A_oo^-1 H_oe in
        h1.cl_mode = kClOut;
        h1.clov[0] = g->clov[prec][1][1];
    }
    WL_TRY(launch_hop(g, h1, s));
    HopLaunch h2 = h1;
    h2.parity0 = 0;
    h2.in[0] = g->tmp[prec];
    h2.out[0] = out;
    h2.a = -kappa * kappa;
    if (g->has_clover) {  // out = A_ee in - kappa^2 H_eo tmp
        h2.x2[0] = in;
        h2.rs_x2 = (long long)fb;
        h2.b1 = 1.0;
        h2.cl_mode = kClX2;
        h2.clov[0] = g->clov[prec][0][0];
    } else {
        h2.x1[0] = in;
        h2.rs_x1 = (long long)fb;
        h2.cl_mode = kClNone;
    }
    return launch_hop(g, h2, s);
}
