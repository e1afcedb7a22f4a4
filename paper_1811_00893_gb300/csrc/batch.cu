// Many independent lattices of uneven size solved together (the batched
// form of the Sec. 2 solve): every BiCGStab iteration of every lattice and
// right-hand side runs as seven launches for the whole batch.
//
// * Hopping term: one persistent kernel.  Its blocks pull work items (a tile
//   of 32 output sites of one lattice, all of that lattice's right-hand
//   sides) from an atomic counter until the batch is exhausted; each item's
//   links are staged in shared memory once for all right-hand sides.  Dot
//   products are written per item and added up, item by item in a fixed
//   order, by a finishing launch; the last block to leave resets the
//   counter.  No block ever waits for another.
// * Vector updates: one launch per update, grid.y = system (lattice, rhs).
// * FP64 work (residuals, reliable updates, reconstruction) stays per lattice
//   through the single-lattice path, on the lattice's own stream, so that
//   the lattices' steps run side by side; between its rounds a lattice's
//   systems are inactive and the batched kernels skip them.
#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>

#include "hop.cuh"
#include "solver.cuh"

namespace wl {

static constexpr int kMaxBatchRhs = 32;
static constexpr int kMaxBatchLat = 64;

struct BLat {
    Geom g;
    const void* links[2];
    double kappa2;
    int nrhs;
    int item0;   // first hop work item of this lattice
    int nitems;  // 32-site tiles of one parity
    int chunks;  // vector-kernel blocks of one parity
    char *r, *rh, *p, *v, *s, *t, *xlo, *tmp;
    long long vb;  // bytes of one rhs vector (inner precision, one half field)
    long long xb;  // bytes of one rhs x_lo vector
    Scal* sc;
    const void* clov[2];  // clover term (Eq. 2) in the inner precision: A_ee, A_oo^-1 (or none)
};

struct BatchArgs {
    const BLat* lats;
    int nlat;
    const int2* sys;  // (lattice, rhs) of every system
    int nsys;
    int total_items;
    unsigned* queue;       // [0] next item, [1] blocks finished
    double* item_partial;  // [item][kMaxBatchRhs][3]
    RedScratch red;        // one slot per system for the vector reductions
};

// OP 0: tmp = H_oe p   OP 1: v = p - k^2 H_eo tmp, (rhat, v)
// OP 2: tmp = H_oe s   OP 3: t = s - k^2 H_eo tmp, (s, t)
// CLOV: the batch holds clover lattices; for those, tmp = A_oo^-1 H_oe (.)
// and v (t) = A_ee p (s) - k^2 H_eo tmp (a block-uniform branch per item).
template <int P, int OP, bool CLOV>
__global__ void __launch_bounds__(256) batch_hop_kernel(const BatchArgs B)
{
    using T = typename Prec<P>::real;
    constexpr bool DOT = (OP & 1) != 0;
    constexpr int par = DOT ? 0 : 1;  // output parity
    extern __shared__ __align__(16) char smem[];
    double* bpart = (double*)(smem + Prec<P>::link_bytes * kTile);
    __shared__ int s_item, s_lat, s_any;
    __shared__ bool last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const int lane = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const int it = (int)atomicAdd(&B.queue[0], 1u);
            int lo = 0, hi = B.nlat - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (B.lats[mid].item0 <= it) lo = mid;
                else hi = mid - 1;
            }
            s_item = it;
            s_lat = lo;
            // a lattice whose systems are all inactive (converged, or between
            // rounds) needs neither its links nor any arithmetic
            int any = 0;
            if (it < B.total_items) {
                const BLat& Lq = B.lats[lo];
                for (int r = 0; r < Lq.nrhs && !any; ++r) any = Lq.sc[r].active != 0;
                // move the counter past the rest of an idle lattice's items at
                // once (every item in between belongs to it)
                if (!any) atomicMax(&B.queue[0], (unsigned)(Lq.item0 + Lq.nitems));
            }
            s_any = any;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= B.total_items) break;
        if (!s_any) {  // (its partial sums are never read: the finishing launch skips inactive systems)
            __syncthreads();
            continue;
        }
        const BLat& L = B.lats[s_lat];
        const int base = (item - L.item0) * kTile;
        const int n = (int)min((long long)kTile, L.g.Vh - base);
        stage_links<P>(smem, (const char*)L.links[par], L.g.Vh, base, n);
        __syncthreads();
        const int i = base + lane;
        const bool valid = lane < n;
        int nb[8];
        if (valid) neighbours(L.g, par, i, nb);
        for (int r = threadIdx.y; r < L.nrhs; r += blockDim.y) {
            const bool act = L.sc[r].active != 0;  // warp-uniform
            T part[3] = {0, 0, 0};
            if (act && valid) {
                const long long o = r * L.vb;
                const char* in;
                char* out;
                const char *x1 = nullptr, *w = nullptr;
                double a = 1.0;
                if (OP == 0) {
                    in = L.p + o;
                    out = L.tmp + o;
                } else if (OP == 1) {
                    in = L.tmp + o;
                    out = L.v + o;
                    x1 = L.p + o;
                    w = L.rh + o;
                    a = -L.kappa2;
                } else if (OP == 2) {
                    in = L.s + o;
                    out = L.tmp + o;
                } else {
                    in = L.tmp + o;
                    out = L.t + o;
                    x1 = L.s + o;
                    w = L.s + o;
                    a = -L.kappa2;
                }
                cx<T> acc[12];
                hop_site<P, false>(acc, nb, L.g.Vh, in, smem, kTile, lane);
                if (CLOV && L.clov[0]) {
                    if (DOT)
                        epilogue_ptrs<P, DOT, kClX2>(acc, a, nullptr, x1, 1.0, w, out, L.g.Vh, i, part,
                                                     L.clov[0]);
                    else
                        epilogue_ptrs<P, DOT, kClOut>(acc, a, nullptr, nullptr, 0.0, nullptr, out, L.g.Vh,
                                                      i, part, L.clov[1]);
                } else {
                    epilogue_ptrs<P, DOT>(acc, a, x1, nullptr, 0.0, w, out, L.g.Vh, i, part);
                }
            }
            if (DOT) {
                typename RedType<T>::type rp[3] = {(typename RedType<T>::type)part[0],
                                                   (typename RedType<T>::type)part[1],
                                                   (typename RedType<T>::type)part[2]};
                warp_sum<3>(rp);
                if (lane == 0)
                    for (int k = 0; k < 3; ++k) bpart[3 * r + k] = (double)rp[k];
            }
        }
        __syncthreads();
        if (DOT)
            for (int e = tid; e < 3 * L.nrhs; e += nt)
                B.item_partial[(long long)item * 3 * kMaxBatchRhs + e] = bpart[e];
        __syncthreads();  // the tile's shared memory is reused by the next item
    }
    // the last block out resets the work counter for the next launch (the
    // per-item partials are added up by batch_finish_kernel)
    __syncthreads();
    if (tid == 0) last = atomicAdd(&B.queue[1], 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && tid == 0) {
        B.queue[0] = 0;
        B.queue[1] = 0;
    }
}

// One block per system adds its lattice's per-item partials in item order:
// (rhat, v) for OP 1, (s, t) for OP 3.
template <int OP>
__global__ void __launch_bounds__(256) batch_finish_kernel(const BatchArgs B)
{
    const int2 ls = B.sys[blockIdx.x];
    const BLat& L = B.lats[ls.x];
    Scal& S = L.sc[ls.y];
    if (!S.active) return;
    __shared__ double sh[3 * 32];
    double v[3];
    sum_partials<3>(B.item_partial + ((long long)L.item0 * kMaxBatchRhs + ls.y) * 3, L.nitems, v,
                    3 * kMaxBatchRhs);
    block_sum<3>(v, sh);
    if (threadIdx.x == 0) {
        double* o = (OP == 1) ? S.rv : S.st;
        o[0] = v[0];
        o[1] = v[1];
        o[2] = v[2];
    }
}

template <int P>
__global__ void __launch_bounds__(256) batch_update_p_kernel(const BatchArgs B)
{
    const int2 ls = B.sys[blockIdx.y];
    const BLat& L = B.lats[ls.x];
    const Scal& S = L.sc[ls.y];
    if (!S.active || (int)blockIdx.x >= L.chunks) return;
    __shared__ double coef[4];
    if (threadIdx.x == 0) {
        double c[4];
        beta_omega(S, c);
        for (int k = 0; k < 4; ++k) coef[k] = c[k];
    }
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= L.g.Vh) return;
    const long long o = ls.y * L.vb;
    const double c[4] = {coef[0], coef[1], coef[2], coef[3]};
    p_update_site<P>(L.p + o, L.r + o, L.v + o, L.g.Vh, i, c);
}

template <int P>
__global__ void __launch_bounds__(256) batch_update_s_kernel(const BatchArgs B)
{
    const int2 ls = B.sys[blockIdx.y];
    const BLat& L = B.lats[ls.x];
    const Scal& S = L.sc[ls.y];
    if (!S.active || (int)blockIdx.x >= L.chunks) return;
    __shared__ double coef[2];
    if (threadIdx.x == 0) {
        const cx<double> al = safe_alpha(S);
        coef[0] = al.re;
        coef[1] = al.im;
    }
    __syncthreads();
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= L.g.Vh) return;
    const long long o = ls.y * L.vb;
    s_update_site<P>(L.s + o, L.r + o, L.v + o, L.g.Vh, i, {coef[0], coef[1]});
}

template <int P, int PX>
__global__ void __launch_bounds__(256) batch_update_xr_kernel(const BatchArgs B)
{
    const int2 ls = B.sys[blockIdx.y];
    const BLat& L = B.lats[ls.x];
    Scal& S = L.sc[ls.y];
    if (!S.active || (int)blockIdx.x >= L.chunks) return;
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
    const double dc[4] = {dcoef[0], dcoef[1], dcoef[2], dcoef[3]};
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    using T = typename Prec<P>::real;
    T pt[3] = {0, 0, 0};
    if (i < L.g.Vh) {
        const long long o = ls.y * L.vb;
        xr_update_site<P, PX>(L.xlo + ls.y * L.xb, L.r + o, L.p + o, L.s + o, L.t + o, L.rh + o,
                              L.g.Vh, i, dc, pt);
    }
    // warp totals in the arithmetic type (FP32 for the narrow types), FP64 from there
    typename RedType<T>::type wp[3] = {(typename RedType<T>::type)pt[0], (typename RedType<T>::type)pt[1],
                                       (typename RedType<T>::type)pt[2]};
    warp_sum<3>(wp);
    double part[3] = {(double)wp[0], (double)wp[1], (double)wp[2]};
    block_sum_warps<3>(part, sh);
    double tot[3];
    if (grid_sum<3>(part, tot, B.red, blockIdx.y, L.chunks, blockIdx.x, sh))
        advance_scalars(S, tot, dc);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct BatchCtx {
    std::vector<wl_gauge> gs;
    std::vector<BLat> lats_h;
    int P = -1, xprec = 0, nlat = 0, nsys = 0, total_items = 0, max_chunks = 0;
    int lanes = 0, grid = 0, sms = 0;
    bool clover = false;  // some lattice of the batch has a clover term
    BLat* lats = nullptr;
    int2* sys = nullptr;
    unsigned* queue = nullptr;
    double* item_partial = nullptr;
    RedScratch red = {nullptr, nullptr, 0};
    double bytes_per_iter = 0.0;
    cudaGraphExec_t graph = nullptr;
    int graph_k = 0;
    long long graph_kernels = 0, graph_bytes = 0;
    cudaStream_t cap = nullptr;

    ~BatchCtx()
    {
        void* d[] = {lats, sys, queue, item_partial, red.partial, red.ticket};
        for (void* q : d)
            if (q) cudaFree(q);
        if (graph) cudaGraphExecDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
};

// Device descriptions of recent batches, most recently used last, found again
// by their gauge objects and workspaces: callers that alternate between
// batches reuse theirs instead of rebuilding (and synchronising the device).
static std::mutex g_batch_mu;
static std::vector<std::shared_ptr<BatchCtx>> g_batches;
static const size_t kBatchCache = 8;

BatchArgs args_of(const BatchCtx& C)
{
    BatchArgs a;
    a.lats = C.lats;
    a.nlat = C.nlat;
    a.sys = C.sys;
    a.nsys = C.nsys;
    a.total_items = C.total_items;
    a.queue = C.queue;
    a.item_partial = C.item_partial;
    a.red = C.red;
    return a;
}

template <int P, bool CLOV>
static void launch_batch_hop_c(const BatchCtx& C, int op, cudaStream_t s)
{
    const BatchArgs a = args_of(C);
    const dim3 block(kTile, C.lanes);
    const size_t smem = link_field_bytes(P, kTile) + sizeof(double) * 3 * kMaxBatchRhs;
    switch (op) {
        case 0: batch_hop_kernel<P, 0, CLOV><<<C.grid, block, smem, s>>>(a); break;
        case 1: batch_hop_kernel<P, 1, CLOV><<<C.grid, block, smem, s>>>(a); break;
        case 2: batch_hop_kernel<P, 2, CLOV><<<C.grid, block, smem, s>>>(a); break;
        default: batch_hop_kernel<P, 3, CLOV><<<C.grid, block, smem, s>>>(a); break;
    }
}

template <int P>
static void launch_batch_hop(const BatchCtx& C, int op, cudaStream_t s)
{
    if (C.clover) launch_batch_hop_c<P, true>(C, op, s);
    else launch_batch_hop_c<P, false>(C, op, s);
}

static void hop_dispatch(const BatchCtx& C, int op, cudaStream_t s)
{
    if (C.P == WL_F64) launch_batch_hop<WL_F64>(C, op, s);
    else if (C.P == WL_F32) launch_batch_hop<WL_F32>(C, op, s);
    else launch_batch_hop<WL_F16>(C, op, s);
}

// Resident blocks per SM of the persistent hopping kernel for `lanes` warps.
static int persistent_grid(const BatchCtx& C, int lanes)
{
    const size_t smem = link_field_bytes(C.P, kTile) + sizeof(double) * 3 * kMaxBatchRhs;
    int per_sm = 0;
    cudaError_t e;
    const void* k;
    if (C.P == WL_F64)
        k = C.clover ? (const void*)batch_hop_kernel<WL_F64, 1, true> : (const void*)batch_hop_kernel<WL_F64, 1, false>;
    else if (C.P == WL_F32)
        k = C.clover ? (const void*)batch_hop_kernel<WL_F32, 1, true> : (const void*)batch_hop_kernel<WL_F32, 1, false>;
    else
        k = C.clover ? (const void*)batch_hop_kernel<WL_F16, 1, true> : (const void*)batch_hop_kernel<WL_F16, 1, false>;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTile * lanes, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * C.sms;
}

// Pick the right-hand-side lanes of the persistent kernel by timing the
// first hopping operation (tmp = H p, which only writes a temporary).
static int tune_batch(BatchCtx& C, cudaStream_t s)
{
    int maxr = 1;
    for (const BLat& L : C.lats_h) maxr = std::max(maxr, L.nrhs);
    std::vector<int> cand;
    for (int l : {1, 2, 4, 8})
        if (l <= maxr || l == 1) cand.push_back(l);
    C.lanes = std::min(maxr, 8);
    C.grid = persistent_grid(C, C.lanes);
    if (is_capturing(s)) return WL_OK;
    const char* e = getenv("WL_AUTOTUNE");
    if (e && e[0] == '0') return WL_OK;
    cudaEvent_t e0, e1;
    WL_CUDA(cudaEventCreate(&e0));
    WL_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_l = C.lanes;
    for (int l : cand) {
        C.lanes = l;
        C.grid = persistent_grid(C, l);
        hop_dispatch(C, 0, s);
        WL_CHECK_LAUNCH(0.0);
        float t = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            hop_dispatch(C, 0, s);
            cudaEventRecord(e1, s);
            WL_CHECK_LAUNCH(0.0);
            WL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, ms);
        }
        if (t < best) {
            best = t;
            best_l = l;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    C.lanes = best_l;
    C.grid = persistent_grid(C, best_l);
    return WL_OK;
}

static int enqueue_batch_iteration(const BatchCtx& C, cudaStream_t s)
{
    const BatchArgs a = args_of(C);
    const dim3 vgrid((unsigned)C.max_chunks, (unsigned)C.nsys);
    const double per_op = C.bytes_per_iter / 7.0;  // accounting only
    auto vec = [&](int which) -> int {
        switch (C.P) {
            case WL_F64:
                if (which == 0) batch_update_p_kernel<WL_F64><<<vgrid, kBlock, 0, s>>>(a);
                else if (which == 1) batch_update_s_kernel<WL_F64><<<vgrid, kBlock, 0, s>>>(a);
                else batch_update_xr_kernel<WL_F64, WL_F64><<<vgrid, kBlock, 0, s>>>(a);
                break;
            case WL_F32:
                if (which == 0) batch_update_p_kernel<WL_F32><<<vgrid, kBlock, 0, s>>>(a);
                else if (which == 1) batch_update_s_kernel<WL_F32><<<vgrid, kBlock, 0, s>>>(a);
                else batch_update_xr_kernel<WL_F32, WL_F32><<<vgrid, kBlock, 0, s>>>(a);
                break;
            default:
                if (which == 0) batch_update_p_kernel<WL_F16><<<vgrid, kBlock, 0, s>>>(a);
                else if (which == 1) batch_update_s_kernel<WL_F16><<<vgrid, kBlock, 0, s>>>(a);
                else batch_update_xr_kernel<WL_F16, WL_F32><<<vgrid, kBlock, 0, s>>>(a);
                break;
        }
        WL_CHECK_LAUNCH(per_op);
        return WL_OK;
    };
    auto hop = [&](int op) -> int {
        hop_dispatch(C, op, s);
        WL_CHECK_LAUNCH(per_op);
        if (op == 1) batch_finish_kernel<1><<<C.nsys, 256, 0, s>>>(a);
        if (op == 3) batch_finish_kernel<3><<<C.nsys, 256, 0, s>>>(a);
        if (op & 1) WL_CHECK_LAUNCH(0.0);
        return WL_OK;
    };
    WL_TRY(vec(0));
    WL_TRY(hop(0));
    WL_TRY(hop(1));
    WL_TRY(vec(1));
    WL_TRY(hop(2));
    WL_TRY(hop(3));
    return vec(2);
}

static int run_batch_chunk(BatchCtx& C, int k, bool use_graph, cudaStream_t s)
{
    if (!use_graph) {
        for (int it = 0; it < k; ++it) WL_TRY(enqueue_batch_iteration(C, s));
        return WL_OK;
    }
    if (!C.graph || C.graph_k != k) {
        if (C.graph) cudaGraphExecDestroy(C.graph);
        C.graph = nullptr;
        if (!C.cap) WL_CUDA(cudaStreamCreateWithFlags(&C.cap, cudaStreamNonBlocking));
        const long long c0 = g_launches.load(), b0 = g_bytes.load();
        WL_CUDA(cudaStreamBeginCapture(C.cap, cudaStreamCaptureModeThreadLocal));
        int rc = WL_OK;
        for (int it = 0; it < k && rc == WL_OK; ++it) rc = enqueue_batch_iteration(C, C.cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(C.cap, &graph);
        if (rc != WL_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return set_error(WL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        C.graph_kernels = g_launches.load() - c0;
        C.graph_bytes = g_bytes.load() - b0;
        g_launches.fetch_sub(C.graph_kernels);
        g_bytes.fetch_sub(C.graph_bytes);
        e = cudaGraphInstantiate(&C.graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return set_error(WL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        C.graph_k = k;
    }
    WL_CUDA(cudaGraphLaunch(C.graph, s));
    count_launch(C.graph_kernels, (double)C.graph_bytes);
    return WL_OK;
}

// Build (or reuse) the device description of the batch.
static int batch_context(const std::vector<SolveState>& st, int P, std::shared_ptr<BatchCtx>* out)
{
    std::vector<BLat> lats(st.size());
    int item = 0, nsys = 0, max_chunks = 1;
    double bytes = 0.0;
    for (size_t l = 0; l < st.size(); ++l) {
        const SolveState& S = st[l];
        BLat& L = lats[l];
        std::memset(&L, 0, sizeof(BLat));
        L.g = S.g->geo;
        L.links[0] = S.g->links[P][0];
        L.links[1] = S.g->links[P][1];
        L.kappa2 = S.g->kappa * S.g->kappa;
        L.nrhs = S.nrhs;
        L.item0 = item;
        L.nitems = (int)((L.g.Vh + kTile - 1) / kTile);
        L.chunks = (int)((L.g.Vh + kBlock - 1) / kBlock);
        L.r = (char*)S.w->r;
        L.rh = (char*)S.w->rh;
        L.p = (char*)S.w->p;
        L.v = (char*)S.w->v;
        L.s = (char*)S.w->s;
        L.t = (char*)S.w->t;
        L.xlo = (char*)S.w->xlo;
        L.tmp = (char*)S.w->tmp;
        L.vb = (long long)S.w->vb;
        L.xb = (long long)spinor_field_bytes(S.w->xlo_prec, L.g.Vh);
        L.sc = S.w->sc;
        if (S.g->has_clover) {
            L.clov[0] = S.g->clov[P][0][0];
            L.clov[1] = S.g->clov[P][1][1];
        }
        item += L.nitems;
        nsys += L.nrhs;
        max_chunks = std::max(max_chunks, L.chunks);
        // one iteration: 4 hopping passes (links once) + the vector passes
        bytes += (double)L.g.Vh *
                 (4.0 * (link_field_bytes(P, 1) + (L.clov[0] ? clover_site_bytes(P) : 0.0)) +
                  L.nrhs * ((2 + 4 + 2 + 4 + 12) * (double)spinor_field_bytes(P, 1) +
                            2.0 * spinor_field_bytes(S.w->xlo_prec, 1)));
    }
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        for (size_t k = 0; k < g_batches.size(); ++k) {
            BatchCtx* C = g_batches[k].get();
            if (C->P == P && C->lats_h.size() == lats.size() &&
                std::memcmp(C->lats_h.data(), lats.data(), sizeof(BLat) * lats.size()) == 0) {
                std::shared_ptr<BatchCtx> keep = g_batches[k];
                g_batches.erase(g_batches.begin() + (long)k);
                g_batches.push_back(keep);
                *out = keep;
                return WL_OK;
            }
        }
    }
    std::shared_ptr<BatchCtx> fresh = std::make_shared<BatchCtx>();
    BatchCtx* C = fresh.get();
    C->lats_h = lats;
    for (const SolveState& S : st) C->gs.push_back(S.g);
    C->P = P;
    for (const BLat& L : lats) C->clover |= L.clov[0] != nullptr;
    C->nlat = (int)lats.size();
    C->nsys = nsys;
    C->total_items = item;
    C->max_chunks = max_chunks;
    C->bytes_per_iter = bytes;
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_CUDA(cudaDeviceGetAttribute(&C->sms, cudaDevAttrMultiProcessorCount, dev));
    std::vector<int2> sys;
    for (int l = 0; l < C->nlat; ++l)
        for (int r = 0; r < lats[l].nrhs; ++r) sys.push_back(make_int2(l, r));
    WL_CUDA(cudaMalloc((void**)&C->lats, sizeof(BLat) * lats.size()));
    WL_CUDA(cudaMemcpy(C->lats, lats.data(), sizeof(BLat) * lats.size(), cudaMemcpyHostToDevice));
    WL_CUDA(cudaMalloc((void**)&C->sys, sizeof(int2) * sys.size()));
    WL_CUDA(cudaMemcpy(C->sys, sys.data(), sizeof(int2) * sys.size(), cudaMemcpyHostToDevice));
    WL_CUDA(cudaMalloc((void**)&C->queue, 2 * sizeof(unsigned)));
    WL_CUDA(cudaMemset(C->queue, 0, 2 * sizeof(unsigned)));
    WL_CUDA(cudaMalloc((void**)&C->item_partial, sizeof(double) * 3 * kMaxBatchRhs * (size_t)item));
    WL_CUDA(cudaMalloc((void**)&C->red.partial, sizeof(double) * 4 * (size_t)nsys * max_chunks));
    WL_CUDA(cudaMalloc((void**)&C->red.ticket, sizeof(unsigned) * nsys));
    WL_CUDA(cudaMemset(C->red.ticket, 0, sizeof(unsigned) * nsys));
    C->red.max_blocks = max_chunks;
    {
        // the least recently used context leaves the cache (its device memory
        // is freed once no solve uses it any more)
        std::lock_guard<std::mutex> lock(g_batch_mu);
        if (g_batches.size() >= kBatchCache) g_batches.erase(g_batches.begin());
        g_batches.push_back(fresh);
    }
    *out = fresh;
    return WL_OK;
}

}  // namespace wl

using namespace wl;

// Drop the cached batch contexts that refer to a gauge object being destroyed
// (the caller has synchronised the device).
void batch_forget(wl_gauge g)
{
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (size_t k = 0; k < g_batches.size();) {
        const auto& gs = g_batches[k]->gs;
        if (std::find(gs.begin(), gs.end(), g) != gs.end()) g_batches.erase(g_batches.begin() + (long)k);
        else ++k;
    }
}

extern "C" int wilson_solve_batch(int nlat, const wl_gauge* gs, double* const* x,
                                  const double* const* b, const int* nrhs,
                                  const wl_solve_params* prm, wl_solve_info* info, void* stream)
{
    WL_ENTRY();
    if (nlat < 1 || nlat > kMaxBatchLat) return set_error(WL_ERR_ARG, "nlat must be in 1..64");
    if (!gs || !x || !b || !nrhs || !prm || !info) return set_error(WL_ERR_ARG, "NULL pointer");
    if (!prm->eo) return set_error(WL_ERR_ARG, "batched solves use the even-odd system (eo = 1)");
    for (int l = 0; l < nlat; ++l) {
        if (nrhs[l] < 1 || nrhs[l] > kMaxBatchRhs)
            return set_error(WL_ERR_ARG, "each lattice of a batch takes 1..32 right-hand sides");
        for (int m = 0; m < l; ++m)
            if (gs[m] == gs[l]) return set_error(WL_ERR_ARG, "a gauge object appears twice in the batch");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Each lattice's own work (set-up, FP64 residuals, final check) runs on its
    // workspace's lane stream, so that the lattices' outer work overlaps on the
    // GPU: every such step is issued for all lattices before the host waits
    // for any of them.  The batched iterations run on s once every lane has
    // been joined; the host waits for each chunk before the lanes go on.
    std::vector<SolveState> st(nlat);
    for (int l = 0; l < nlat; ++l) WL_TRY(st[l].begin_issue(gs[l], x[l], b[l], nrhs[l], prm, s, true));
    for (int l = 0; l < nlat; ++l) {
        WL_CUDA(cudaStreamSynchronize(st[l].s));
        st[l].begin_collect();
    }
    std::shared_ptr<BatchCtx> ctx;
    WL_TRY(batch_context(st, prm->inner, &ctx));
    BatchCtx* C = ctx.get();
    enum { PLAN, ITER, FINAL, DONE };
    std::vector<int> phase(nlat, PLAN);
    const int chunk = st[0].chunk;
    const bool use_graph = st[0].use_graph;
    // end the round of every lattice in `ending` (its steps issued for all first)
    auto end_rounds = [&](const std::vector<int>& ending) -> int {
        std::vector<char> pending(nlat, 0);
        for (int l : ending) {
            bool p = false;
            WL_TRY(st[l].finish_round_issue(&p));
            pending[l] = p;
        }
        for (int l : ending) {
            if (pending[l]) {
                WL_CUDA(cudaStreamSynchronize(st[l].s));
                st[l].finish_round_collect();
            }
            phase[l] = PLAN;
        }
        return WL_OK;
    };
    for (;;) {
        for (int l = 0; l < nlat; ++l)
            if (phase[l] == PLAN) {
                bool any = false;
                WL_TRY(st[l].plan(&any));
                phase[l] = any ? ITER : FINAL;
            }
        {
            std::vector<int> fin;
            for (int l = 0; l < nlat; ++l)
                if (phase[l] == FINAL) fin.push_back(l);
            for (int l : fin) WL_TRY(st[l].finalize_issue());
            for (int l : fin) {
                WL_CUDA(cudaStreamSynchronize(st[l].s));
                bool retry = false;
                WL_TRY(st[l].finalize_collect(&retry));
                phase[l] = retry ? PLAN : DONE;
            }
        }
        bool all_done = true, any_iter = false;
        for (int l = 0; l < nlat; ++l) {
            all_done &= phase[l] == DONE;
            any_iter |= phase[l] == ITER;
        }
        if (all_done) break;
        if (!any_iter) continue;
        // within every lattice's iteration cap; as long as the lattice that
        // predicts the most iterations needs (the others skip once done)
        int k = chunk, wanted = 0;
        for (int l = 0; l < nlat; ++l)
            if (phase[l] == ITER) {
                k = std::min(k, st[l].cap());
                wanted = std::max(wanted, st[l].want());
            }
        if (wanted > 0) k = std::min(k, wanted);
        if (k <= 0) {  // a lattice ran out of iterations: end its round
            std::vector<int> ending;
            for (int l = 0; l < nlat; ++l)
                if (phase[l] == ITER && st[l].cap() <= 0) ending.push_back(l);
            WL_TRY(end_rounds(ending));
            continue;
        }
        // the chunk reads every lattice's fields and scalars: after all lane work
        for (int l = 0; l < nlat; ++l) WL_TRY(stream_join(s, st[l].s, st[l].w->ev_lane));
        if (C->lanes == 0) WL_TRY(tune_batch(*C, s));  // with the first round's systems active
        WL_TRY(run_batch_chunk(*C, k, use_graph && k == chunk, s));
        for (int l = 0; l < nlat; ++l)
            if (phase[l] == ITER)
                WL_CUDA(cudaMemcpyAsync(st[l].w->sc_h, st[l].w->sc, sizeof(Scal) * st[l].nrhs,
                                        cudaMemcpyDeviceToHost, s));
        WL_CUDA(cudaStreamSynchronize(s));  // (the lanes' next work follows the chunk)
        std::vector<int> ending;
        for (int l = 0; l < nlat; ++l) {
            if (phase[l] != ITER) continue;
            bool alive = false;
            WL_TRY(st[l].after_chunk(&alive));
            if (!alive) ending.push_back(l);
        }
        WL_TRY(end_rounds(ending));
    }
    int rc = WL_OK, off = 0;
    for (int l = 0; l < nlat; ++l) {
        const int r = st[l].end(info + off);
        if (r != WL_OK && rc == WL_OK) rc = r;
        off += nrhs[l];
    }
    if (rc != WL_OK) set_error(rc, "at least one right-hand side of the batch did not reach tol");
    return rc;
}
