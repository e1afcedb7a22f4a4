// Host side of the domain decomposition (dd.cuh): the block objects, halo
// regions, the exchange of packed faces, the launch sequence of one
// decomposed hopping application (Sec. 4.4: pack -> exchange || interior ->
// boundary) and the sum of the blocks' local reductions.  Entry points:
// wl_dd_create / destroy / blocks / block / set_exchange, wl_dd_scatter /
// gather, wilson_dslash_dd, wilson_mult_dd, wl_cdot_dd.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dd_kernels.cuh"

namespace wl {

extern template struct DDKernels<0, kClNone>;  // dd_hop.cu
extern template struct DDKernels<1, kClNone>;  // dd_hop_r12.cu
extern template struct DDKernels<0, kClX2>;    // dd_hop_clover.cu
extern template struct DDKernels<0, kClOut>;
extern template struct DDKernels<1, kClX2>;    // dd_hop_r12_clover.cu
extern template struct DDKernels<1, kClOut>;

// the kernel family of a launch: link format and clover mode
static void dd_hop_family(int lf, int cl, int prec, bool dagger, bool dot, bool bnd, const DDArgs& A, dim3 grid,
                          cudaStream_t s)
{
    if (lf) {
        if (cl == kClX2) DDKernels<1, kClX2>::hop(prec, dagger, dot, bnd, A, grid, s);
        else if (cl == kClOut) DDKernels<1, kClOut>::hop(prec, dagger, dot, bnd, A, grid, s);
        else DDKernels<1, kClNone>::hop(prec, dagger, dot, bnd, A, grid, s);
    } else {
        if (cl == kClX2) DDKernels<0, kClX2>::hop(prec, dagger, dot, bnd, A, grid, s);
        else if (cl == kClOut) DDKernels<0, kClOut>::hop(prec, dagger, dot, bnd, A, grid, s);
        else DDKernels<0, kClNone>::hop(prec, dagger, dot, bnd, A, grid, s);
    }
}

// ---------------------------------------------------------------------------
// canonical global field <-> block-local canonical fields
// ---------------------------------------------------------------------------

struct Origin {
    int o[4];
};

// dir = 0: local <- global; dir = 1: global <- local; nd doubles per site
// (24: a spinor, 144: a clover matrix)
__global__ void dd_copy_canonical_kernel(double* loc, double* glob, Geom gl, Geom gg, Origin org,
                                         long long Vl, long long Vg, int dir, int nd)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (s >= Vl) return;
    long long r = s;
    int c[4];
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(r % gl.L[mu]) + org.o[mu];
        r /= gl.L[mu];
    }
    const long long sg = c[0] + (long long)gg.L[0] * (c[1] + (long long)gg.L[1] * (c[2] + (long long)gg.L[2] * c[3]));
    double2* pl = (double2*)(loc + ((long long)rhs * Vl + s) * nd);
    double2* pg = (double2*)(glob + ((long long)rhs * Vg + sg) * nd);
    if (dir == 0)
        for (int k = 0; k < nd / 2; ++k) pl[k] = pg[k];
    else
        for (int k = 0; k < nd / 2; ++k) pg[k] = pl[k];
}

// ---------------------------------------------------------------------------
// the exchange between blocks held here: one copy kernel over all faces
// ---------------------------------------------------------------------------

static constexpr int kCopySegs = 64;  // face copies per launch

struct DDCopies {
    const uint4* src[kCopySegs];
    uint4* dst[kCopySegs];
    long long n16[kCopySegs];  // 16-byte words of each copy
    long long start[kCopySegs + 1];  // prefix sums of n16
    int n;
};

// grid-stride over the concatenated copies (every face segment is a multiple
// of 16 bytes: 48 or 96 bytes per face site)
__global__ void __launch_bounds__(256) dd_copy_kernel(const DDCopies C)
{
    const long long total = C.start[C.n];
    for (long long j = blockIdx.x * 256LL + threadIdx.x; j < total; j += (long long)gridDim.x * 256) {
        int k = 0;
        while (k + 1 < C.n && j >= C.start[k + 1]) ++k;
        const long long o = j - C.start[k];
        C.dst[k][o] = __ldcs(C.src[k] + o);
    }
}

static int launch_copies(DDCopies& C, cudaStream_t s)
{
    if (C.n == 0) return WL_OK;
    C.start[0] = 0;
    for (int k = 0; k < C.n; ++k) C.start[k + 1] = C.start[k] + C.n16[k];
    const long long total = C.start[C.n];
    const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, 4 * 152);
    dd_copy_kernel<<<grid, 256, 0, s>>>(C);
    WL_CHECK_LAUNCH(32.0 * total);
    C.n = 0;
    return WL_OK;
}

// ---------------------------------------------------------------------------
// sums over the blocks
// ---------------------------------------------------------------------------

struct DDFinish {
    const double* partial;  // block partials (fused hop reductions), or
    const double* loc[kMaxDomains];  // per-block local 3-tuples (nblocks = 0)
    long long dom_stride;
    int max_blocks, nblocks, ndom;
    double* out[kMaxDomains];
    int out_stride;
    const int* active;  // right-hand-side flags (every block holds the same)
    int active_stride;
    // mode 0: write the total to every out; 1: write this process's total to
    // stage (summed over the processes next); 2: copy stage to every out
    int mode;
    double* stage;
};

// One block per right-hand side: the total over the held blocks, in block
// order (the allreduce when every block is held here), written for every
// block or staged for the sum over the processes.
__global__ void __launch_bounds__(256) dd_finish_kernel(const DDFinish F)
{
    const int rhs = blockIdx.x;
    if (F.active && !F.active[(long long)rhs * F.active_stride]) return;
    __shared__ double sh[3 * 32];
    double tot[3] = {0.0, 0.0, 0.0};
    if (F.mode == 2) {
        for (int k = 0; k < 3; ++k) tot[k] = F.stage[3 * rhs + k];
    } else {
        for (int d = 0; d < F.ndom; ++d) {
            double v[3];
            if (F.nblocks > 0) {
                sum_partials<3>(F.partial + d * F.dom_stride + (long long)rhs * F.max_blocks * 3, F.nblocks, v);
                block_sum<3>(v, sh);
            } else {
                for (int k = 0; k < 3; ++k) v[k] = F.loc[d][3 * rhs + k];
            }
            if (threadIdx.x == 0)
                for (int k = 0; k < 3; ++k) tot[k] += v[k];
        }
    }
    if (threadIdx.x != 0) return;
    if (F.mode == 1) {
        for (int k = 0; k < 3; ++k) F.stage[3 * rhs + k] = tot[k];
        return;
    }
    for (int d = 0; d < F.ndom; ++d)
        if (F.out[d])
            for (int k = 0; k < 3; ++k) F.out[d][(long long)rhs * F.out_stride + k] = tot[k];
}

int dd_ensure_stage(wl_dd dd, int nrhs)
{
    if (nrhs <= dd->stage_rhs) return WL_OK;
    WL_CUDA(cudaDeviceSynchronize());
    if (dd->stage) cudaFree(dd->stage);
    dd->stage = nullptr;
    WL_CUDA(cudaMalloc((void**)&dd->stage, sizeof(double) * 3 * nrhs));
    dd->stage_rhs = nrhs;
    return WL_OK;
}

int dd_cross_sum(wl_dd dd, int nrhs, cudaStream_t s)
{
    if (!dd->has_tr) return WL_OK;
    const int rc = dd->tr.allreduce(dd->tr.ctx, dd->stage, 3 * nrhs, (void*)s);
    if (rc != 0) return set_error(WL_ERR_CUDA, "transport allreduce failed");
    return WL_OK;
}

// Launch the finish kernel; with a transport, as local total -> sum over the
// processes -> copy to every held block.
static int dd_finish(wl_dd dd, DDFinish F, int nrhs, cudaStream_t s)
{
    if (!dd->has_tr) {
        F.mode = 0;
        dd_finish_kernel<<<nrhs, 256, 0, s>>>(F);
        WL_CHECK_LAUNCH(0.0);
        return WL_OK;
    }
    WL_TRY(dd_ensure_stage(dd, nrhs));
    F.stage = dd->stage;
    F.mode = 1;
    dd_finish_kernel<<<nrhs, 256, 0, s>>>(F);
    WL_CHECK_LAUNCH(0.0);
    WL_TRY(dd_cross_sum(dd, nrhs, s));
    F.mode = 2;
    dd_finish_kernel<<<nrhs, 256, 0, s>>>(F);
    WL_CHECK_LAUNCH(0.0);
    return WL_OK;
}

int dd_allreduce(wl_dd dd, double* const* loc, double* const* out, int out_stride, int nrhs,
                 const int* const* active, int active_stride, cudaStream_t s)
{
    DDFinish F;
    std::memset(&F, 0, sizeof F);
    F.nblocks = 0;
    F.ndom = dd->ndom;
    for (int d = 0; d < dd->ndom; ++d) {
        F.loc[d] = loc[d];
        F.out[d] = out[d];
    }
    F.out_stride = out_stride;
    F.active = active ? active[0] : nullptr;
    F.active_stride = active_stride;
    return dd_finish(dd, F, nrhs, s);
}

// ---------------------------------------------------------------------------
// buffers
// ---------------------------------------------------------------------------

static int ensure_regions(wl_dd dd, size_t bytes)
{
    if (bytes <= dd->region_bytes) return WL_OK;
    WL_CUDA(cudaDeviceSynchronize());
    for (int d = 0; d < dd->ndom; ++d) {
        if (dd->recv[d]) cudaFree(dd->recv[d]);
        if (dd->send[d]) cudaFree(dd->send[d]);
        dd->recv[d] = dd->send[d] = nullptr;
    }
    dd->region_bytes = 0;
    for (int d = 0; d < dd->ndom; ++d) {
        WL_CUDA(cudaMalloc((void**)&dd->recv[d], bytes));
        WL_CUDA(cudaMalloc((void**)&dd->send[d], bytes));
    }
    dd->region_bytes = bytes;
    return WL_OK;
}

static int ensure_partials(wl_dd dd, int nrhs, int blocks)
{
    if (nrhs <= dd->part_rhs && blocks <= dd->part_max_blocks) return WL_OK;
    WL_CUDA(cudaDeviceSynchronize());
    if (dd->partial) cudaFree(dd->partial);
    dd->partial = nullptr;
    dd->part_rhs = std::max(nrhs, dd->part_rhs);
    dd->part_max_blocks = std::max(blocks, dd->part_max_blocks);
    dd->part_dom_stride = (long long)dd->part_rhs * dd->part_max_blocks * 3;
    WL_CUDA(cudaMalloc((void**)&dd->partial, sizeof(double) * dd->part_dom_stride * dd->ndom));
    return WL_OK;
}

static int ensure_loc(wl_dd dd, int nrhs)
{
    if (nrhs <= dd->loc_rhs) return WL_OK;
    WL_CUDA(cudaDeviceSynchronize());
    if (dd->loc) cudaFree(dd->loc);
    dd->loc = nullptr;
    WL_CUDA(cudaMalloc((void**)&dd->loc, sizeof(double) * 3 * nrhs * dd->ndom));
    dd->loc_rhs = nrhs;
    return WL_OK;
}

// ---------------------------------------------------------------------------
// one decomposed hopping application
// ---------------------------------------------------------------------------

void dd_segments(const Geom& g, int cut, int P, int nrhs, int np, long long (&hoff)[2][4][2], DDSeg (&seg)[12],
                 int& nseg, long long& total, long long& bytes)
{
    std::memset(hoff, 0, sizeof hoff);
    nseg = 0;
    total = 0;
    bytes = 0;
    for (int k = 0; k < np; ++k)
        for (int mu = 1; mu < 4; ++mu)
            if (cut & (1 << mu))
                for (int side = 0; side < 2; ++side) {
                    const long long fs = g.Vh / g.L[mu];
                    hoff[k][mu][side] = bytes;
                    bytes += halo_face_bytes(P, fs) * nrhs;
                    seg[nseg++] = {k, mu, side, total, fs};
                    total += fs;
                }
}

// segment number of (launch parity, mu, side) in message tags
static int seg_code(const DDSeg& S) { return 6 * S.pidx + 2 * (S.mu - 1) + S.side; }

int dd_launch_hop(wl_dd dd, const DDLaunch& h, cudaStream_t s)
{
    const int P = h.prec;
    for (int d = 0; d < dd->ndom; ++d)
        if (!dd->dom[d]->links[P][0])
            return set_error(WL_ERR_STATE, "domain decomposition was created without the requested precision");
    static const bool r12_off = getenv("WL_NO_R12") != nullptr;
    const int lf = (P == WL_F32 || P == WL_F16) && dd->dom[0]->links_r12[P][0] && !r12_off ? 1 : 0;
    const int np = h.nparity, nrhs = h.nrhs;
    const Geom& g = dd->gloc;

    // halo segments of (launch parity, mu, side), all right-hand sides each
    long long hoff[2][4][2];
    DDSeg seg[12];
    int nseg = 0;
    long long total = 0, off = 0;
    dd_segments(g, dd->cut, P, nrhs, np, hoff, seg, nseg, total, off);
    WL_TRY(ensure_regions(dd, (size_t)off));
    const size_t sb = spinor_field_bytes(P, 1);
    const bool route_all = dd->has_tr && dd->tr.all;
    // a face goes straight into a held neighbour's halo in the direct mode
    auto direct_to = [&](int to) { return dd->direct && !route_all && dd->local_of[to] >= 0; };

    // Two streams: the interior sweep on `s`; pack -> exchange -> boundary on
    // the side stream, at the same time (the interior needs no face, and the
    // two sweeps write disjoint sites and reduction slots).  The side stream
    // first waits for everything issued on `s` before this call.
    DDArgs A;
    std::memset(&A, 0, sizeof A);
    A.g = g;
    for (int mu = 1; mu < 4; ++mu)
        if (dd->cut & (1 << mu)) {
            A.cutmask |= 3u << (2 * mu);
            A.fs[mu] = dd->fs[mu];
        }
    std::memcpy(A.hoff, hoff, sizeof hoff);
    A.active_stride = h.active_stride;
    A.parity0 = h.parity0;
    A.rs_in = h.rs_in;
    A.rs_out = h.rs_out;
    A.rs_x1 = h.rs_x1;
    A.rs_x2 = h.rs_x2;
    A.rs_w = h.rs_w;
    A.a = h.a;
    A.b1 = h.b1;
    for (int mu = 0; mu < 4; ++mu) A.ph[mu] = {(float)dd->global.bc_re[mu], (float)dd->global.bc_im[mu]};
    for (int d = 0; d < dd->ndom; ++d) {
        DDDom& D = A.d[d];
        wl_gauge gd = dd->dom[d];
        for (int k = 0; k < np; ++k) {
            const int p = h.parity0 + k;
            D.links[k] = lf ? gd->links_r12[P][p] : gd->links[P][p];
            D.in[k] = (const char*)h.in[d][k];
            D.out[k] = (char*)h.out[d][k];
            D.x1[k] = (const char*)h.x1[d][k];
            D.x2[k] = (const char*)h.x2[d][k];
            D.w[k] = (const char*)h.w[d][k];
            // clover epilogue: A (kClX2, on x2) or A^-1 (kClOut) of the output parity
            D.cl[k] = h.cl_mode ? gd->clov[P][p][h.cl_mode == kClOut ? 1 : 0] : nullptr;
            if (h.cl_mode && !D.cl[k])
                return set_error(WL_ERR_STATE, "decomposition has no clover term in the requested precision");
        }
        D.halo = dd->recv[d];
        D.active = h.active[d];
        D.edge = dd->edge[d];
    }
    const bool t_only = dd->cut == (1 << 3);
    const int bi = (int)((dd->nint + kDDBlock - 1) / kDDBlock);
    const int bb = (int)((dd->nbnd + kDDBlock - 1) / kDDBlock);
    // reducing launches: capped grids looping over both parities' sites
    const int gi = h.dot && dd->nint ? dd_reducing_grid(np * dd->nint, dd->ndom, dd->dom[0]->num_sms) : 0;
    const int gb = h.dot && dd->nbnd ? dd_reducing_grid(np * dd->nbnd, dd->ndom, dd->dom[0]->num_sms) : 0;
    if (h.dot) {
        WL_TRY(ensure_partials(dd, nrhs, gi + gb));
        A.partial = dd->partial;
        A.dom_stride = dd->part_dom_stride;
        A.max_blocks = dd->part_max_blocks;
    }
    const int extra = (h.x1[0][0] ? 1 : 0) + (h.x2[0][0] ? 1 : 0) + (h.w[0][0] ? 1 : 0);
    const double site_bytes = (double)(lf ? (P == WL_F32 ? 384 : 192) : link_field_bytes(P, 1)) +
                              (h.cl_mode ? (double)clover_site_bytes(P) : 0.0) + (double)nrhs * (2 + extra) * sb;
    // the interior of a y or z cut as a box (no site list to read)
    bool box_ok = false;
    {
        long long nbox = g.Lxh;
        for (int mu = 1; mu < 4; ++mu) {
            const bool cut_mu = (dd->cut >> mu) & 1;
            A.bo[mu] = cut_mu ? 1 : 0;
            A.bn[mu] = cut_mu ? g.L[mu] - 2 : g.L[mu];
            nbox *= A.bn[mu];
        }
        for (int k = 1; k <= 2; ++k) fast_div_magic(A.bn[k], &A.bm[k], &A.bsh[k]);
        box_ok = nbox == dd->nint;
    }
    // part 0: interior (one contiguous range when only t is cut), part 1: boundary
    auto run = [&](int part, DDArgs AA, cudaStream_t st_) -> int {
        const long long n = part ? dd->nbnd : dd->nint;
        if (n == 0) return WL_OK;
        AA.sites = part ? dd->bsites : (t_only || box_ok ? nullptr : dd->isites);
        AA.site0 = (!part && t_only) ? g.st : 0;
        AA.box = (!part && !t_only && box_ok) ? 1 : 0;
        AA.nsites = n;
        AA.nparity = np;
        AA.blocks_per_parity = part ? bb : bi;
        AA.block0 = h.dot ? (part ? gi : 0) : (part ? np * bi : 0);
        const unsigned gx = h.dot ? (unsigned)(part ? gb : gi) : (unsigned)(AA.blocks_per_parity * np);
        const dim3 grid(gx, (unsigned)nrhs, (unsigned)dd->ndom);
        dd_hop_family(lf, h.cl_mode, P, h.dagger != 0, h.dot, part == 1, AA, grid, st_);
        WL_CHECK_LAUNCH((double)dd->ndom * np * n * site_bytes);
        return WL_OK;
    };
    if (!nseg) {  // nothing cut: every site is interior
        WL_TRY(run(0, A, s));
    } else {
        WL_CUDA(cudaEventRecord(dd->ev_packed, s));
        WL_CUDA(cudaStreamWaitEvent(dd->comm, dd->ev_packed, 0));
        WL_TRY(run(0, A, s));
        // 1. pack
        DDPackArgs PA;
        std::memset(&PA, 0, sizeof PA);
        PA.g = g;
        std::memcpy(PA.seg, seg, sizeof seg);
        PA.nseg = nseg;
        PA.total = total;
        std::memcpy(PA.hoff, hoff, sizeof hoff);
        PA.rs_in = h.rs_in;
        for (int d = 0; d < dd->ndom; ++d) {
            for (int k = 0; k < np; ++k) PA.in[d][k] = (const char*)h.in[d][k];
            for (int mu = 1; mu < 4; ++mu)
                for (int side = 0; side < 2; ++side) {
                    // side 0 feeds the backward neighbour, side 1 the forward one
                    const int to = dd->peer[d][mu][side];
                    PA.dst[d][mu][side] = direct_to(to) ? dd->recv[dd->local_of[to]] : dd->send[d];
                }
        }
        const dim3 grid((unsigned)((total + kDDBlock - 1) / kDDBlock), (unsigned)nrhs, (unsigned)dd->ndom);
        dd_pack(P, h.dagger != 0, PA, grid, dd->comm);
        WL_CHECK_LAUNCH((double)nrhs * dd->ndom * total * (sb + 16 * halo_planes(P) + (P == WL_F16 ? 4 : 0)));
        // 2. exchange: device copies between held blocks, messages through the
        // transport for the rest
        dd->msgs.clear();
        DDCopies C;
        C.n = 0;
        for (int d = 0; d < dd->ndom; ++d)
            for (int k = 0; k < nseg; ++k) {
                const DDSeg& S = seg[k];
                const long long o = hoff[S.pidx][S.mu][S.side];
                const size_t bytes = (size_t)(halo_face_bytes(P, S.count) * nrhs);
                const int to = dd->peer[d][S.mu][S.side], from = dd->peer[d][S.mu][1 - S.side];
                if (dd->local_of[to] < 0 || route_all) {
                    dd->msgs.push_back({1, dd->gid[d], to, 12 * to + seg_code(S), (size_t)o, bytes, dd->send[d] + o});
                } else if (!direct_to(to)) {
                    C.src[C.n] = (const uint4*)(dd->send[d] + o);
                    C.dst[C.n] = (uint4*)(dd->recv[dd->local_of[to]] + o);
                    C.n16[C.n] = (long long)(bytes / 16);
                    if (++C.n == kCopySegs) WL_TRY(launch_copies(C, dd->comm));
                }
                if (dd->local_of[from] < 0 || route_all)
                    dd->msgs.push_back({0, dd->gid[d], from, 12 * dd->gid[d] + seg_code(S), (size_t)o, bytes,
                                        dd->recv[d] + o});
            }
        WL_TRY(launch_copies(C, dd->comm));
        if (!dd->msgs.empty() &&
            dd->tr.exchange(dd->tr.ctx, (int)dd->msgs.size(), dd->msgs.data(), (void*)dd->comm) != 0)
            return set_error(WL_ERR_CUDA, "transport exchange failed");
        // 3. boundary on the side stream, then the main stream waits for it
        WL_TRY(run(1, A, dd->comm));
        WL_CUDA(cudaEventRecord(dd->ev_exchanged, dd->comm));
        WL_CUDA(cudaStreamWaitEvent(s, dd->ev_exchanged, 0));
    }

    // 5. the fused reductions, summed over the blocks
    if (h.dot) {
        DDFinish F;
        std::memset(&F, 0, sizeof F);
        F.partial = dd->partial;
        F.dom_stride = dd->part_dom_stride;
        F.max_blocks = dd->part_max_blocks;
        F.nblocks = gi + gb;
        F.ndom = dd->ndom;
        for (int d = 0; d < dd->ndom; ++d) F.out[d] = h.dot_out[d];
        F.out_stride = h.dot_stride;
        F.active = h.active[0];
        F.active_stride = h.active_stride;
        WL_TRY(dd_finish(dd, F, nrhs, s));
    }
    return WL_OK;
}

}  // namespace wl

using namespace wl;

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------

extern "C" int wl_dd_destroy(wl_dd dd)
{
    if (!dd) return WL_OK;
    cudaDeviceSynchronize();
    dd_free_solver(dd);
    for (int d = 0; d < dd->ndom; ++d) {
        if (dd->dom[d]) wl_gauge_destroy(dd->dom[d]);
        if (dd->recv[d]) cudaFree(dd->recv[d]);
        if (dd->send[d]) cudaFree(dd->send[d]);
    }
    if (dd->isites) cudaFree(dd->isites);
    if (dd->bsites) cudaFree(dd->bsites);
    if (dd->partial) cudaFree(dd->partial);
    if (dd->loc) cudaFree(dd->loc);
    if (dd->stage) cudaFree(dd->stage);
    if (dd->ev_packed) cudaEventDestroy(dd->ev_packed);
    if (dd->ev_exchanged) cudaEventDestroy(dd->ev_exchanged);
    if (dd->comm) cudaStreamDestroy(dd->comm);
    delete dd;
    return WL_OK;
}

// Block extents of a decomposition (WL_ERR_ARG when the grid does not fit).
static int dd_local_dims(const int* dims, const int* grid, int* loc, int* nblk)
{
    if (!grid) return set_error(WL_ERR_ARG, "NULL block grid");
    if (grid[0] != 1) return set_error(WL_ERR_ARG, "the x direction is never cut: grid[0] must be 1");
    long long n = 1;
    loc[0] = dims[0];
    for (int mu = 1; mu < 4; ++mu) {
        if (grid[mu] < 1) return set_error(WL_ERR_ARG, "grid entries must be >= 1");
        if (dims[mu] % grid[mu]) return set_error(WL_ERR_ARG, "grid must divide the lattice extents");
        loc[mu] = dims[mu] / grid[mu];
        if (loc[mu] < 2 || loc[mu] % 2) return set_error(WL_ERR_ARG, "block extents must be even and >= 2");
        n *= grid[mu];
    }
    if (n > (1 << 20)) return set_error(WL_ERR_ARG, "too many blocks");
    *nblk = (int)n;
    return WL_OK;
}

// Grid coordinates of block b and of its neighbours.
static void block_coords(const int* grid, int b, int (&c)[4])
{
    c[0] = 0;
    c[1] = b % grid[1];
    c[2] = (b / grid[1]) % grid[2];
    c[3] = b / (grid[1] * grid[2]);
}
static int block_peer(const int* grid, const int (&c)[4], int mu, int side)
{
    int cc[4] = {c[0], c[1], c[2], c[3]};
    cc[mu] = (c[mu] + (side ? 1 : grid[mu] - 1)) % grid[mu];
    return cc[1] + grid[1] * (cc[2] + grid[2] * cc[3]);
}

extern "C" int wl_dd_create_part(wl_dd* out, const wl_lattice* lat, const int* grid, int first, int count,
                                 const double* U, int prec_mask, const wl_dd_transport* tr, void* stream)
{
    WL_ENTRY();
    if (!out) return set_error(WL_ERR_ARG, "NULL output handle");
    *out = nullptr;
    WL_TRY(validate_lattice(lat));
    wl_lattice loc = *lat;
    int nblk = 0;
    WL_TRY(dd_local_dims(lat->dims, grid, loc.dims, &nblk));
    if (first < 0 || count < 1 || first + count > nblk)
        return set_error(WL_ERR_ARG, "held blocks must lie in 0 .. (number of blocks) - 1");
    if (count > kMaxDomains) return set_error(WL_ERR_ARG, "at most 16 blocks per process");
    if (count < nblk && !tr) return set_error(WL_ERR_ARG, "blocks held elsewhere need a transport");
    if (tr && (!tr->exchange || !tr->allreduce)) return set_error(WL_ERR_ARG, "transport without callbacks");
    cudaStream_t s = (cudaStream_t)stream;
    auto dd = new wl_dd_s();
    dd->global = *lat;
    dd->gglob = make_geom(lat->dims);
    dd->gloc = make_geom(loc.dims);
    for (int mu = 0; mu < 4; ++mu) dd->grid[mu] = grid[mu];
    dd->nblk = nblk;
    dd->ndom = count;
    dd->local_of.assign(nblk, -1);
    if (tr) {
        dd->tr = *tr;
        dd->has_tr = true;
    }
    for (int mu = 1; mu < 4; ++mu)
        if (grid[mu] > 1) {
            dd->cut |= 1 << mu;
            dd->fs[mu] = dd->gloc.Vh / loc.dims[mu];
        }
    int rc = WL_OK;
    do {
        if (cudaGetDevice(&dd->device) != cudaSuccess) { rc = set_error(WL_ERR_CUDA, "cudaGetDevice"); break; }
        for (int d = 0; d < count && rc == WL_OK; ++d) {
            const int b = first + d;
            dd->gid[d] = b;
            dd->local_of[b] = d;
            int c[4];
            block_coords(grid, b, c);
            int org[4];
            for (int mu = 0; mu < 4; ++mu) {
                dd->coord[d][mu] = c[mu];
                org[mu] = c[mu] * loc.dims[mu];
                for (int side = 0; side < 2; ++side) dd->peer[d][mu][side] = block_peer(grid, c, mu, side);
            }
            unsigned edge = 0;
            for (int mu = 0; mu < 4; ++mu) {
                if (c[mu] == grid[mu] - 1) edge |= 1u << (2 * mu);  // forward face is the lattice's
                if (c[mu] == 0) edge |= 1u << (2 * mu + 1);
            }
            dd->edge[d] = edge;
            // the decomposed kernels read full or twelve-real links only
            rc = gauge_create(&dd->dom[d], &loc, lat, org, U, prec_mask & ~WL_LINKS_R8, s);
            if (rc == WL_OK) dd->dom[d]->dd_part = 1;
        }
        if (rc != WL_OK) break;
        // interior / boundary half indices of a block
        const Geom& g = dd->gloc;
        std::vector<int> is, bs;
        for (long long i = 0; i < g.Vh; ++i) {
            const long long row = i / g.Lxh;
            const int c[4] = {0, (int)(row % g.L[1]), (int)((row / g.L[1]) % g.L[2]), (int)(row / ((long long)g.L[1] * g.L[2]))};
            bool bnd = false;
            for (int mu = 1; mu < 4; ++mu)
                if ((dd->cut >> mu) & 1) bnd |= c[mu] == 0 || c[mu] == g.L[mu] - 1;
            (bnd ? bs : is).push_back((int)i);
        }
        dd->nint = (long long)is.size();
        dd->nbnd = (long long)bs.size();
        if (cudaMalloc((void**)&dd->isites, sizeof(int) * std::max<size_t>(1, is.size())) != cudaSuccess ||
            cudaMalloc((void**)&dd->bsites, sizeof(int) * std::max<size_t>(1, bs.size())) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(WL_ERR_CUDA, "cudaMalloc site lists");
            break;
        }
        if ((!is.empty() && cudaMemcpy(dd->isites, is.data(), sizeof(int) * is.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
            (!bs.empty() && cudaMemcpy(dd->bsites, bs.data(), sizeof(int) * bs.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
            rc = set_error(WL_ERR_CUDA, "site list upload");
            break;
        }
        // the side stream (pack, exchange, boundary) at the highest priority:
        // its blocks are scheduled ahead of the interior's waiting blocks, so
        // the faces move early instead of after the interior sweep
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
            cudaGetLastError();
            least = greatest = 0;
        }
        if (cudaStreamCreateWithPriority(&dd->comm, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&dd->ev_packed, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&dd->ev_exchanged, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(WL_ERR_CUDA, "exchange stream / events");
            break;
        }
        const char* e = getenv("WL_DD_EXCHANGE");
        dd->direct = (e && std::strcmp(e, "direct") == 0) ? 1 : 0;
    } while (0);
    if (rc != WL_OK) {
        wl_dd_destroy(dd);
        return rc;
    }
    *out = dd;
    return WL_OK;
}

extern "C" int wl_dd_create(wl_dd* out, const wl_lattice* lat, const int* grid, const double* U, int prec_mask,
                            void* stream)
{
    WL_ENTRY();
    if (!out) return set_error(WL_ERR_ARG, "NULL output handle");
    *out = nullptr;
    WL_TRY(validate_lattice(lat));
    int loc[4], nblk = 0;
    WL_TRY(dd_local_dims(lat->dims, grid, loc, &nblk));
    if (nblk > kMaxDomains) return set_error(WL_ERR_ARG, "at most 16 blocks per decomposition");
    return wl_dd_create_part(out, lat, grid, 0, nblk, U, prec_mask, nullptr, stream);
}

extern "C" int wl_dd_plan(const int* dims, const int* grid, int block, wl_prec prec, int nrhs, int nparity,
                          wl_dd_msg* msgs, int max_msgs)
{
    if (!dims) return set_error(WL_ERR_ARG, "NULL extents");
    int loc[4], nblk = 0;
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 2 || dims[mu] % 2) return set_error(WL_ERR_ARG, "lattice extents must be even and >= 2");
    WL_TRY(dd_local_dims(dims, grid, loc, &nblk));
    if (block < 0 || block >= nblk) return set_error(WL_ERR_ARG, "block index out of range");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (nrhs < 1 || (nparity != 1 && nparity != 2)) return set_error(WL_ERR_ARG, "nrhs >= 1, nparity 1 or 2");
    if (max_msgs > 0 && !msgs) return set_error(WL_ERR_ARG, "NULL message array");
    int cut = 0;
    for (int mu = 1; mu < 4; ++mu)
        if (grid[mu] > 1) cut |= 1 << mu;
    long long hoff[2][4][2];
    DDSeg seg[12];
    int nseg = 0;
    long long total = 0, bytes = 0;
    dd_segments(make_geom(loc), cut, prec, nrhs, nparity, hoff, seg, nseg, total, bytes);
    int c[4];
    block_coords(grid, block, c);
    int n = 0;
    for (int k = 0; k < nseg; ++k) {
        const DDSeg& S = seg[k];
        const size_t o = (size_t)hoff[S.pidx][S.mu][S.side];
        const size_t b = (size_t)(halo_face_bytes(prec, S.count) * nrhs);
        const int to = block_peer(grid, c, S.mu, S.side), from = block_peer(grid, c, S.mu, 1 - S.side);
        const wl_dd_msg m[2] = {{1, block, to, 12 * to + seg_code(S), o, b, nullptr},
                                {0, block, from, 12 * block + seg_code(S), o, b, nullptr}};
        for (const wl_dd_msg& q : m) {
            if (n < max_msgs) msgs[n] = q;
            ++n;
        }
    }
    return n;
}

extern "C" int wl_dd_blocks(wl_dd dd) { return dd ? dd->ndom : 0; }

extern "C" int wl_dd_block(wl_dd dd, int k, wl_gauge* g, int* coord)
{
    if (!dd) return set_error(WL_ERR_ARG, "NULL decomposition");
    if (k < 0 || k >= dd->ndom) return set_error(WL_ERR_ARG, "held-block index out of range");
    if (g) *g = dd->dom[k];
    if (coord)
        for (int mu = 0; mu < 4; ++mu) coord[mu] = dd->coord[k][mu];
    return WL_OK;
}

extern "C" int wl_dd_set_exchange(wl_dd dd, int mode)
{
    if (!dd) return set_error(WL_ERR_ARG, "NULL decomposition");
    if (mode != 0 && mode != 1) return set_error(WL_ERR_ARG, "exchange mode must be 0 (copy) or 1 (direct)");
    cudaDeviceSynchronize();
    dd->direct = mode;
    return WL_OK;
}

static int dd_canonical(wl_dd dd, double* const* loc, double* glob, int nrhs, int dir, cudaStream_t s)
{
    if (!dd) return set_error(WL_ERR_ARG, "NULL decomposition");
    if (!loc || !glob) return set_error(WL_ERR_ARG, "NULL pointer");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    const long long Vl = 2 * dd->gloc.Vh, Vg = 2 * dd->gglob.Vh;
    for (int d = 0; d < dd->ndom; ++d) {
        if (!loc[d]) return set_error(WL_ERR_ARG, "NULL block field");
        Origin org;
        for (int mu = 0; mu < 4; ++mu) org.o[mu] = dd->coord[d][mu] * dd->gloc.L[mu];
        const dim3 grid((unsigned)((Vl + 127) / 128), (unsigned)nrhs);
        dd_copy_canonical_kernel<<<grid, 128, 0, s>>>(loc[d], glob, dd->gloc, dd->gglob, org, Vl, Vg, dir, 24);
        WL_CHECK_LAUNCH(2.0 * 192.0 * Vl * nrhs);
    }
    return WL_OK;
}

extern "C" int wl_dd_scatter(wl_dd dd, double* const* local, const double* global, int nrhs, void* stream)
{
    WL_ENTRY();
    return dd_canonical(dd, local, (double*)global, nrhs, 0, (cudaStream_t)stream);
}

extern "C" int wl_dd_gather(wl_dd dd, double* global, const double* const* local, int nrhs, void* stream)
{
    WL_ENTRY();
    return dd_canonical(dd, (double* const*)local, global, nrhs, 1, (cudaStream_t)stream);
}

extern "C" int wl_dd_clover_set(wl_dd dd, const double* F, void* stream)
{
    WL_ENTRY();
    if (!dd) return set_error(WL_ERR_ARG, "NULL decomposition");
    cudaStream_t s = (cudaStream_t)stream;
    if (!F) {
        for (int d = 0; d < dd->ndom; ++d) WL_TRY(clover_set(dd->dom[d], nullptr, s));
        return WL_OK;
    }
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, F) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return set_error(WL_ERR_ARG, "clover field must be device memory");
    }
    const long long Vl = 2 * dd->gloc.Vh, Vg = 2 * dd->gglob.Vh;
    double* loc = nullptr;  // one block's F at a time
    WL_CUDA(cudaMalloc((void**)&loc, sizeof(double) * 144 * Vl));
    int rc = WL_OK;
    for (int d = 0; d < dd->ndom && rc == WL_OK; ++d) {
        Origin org;
        for (int mu = 0; mu < 4; ++mu) org.o[mu] = dd->coord[d][mu] * dd->gloc.L[mu];
        dd_copy_canonical_kernel<<<(unsigned)((Vl + 127) / 128), 128, 0, s>>>(loc, (double*)F, dd->gloc, dd->gglob,
                                                                              org, Vl, Vg, 0, 144);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(WL_ERR_CUDA, "clover scatter launch failed");
        count_launch(1, 2.0 * 1152.0 * Vl);
        if (rc == WL_OK) rc = clover_set(dd->dom[d], loc, s);  // synchronises the stream
    }
    cudaFree(loc);
    if (rc != WL_OK)  // all blocks or none
        for (int d = 0; d < dd->ndom; ++d) clover_set(dd->dom[d], nullptr, s);
    return rc;
}

static int dd_check(wl_dd dd, const void* const* out, const void* const* in, wl_prec prec, int nrhs, int nhalf)
{
    if (!dd) return set_error(WL_ERR_ARG, "NULL decomposition");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    if (!out || !in) return set_error(WL_ERR_ARG, "NULL pointer");
    const size_t fb = spinor_field_bytes(prec, dd->gloc.Vh) * nhalf * nrhs;
    for (int d = 0; d < dd->ndom; ++d) {
        if (!out[d] || !in[d]) return set_error(WL_ERR_ARG, "NULL block field");
        if (!dd->dom[d]->links[prec][0])
            return set_error(WL_ERR_STATE, "decomposition was created without this precision");
        const char *o = (const char*)out[d], *i = (const char*)in[d];
        if (o < i + fb && i < o + fb) return set_error(WL_ERR_ARG, "out and in overlap");
    }
    return WL_OK;
}

extern "C" int wilson_dslash_dd(wl_dd dd, void* const* out, const void* const* in, int out_parity, int dagger,
                                wl_prec prec, int nrhs, void* stream)
{
    WL_ENTRY();
    WL_TRY(dd_check(dd, (const void* const*)out, in, prec, nrhs, 1));
    if (out_parity != 0 && out_parity != 1) return set_error(WL_ERR_ARG, "out_parity must be 0 or 1");
    const size_t fb = spinor_field_bytes(prec, dd->gloc.Vh);
    DDLaunch h;
    h.prec = prec;
    h.dagger = dagger ? 1 : 0;
    h.parity0 = out_parity;
    h.nrhs = nrhs;
    for (int d = 0; d < dd->ndom; ++d) {
        h.in[d][0] = in[d];
        h.out[d][0] = out[d];
    }
    h.rs_in = h.rs_out = (long long)fb;
    return dd_launch_hop(dd, h, (cudaStream_t)stream);
}

extern "C" int wilson_mult_dd(wl_dd dd, void* const* out, const void* const* in, int eo, int dagger, wl_prec prec,
                              int nrhs, void* stream)
{
    WL_ENTRY();
    WL_TRY(dd_check(dd, (const void* const*)out, in, prec, nrhs, eo ? 1 : 2));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fb = spinor_field_bytes(prec, dd->gloc.Vh);
    const double kappa = dd->global.kappa;
    const bool clov = dd->dom[0]->has_clover;
    if (!eo) {  // out_p = in_p - kappa H in_{1-p} on [even | odd] block fields
        DDLaunch h;
        h.prec = prec;
        h.dagger = dagger ? 1 : 0;
        h.parity0 = 0;
        h.nparity = 2;
        h.nrhs = nrhs;
        for (int d = 0; d < dd->ndom; ++d) {
            h.in[d][0] = (const char*)in[d] + fb;
            h.in[d][1] = in[d];
            h.out[d][0] = out[d];
            h.out[d][1] = (char*)out[d] + fb;
            if (clov) {  // out_p = A_pp in_p - kappa H in_{1-p}
                h.x2[d][0] = in[d];
                h.x2[d][1] = (const char*)in[d] + fb;
            } else {
                h.x1[d][0] = in[d];
                h.x1[d][1] = (const char*)in[d] + fb;
            }
        }
        h.rs_in = h.rs_out = h.rs_x1 = h.rs_x2 = (long long)(2 * fb);
        if (clov) {
            h.b1 = 1.0;
            h.cl_mode = kClX2;
        }
        h.a = -kappa;
        return dd_launch_hop(dd, h, s);
    }
    // M_ee = 1 - kappa^2 H_eo H_oe, through each block's odd temporary
    for (int d = 0; d < dd->ndom; ++d) WL_TRY(ensure_tmp(dd->dom[d], prec, fb * nrhs));
    DDLaunch h1;
    h1.prec = prec;
    h1.dagger = dagger ? 1 : 0;
    h1.parity0 = 1;
    h1.nrhs = nrhs;
    for (int d = 0; d < dd->ndom; ++d) {
        h1.in[d][0] = in[d];
        h1.out[d][0] = dd->dom[d]->tmp[prec];
    }
    h1.rs_in = h1.rs_out = (long long)fb;
    if (clov) h1.cl_mode = kClOut;  // tmp = A_oo^-1 H_oe in
    WL_TRY(dd_launch_hop(dd, h1, s));
    DDLaunch h2 = h1;
    h2.parity0 = 0;
    for (int d = 0; d < dd->ndom; ++d) {
        h2.in[d][0] = dd->dom[d]->tmp[prec];
        h2.out[d][0] = out[d];
        if (clov) h2.x2[d][0] = in[d];  // out = A_ee in - kappa^2 H_eo tmp
        else h2.x1[d][0] = in[d];
    }
    h2.rs_x1 = h2.rs_x2 = (long long)fb;
    if (clov) {
        h2.b1 = 1.0;
        h2.cl_mode = kClX2;
    } else {
        h2.cl_mode = kClNone;
    }
    h2.a = -kappa * kappa;
    return dd_launch_hop(dd, h2, s);
}

extern "C" int wl_cdot_dd(wl_dd dd, double* out, const void* const* a, const void* const* b, wl_prec prec, int nrhs,
                          void* stream)
{
    WL_ENTRY();
    if (!dd) return set_error(WL_ERR_ARG, "NULL decomposition");
    if (!out || !a || !b) return set_error(WL_ERR_ARG, "NULL pointer");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    cudaStream_t s = (cudaStream_t)stream;
    WL_TRY(ensure_loc(dd, nrhs));
    double* loc[kMaxDomains];
    double* outs[kMaxDomains] = {};
    for (int d = 0; d < dd->ndom; ++d) {
        if (!a[d] || !b[d]) return set_error(WL_ERR_ARG, "NULL block field");
        loc[d] = dd->loc + (size_t)3 * nrhs * d;
        WL_TRY(launch_cdot(dd->dom[d], prec, a[d], b[d], 1, nrhs, loc[d], 3, nullptr, s));
    }
    outs[0] = out;
    return dd_allreduce(dd, loc, outs, 3, nrhs, nullptr, 1, s);
}
