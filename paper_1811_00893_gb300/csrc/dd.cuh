// Domain decomposition of the hopping term (Sec. 4.4, "Thread Task
// Assignment": pack the faces, communicate while the bulk is computed, then
// finish the boundary).  The lattice is cut into equal blocks along t, then z,
// then y (x is never cut, as in Sec. 4.1).  Each block is a gauge object of its
// own whose link fields are the global ones at its sites (hop matrices of face
// sites already point across the cut), so the blocks differ from an undivided
// lattice only in where the spinor of a hop that leaves the block comes from:
//
//   pack      the spin-projected half spinors (12 reals, Eq. 1's (1 -+ gamma)
//             acting on the neighbour) of the block's faces, per cut
//             direction and side, for the neighbouring blocks;
//   exchange  the packed faces travel to the neighbours' halo buffers (a copy
//             kernel between blocks of one process -- the paper's
//             "communication = copy" mode of Sec. 5.2.3 -- or a transport);
//   interior  sites none of whose hops leave the block, on the main stream;
//   boundary  the remaining sites, with the hops that leave the block read from
//             the halo.
// Pack, exchange and boundary run on a side stream while the interior runs,
// so the exchange and the boundary sweep's latency hide behind the bulk.
//
// Every output site is computed once, by one thread, with the same
// operations as the undivided kernel.  Global sums (the BiCGStab dots) are
// formed per block and then summed over the blocks in a fixed order (the
// allreduce).
#pragma once

#include <vector>

#include "hop.cuh"
#include "solver.cuh"

namespace wl {

static constexpr int kMaxDomains = 16;  // blocks one process holds (one launch covers all)

// Halo planes: a projected half spinor is 6 complex numbers, stored as 16-byte
// planes over the face sites (3 float4 of two complex in FP32 arithmetic, 6
// double2 in FP64, 6 float4 hi/lo pairs in df64).  FP16 storage computes in
// FP32, so its halo is FP32, and like the undivided FP16 kernel it keeps the
// half spinor of the neighbour's stored values unscaled, followed by a plane
// of the neighbour's FP32 norms: the boundary sites then see exactly the
// operands the undivided kernel would have formed.
__host__ __device__ constexpr int halo_planes(int P) { return (P == WL_F32 || P == WL_F16) ? 3 : 6; }
// Bytes of one right-hand side's face of fs sites (a multiple of 16)
__host__ __device__ constexpr long long halo_face_bytes(int P, long long fs)
{
    return 16 * halo_planes(P) * fs + (P == WL_F16 ? 16 * ((fs + 3) / 4) : 0);
}

// nrm: the FP16 neighbour's per-site norm (unused for the other types)
template <int P>
__device__ __forceinline__ void store_half(char* base, long long fs, long long f,
                                           const cx<typename Prec<P>::real> (&h0)[3],
                                           const cx<typename Prec<P>::real> (&h1)[3], float nrm)
{
    if constexpr (P == WL_F32 || P == WL_F16) {
        float4* q = (float4*)base;
        q[0 * fs + f] = make_float4(h0[0].re, h0[0].im, h0[1].re, h0[1].im);
        q[1 * fs + f] = make_float4(h0[2].re, h0[2].im, h1[0].re, h1[0].im);
        q[2 * fs + f] = make_float4(h1[1].re, h1[1].im, h1[2].re, h1[2].im);
        if constexpr (P == WL_F16) ((float*)(q + 3 * fs))[f] = nrm;
    } else if constexpr (P == WL_F64) {
        double2* q = (double2*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            q[c * fs + f] = make_double2(h0[c].re, h0[c].im);
            q[(3 + c) * fs + f] = make_double2(h1[c].re, h1[c].im);
        }
    } else {
        float4* q = (float4*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            q[c * fs + f] = make_float4(h0[c].re.hi, h0[c].re.lo, h0[c].im.hi, h0[c].im.lo);
            q[(3 + c) * fs + f] = make_float4(h1[c].re.hi, h1[c].re.lo, h1[c].im.hi, h1[c].im.lo);
        }
    }
}

template <int P>
__device__ __forceinline__ void load_half(cx<typename Prec<P>::real> (&h0)[3], cx<typename Prec<P>::real> (&h1)[3],
                                          float& nrm, const char* base, long long fs, long long f)
{
    nrm = 1.0f;
    if constexpr (P == WL_F32 || P == WL_F16) {
        const float4* q = (const float4*)base;
        const float4 a = __ldg(q + f), b = __ldg(q + fs + f), c = __ldg(q + 2 * fs + f);
        h0[0] = {a.x, a.y};
        h0[1] = {a.z, a.w};
        h0[2] = {b.x, b.y};
        h1[0] = {b.z, b.w};
        h1[1] = {c.x, c.y};
        h1[2] = {c.z, c.w};
        if constexpr (P == WL_F16) nrm = __ldg((const float*)(q + 3 * fs) + f);
    } else if constexpr (P == WL_F64) {
        const double2* q = (const double2*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 u = __ldg(q + c * fs + f), v = __ldg(q + (3 + c) * fs + f);
            h0[c] = {u.x, u.y};
            h1[c] = {v.x, v.y};
        }
    } else {
        const float4* q = (const float4*)base;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 u = __ldg(q + c * fs + f), v = __ldg(q + (3 + c) * fs + f);
            h0[c] = {df64(u.x, u.y), df64(u.z, u.w)};
            h1[c] = {df64(v.x, v.y), df64(v.z, v.w)};
        }
    }
}

// Coordinates (xh = x / 2, y, z, t) of half site i, and x itself on parity p.
__device__ __forceinline__ void half_coords(const Geom& g, int p, int i, int (&c)[4], int& xh)
{
    const int r0 = geo_div(g, 0, i);
    xh = i - r0 * g.Lxh;
    const int r1 = geo_div(g, 1, r0);
    c[1] = r0 - r1 * g.L[1];
    c[3] = geo_div(g, 2, r1);
    c[2] = r1 - c[3] * g.L[2];
    c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
}

// Neighbour half indices (periodic inside the block) and the face mask (bit
// 2 mu: x_mu = L_mu - 1, bit 2 mu + 1: x_mu = 0) of a site with coordinates c.
__device__ __forceinline__ unsigned block_neighbours(const Geom& g, int i, const int (&c)[4], int xh, int (&nb)[8])
{
    const int row = i - xh;
    const int sy = (int)g.sy, sz = (int)g.sz, st = (int)g.st;
    nb[0] = row + ((c[0] + 1 == g.L[0] ? 0 : c[0] + 1) >> 1);
    nb[1] = row + ((c[0] == 0 ? g.L[0] - 1 : c[0] - 1) >> 1);
    nb[2] = (c[1] == g.L[1] - 1) ? i - (g.L[1] - 1) * sy : i + sy;
    nb[3] = (c[1] == 0) ? i + (g.L[1] - 1) * sy : i - sy;
    nb[4] = (c[2] == g.L[2] - 1) ? i - (g.L[2] - 1) * sz : i + sz;
    nb[5] = (c[2] == 0) ? i + (g.L[2] - 1) * sz : i - sz;
    nb[6] = (c[3] == g.L[3] - 1) ? i - (g.L[3] - 1) * st : i + st;
    nb[7] = (c[3] == 0) ? i + (g.L[3] - 1) * st : i - st;
    unsigned faces = 0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        if (c[mu] == g.L[mu] - 1) faces |= 1u << (2 * mu);
        if (c[mu] == 0) faces |= 1u << (2 * mu + 1);
    }
    return faces;
}

// Index of a site in the face of direction mu (1..3): its half index with
// the mu coordinate dropped (x / 2 fastest, then the remaining directions).
__device__ __forceinline__ long long face_index(const Geom& g, int mu, const int (&c)[4], int xh)
{
    if (mu == 1) return xh + (long long)g.Lxh * (c[2] + (long long)g.L[2] * c[3]);
    if (mu == 2) return xh + (long long)g.Lxh * (c[1] + (long long)g.L[1] * c[3]);
    return xh + (long long)g.Lxh * (c[1] + (long long)g.L[1] * c[2]);
}

// Per-block pointers of one launch (launch parity k = 0, 1 where two).
struct DDDom {
    const void* links[2];
    const char* in[2];
    char* out[2];
    const char* x1[2];
    const char* x2[2];
    const char* w[2];
    const void* cl[2];
    const char* halo;    // this block's received faces (offsets in DDArgs::hoff)
    const int* active;   // per right-hand side: 0 skips it (nullptr: all run)
    unsigned edge;       // hops that cross the global boundary when they leave the block
};

struct DDArgs {
    Geom g;
    unsigned cutmask;      // bits 2 mu, 2 mu + 1 of every cut direction mu
    long long fs[4];       // face half sites per direction (0: not cut)
    // byte offset of the halo segment of (launch parity, mu, side) in a
    // block's region; a segment holds all right-hand sides back to back
    // (fs[mu] face sites of halo_planes(P) planes each)
    long long hoff[2][4][2];
    int active_stride;
    const int* sites;      // the launch's sites: interior or boundary half indices, or
    long long site0;       // (sites == nullptr, box == 0) the contiguous range site0 .. site0 + nsites - 1
    long long nsites;
    // box == 1 (sites == nullptr): the interior as the box of sites with
    // bo[mu] <= x_mu < bo[mu] + bn[mu] (mu = y, z, t; x whole), in half-index
    // order; bm / bsh: round-up reciprocals of bn[1], bn[2]
    int box;
    int bo[4], bn[4];
    unsigned bm[4];
    int bsh[4];
    int blocks_per_parity;  // plain launches: one site per thread, a block's parity fixed
    int parity0, nparity;   // launches with a fused reduction loop over both parities' sites
    long long rs_in, rs_out, rs_x1, rs_x2, rs_w;
    double a, b1;
    cx<float> ph[4];
    // fused reduction: each block's partial (w, out), ||out||^2 at
    // partial[dom * dom_stride + (rhs * max_blocks + block0 + blockIdx.x) * 3]
    double* partial;
    long long dom_stride;
    int max_blocks, block0;
    DDDom d[kMaxDomains];
};

// Loop-form spin projection of hop d for the double-float type (the
// hop_site_loop arithmetic of hop.cuh).
template <int P, bool DAG>
__device__ __forceinline__ void project_loop(cx<typename Prec<P>::real> (&h0)[3], cx<typename Prec<P>::real> (&h1)[3],
                                             const cx<typename Prec<P>::real> (&q)[12], int d)
{
    const unsigned code = hop_code(d >> 1);
    const int sflip = ((d & 1) ? DAG == false : DAG == true) ? 0 : 2;
    const int a0 = code & 1, k0 = ((code >> 1) + sflip) & 3;
    const int a1 = (code >> 3) & 1, k1 = ((code >> 4) + sflip) & 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h0[c] = q[c] + mul_ik(a0 ? q[9 + c] : q[6 + c], k0);
        h1[c] = q[3 + c] + mul_ik(a1 ? q[9 + c] : q[6 + c], k1);
    }
}

// One hop of an unrolled site sum: the half spinor from the halo (remote)
// or projected from the local neighbour.
template <int P, int D, int MU, int S, int LF, bool HALO>
__device__ __forceinline__ void dd_hop_one(cx<typename Prec<P>::real> (&acc)[12], const char* in, long long Vh,
                                           int nb, const void* links, long long li, unsigned cross,
                                           const cx<float>* ph, const char* halo, long long fs, long long f,
                                           bool remote)
{
    using T = typename Prec<P>::real;
    if (HALO && remote) {
        cx<T> h0[3], h1[3];
        float nrm;
        load_half<P>(h0, h1, nrm, halo, fs, f);
        hop_apply<P, D, MU, S, LF>(acc, h0, h1, links, Vh, li, cross, ph, nrm);
    } else {  // the undivided kernel's own hop (its load schedule and arithmetic)
        hop_one<P, D, MU, S, LF>(acc, in, Vh, nb, links, Vh, (int)li, cross, ph);
    }
}

// acc = H in at block site i: like hop_site, with the hops in `remote` read
// from the halo (halo(mu, side) at face index f[mu]).
template <int P, bool DAG, int LF, bool HALO>
__device__ __forceinline__ void dd_hop_site(cx<typename Prec<P>::real> (&acc)[12], const DDArgs& A, const char* in,
                                            const void* links, int i, const int (&nb)[8], unsigned cross,
                                            unsigned remote, const char* const (&halo)[4][2], const long long (&f)[4])
{
    using T = typename Prec<P>::real;
    const long long Vh = A.g.Vh;
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = {(T)0, (T)0};
    if constexpr (P == WL_DF64 && LF == 0) {
#pragma unroll 1
        for (int d = 0; d < 8; ++d) {
            cx<T> h0[3], h1[3];
            if (HALO && ((remote >> d) & 1)) {
                float unused;
                load_half<P>(h0, h1, unused, halo[d >> 1][d & 1], A.fs[d >> 1], f[d >> 1]);
            } else {
                cx<T> q[12];
                load_spinor_ro<P>(q, in, Vh, nb[d]);
                project_loop<P, DAG>(h0, h1, q, d);
            }
            const unsigned code = hop_code(d >> 1);
            const int sflip = ((d & 1) ? DAG == false : DAG == true) ? 0 : 2;
            const int b2 = (code >> 6) & 1, k2 = ((code >> 7) + sflip) & 3;
            const int b3 = (code >> 9) & 1, k3 = ((code >> 10) + sflip) & 3;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                cx<T> w[3];
                load_link_row<P>(w, links, Vh, d, i, a);
                const cx<T> u0 = dot3(w[0], w[1], w[2], h0), u1 = dot3(w[0], w[1], w[2], h1);
                acc[a] = acc[a] + u0;
                acc[3 + a] = acc[3 + a] + u1;
                acc[6 + a] = acc[6 + a] + mul_ik(b2 ? u1 : u0, k2);
                acc[9 + a] = acc[9 + a] + mul_ik(b3 ? u1 : u0, k3);
            }
        }
    } else {
        constexpr int F = DAG ? +1 : -1;
        constexpr int B = -F;
        const cx<float>* ph = A.ph;
        // x is never cut: its hops are always local
        dd_hop_one<P, 0, 0, F, LF, false>(acc, in, Vh, nb[0], links, i, cross, ph, nullptr, 0, 0, false);
        dd_hop_one<P, 1, 0, B, LF, false>(acc, in, Vh, nb[1], links, i, cross, ph, nullptr, 0, 0, false);
        dd_hop_one<P, 2, 1, F, LF, HALO>(acc, in, Vh, nb[2], links, i, cross, ph, halo[1][0], A.fs[1], f[1], (remote >> 2) & 1);
        dd_hop_one<P, 3, 1, B, LF, HALO>(acc, in, Vh, nb[3], links, i, cross, ph, halo[1][1], A.fs[1], f[1], (remote >> 3) & 1);
        dd_hop_one<P, 4, 2, F, LF, HALO>(acc, in, Vh, nb[4], links, i, cross, ph, halo[2][0], A.fs[2], f[2], (remote >> 4) & 1);
        dd_hop_one<P, 5, 2, B, LF, HALO>(acc, in, Vh, nb[5], links, i, cross, ph, halo[2][1], A.fs[2], f[2], (remote >> 5) & 1);
        dd_hop_one<P, 6, 3, F, LF, HALO>(acc, in, Vh, nb[6], links, i, cross, ph, halo[3][0], A.fs[3], f[3], (remote >> 6) & 1);
        dd_hop_one<P, 7, 3, B, LF, HALO>(acc, in, Vh, nb[7], links, i, cross, ph, halo[3][1], A.fs[3], f[3], (remote >> 7) & 1);
    }
}

// ---------------------------------------------------------------------------
// pack: the faces of the input field a launch will need from this block
// ---------------------------------------------------------------------------

// A segment of the concatenated face index space of one pack launch: the
// sites of one (launch parity, direction, side) face.  Side 0 is the block's
// x_mu = 0 face, projected for the forward hop of the backward neighbour;
// side 1 the x_mu = L_mu - 1 face, for the backward hop of the forward
// neighbour.
struct DDSeg {
    int pidx, mu, side;
    long long start, count;
};

struct DDPackArgs {
    Geom g;
    DDSeg seg[12];
    int nseg;
    long long total;        // sum of the segment counts
    long long hoff[2][4][2];
    long long rs_in;
    const char* in[kMaxDomains][2];  // input field of launch parity k (parity 1 - p)
    // region the (mu, side) faces of a block are written to: its own send
    // region, or (direct exchange) the receiving neighbour's halo region
    char* dst[kMaxDomains][4][2];
};

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// One launch description of the decomposed hopping term over all blocks:
// like HopLaunch, with per-block field pointers.
struct DDLaunch {
    int prec = WL_F32;
    int dagger = 0;
    int parity0 = 0, nparity = 1;
    int nrhs = 1;
    const void* in[kMaxDomains][2] = {};
    void* out[kMaxDomains][2] = {};
    const void* x1[kMaxDomains][2] = {};
    const void* x2[kMaxDomains][2] = {};
    const void* w[kMaxDomains][2] = {};
    long long rs_in = 0, rs_out = 0, rs_x1 = 0, rs_x2 = 0, rs_w = 0;
    double a = 1.0, b1 = 0.0;
    int cl_mode = 0;  // clover epilogue mode (hop.cuh kClNone / kClX2 / kClOut)
    int cl_inv[2] = {0, 0};  // per launch parity: 0 = A, 1 = A^-1
    // fused reduction: the per-block local sums are added over the blocks and
    // the global (w, out), ||out||^2 written to dot_out[dom] + rhs * dot_stride
    bool dot = false;
    double* dot_out[kMaxDomains] = {};
    int dot_stride = 3;
    const int* active[kMaxDomains] = {};  // skip right-hand sides whose flag is 0
    int active_stride = 1;
};

struct DDSolveWork;  // dd_solve.cu

}  // namespace wl

// A lattice cut into blocks; this process holds blocks gid[0..ndom) on one
// GPU, the others (if any) are reached through the transport.  Blocks are
// numbered lexicographically over the grid, y fastest.  Arrays indexed by d
// are per held block; peer[] holds global block numbers.
struct wl_dd_s {
    wl_lattice global;
    wl::Geom gglob;
    wl::Geom gloc;  // one block
    int grid[4];
    int nblk = 0;  // blocks of the whole decomposition
    int ndom = 0;  // blocks held here
    int cut = 0;   // bit mu: direction mu cut
    int device = 0;
    int gid[wl::kMaxDomains] = {};
    std::vector<int> local_of;  // global block -> held index, -1 when held elsewhere
    wl_gauge dom[wl::kMaxDomains] = {};
    int coord[wl::kMaxDomains][4] = {};
    int peer[wl::kMaxDomains][4][2] = {};  // neighbour block [mu][0: backward, 1: forward]
    unsigned edge[wl::kMaxDomains] = {};
    long long fs[4] = {0, 0, 0, 0};
    // interior and boundary half indices (the same for every block)
    int* isites = nullptr;
    int* bsites = nullptr;
    long long nint = 0, nbnd = 0;
    // halo regions: recv (faces received) and send (packed faces), per block,
    // each holding [launch parity][mu][side] segments (offsets from dd_segments)
    char* recv[wl::kMaxDomains] = {};
    char* send[wl::kMaxDomains] = {};
    size_t region_bytes = 0;  // capacity of each recv / send region
    // per-block local sums of the reductions (3 doubles per right-hand side)
    double* loc = nullptr;
    int loc_rhs = 0;
    int direct = 0;  // 1: the pack writes straight into held neighbours' halos (no copy kernel)
    cudaStream_t comm = nullptr;
    cudaEvent_t ev_packed = nullptr, ev_exchanged = nullptr;
    // reduction partials of all blocks and the per-block local sums
    double* partial = nullptr;
    long long part_dom_stride = 0;
    int part_max_blocks = 0, part_rhs = 0;
    // transport to the blocks held elsewhere; stage holds the sums that cross
    // processes (3 doubles per right-hand side)
    bool has_tr = false;
    wl_dd_transport tr = {};
    double* stage = nullptr;
    int stage_rhs = 0;
    std::vector<wl_dd_msg> msgs;
    wl::DDSolveWork* sw = nullptr;  // solver workspace (dd_solve.cu)
};

namespace wl {

// The decomposed hopping term over all blocks (dd.cu): pack, exchange,
// interior, boundary and, with h.dot, the reduction over the blocks.
int dd_launch_hop(wl_dd dd, const DDLaunch& h, cudaStream_t s);
// Sum each block's local 3-tuples (loc[dom] + rhs * 3) over the blocks in
// block order and write the totals to out[dom] + rhs * out_stride for every
// block: the allreduce of the solver's dots.
int dd_allreduce(wl_dd dd, double* const* loc, double* const* out, int out_stride, int nrhs,
                 const int* const* active, int active_stride, cudaStream_t s);
// Solver workspace release (dd_solve.cu).
void dd_free_solver(wl_dd dd);
// Halo segments of one hopping application (launch parities np, precision P,
// nrhs): offsets hoff[k][mu][side] within a region, segment list and the
// region size; identical on every block of the decomposition.
void dd_segments(const Geom& g, int cut, int P, int nrhs, int np, long long (&hoff)[2][4][2], DDSeg (&seg)[12],
                 int& nseg, long long& total, long long& bytes);
// Make dd->stage hold 3 * nrhs doubles.
int dd_ensure_stage(wl_dd dd, int nrhs);
// Sum the 3 * nrhs doubles of dd->stage over the processes (no-op without a
// transport).
int dd_cross_sum(wl_dd dd, int nrhs, cudaStream_t s);

}  // namespace wl
