// Kernels of the domain-decomposed hopping term (dd.cuh): face packing,
// interior and boundary sweeps, and the sum over the blocks.  Templates over
// precision P, dagger DAG, fused reduction DOT, link format LF, clover mode CL
// (the epilogue's, as in hop.cuh) and the site set (BND: boundary sites, whose
// hops may read the halo).  Each translation unit instantiates one (LF, CL)
// family, so they compile in parallel: dd_hop.cu (LF = 0, no clover, and the
// pack kernel), dd_hop_r12.cu (LF = 1), dd_hop_clover.cu and
// dd_hop_r12_clover.cu (the two clover modes).
#pragma once

#include "dd.cuh"
#include "hop_kernels.cuh"

namespace wl {

static constexpr int kDDBlock = 128;

// Half index of the j-th site of the interior box (the order of increasing
// half index, as the site list it replaces).
__device__ __forceinline__ int box_site(const DDArgs& A, long long j)
{
    const int q = (int)j;
    const int r0 = geo_div(A.g, 0, q);  // j / Lxh
    const int xh = q - r0 * A.g.Lxh;
    const int r1 = A.bm[1] ? (int)(__umulhi((unsigned)r0, A.bm[1]) >> A.bsh[1]) : r0;
    const int y = r0 - r1 * A.bn[1];
    const int t = A.bm[2] ? (int)(__umulhi((unsigned)r1, A.bm[2]) >> A.bsh[2]) : r1;
    const int z = r1 - t * A.bn[2];
    return xh + A.g.Lxh * ((A.bo[1] + y) + A.g.L[1] * ((A.bo[2] + z) + A.g.L[2] * (A.bo[3] + t)));
}

// Output site j of the launch's site set, launch parity pidx: the hopping
// term (halo reads on boundary sites) and the epilogue; with DOT its (w, out),
// ||out||^2 are added to part.
template <int P, bool DAG, bool DOT, int LF, bool BND, int CL>
__device__ __forceinline__ void dd_site(const DDArgs& A, const DDDom& D, int rhs, int pidx, long long j,
                                        typename Prec<P>::real (&part)[3])
{
    using T = typename Prec<P>::real;
    const int i = A.sites ? A.sites[j] : A.box ? box_site(A, j) : (int)(A.site0 + j);
    const int p = A.parity0 + pidx;
    int c[4], xh, nb[8];
    half_coords(A.g, p, i, c, xh);
    const unsigned faces = block_neighbours(A.g, i, c, xh, nb);
    const unsigned cross = faces & D.edge;  // hops that cross the global boundary
    const char* halo[4][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    long long f[4] = {0, 0, 0, 0};
    unsigned remote = 0;
    if constexpr (BND) {
        remote = faces & A.cutmask;
#pragma unroll
        for (int mu = 1; mu < 4; ++mu)
            if (A.fs[mu]) {
                f[mu] = face_index(A.g, mu, c, xh);
                const long long seg_rs = halo_face_bytes(P, A.fs[mu]);
                halo[mu][0] = D.halo + A.hoff[pidx][mu][0] + rhs * seg_rs;
                halo[mu][1] = D.halo + A.hoff[pidx][mu][1] + rhs * seg_rs;
            }
    }
    cx<T> acc[12];
    dd_hop_site<P, DAG, LF, BND>(acc, A, D.in[pidx] + rhs * A.rs_in, D.links[pidx], i, nb, cross, remote, halo, f);
    auto at = [&](const char* q, long long rs) -> const char* { return q ? q + rhs * rs : nullptr; };
    T pt[3] = {0, 0, 0};
    epilogue_ptrs<P, DOT, CL>(acc, A.a, at(D.x1[pidx], A.rs_x1), at(D.x2[pidx], A.rs_x2), A.b1,
                              at(D.w[pidx], A.rs_w), D.out[pidx] + rhs * A.rs_out, A.g.Vh, i, pt, D.cl[pidx]);
    if (DOT)
        for (int k = 0; k < 3; ++k) part[k] += pt[k];
}

// Plain launches: one site per thread, grid.x = blocks_per_parity x parities.
// Launches with a fused reduction: a capped grid loops over the sites of both
// parities, so the per-block partials the finishing launch adds up are few.
template <int P, bool DAG, bool DOT, int LF, bool BND, int CL>
__global__ void __launch_bounds__(kDDBlock, (MinBlocks<P, DOT>::value * 2)) dd_hop_kernel(const DDArgs A)
{
    using T = typename Prec<P>::real;
    const int rhs = blockIdx.y, dom = blockIdx.z;
    const DDDom& D = A.d[dom];
    if (D.active && D.active[(long long)rhs * A.active_stride] == 0) return;  // uniform per block
    T part[3] = {0, 0, 0};
    if constexpr (!DOT) {
        const int pidx = blockIdx.x / A.blocks_per_parity;
        const long long j = (long long)(blockIdx.x - pidx * A.blocks_per_parity) * kDDBlock + threadIdx.x;
        if (j < A.nsites) dd_site<P, DAG, DOT, LF, BND, CL>(A, D, rhs, pidx, j, part);
    } else {
        const long long total = (long long)A.nparity * A.nsites;
        for (long long q = blockIdx.x * (long long)kDDBlock + threadIdx.x; q < total;
             q += (long long)gridDim.x * kDDBlock) {
            const int pidx = q >= A.nsites ? 1 : 0;
            dd_site<P, DAG, DOT, LF, BND, CL>(A, D, rhs, pidx, q - pidx * A.nsites, part);
        }
        typename RedType<T>::type wp[3] = {(typename RedType<T>::type)part[0], (typename RedType<T>::type)part[1],
                                           (typename RedType<T>::type)part[2]};
        warp_sum<3>(wp);
        double bp[3] = {(double)wp[0], (double)wp[1], (double)wp[2]};
        __shared__ double sh[3 * 32];
        block_sum_warps<3>(bp, sh);
        if (threadIdx.x == 0) {
            double* o = A.partial + dom * A.dom_stride + ((long long)rhs * A.max_blocks + A.block0 + blockIdx.x) * 3;
            o[0] = bp[0];
            o[1] = bp[1];
            o[2] = bp[2];
        }
    }
}

// The half spinor a face carries: FP16 storage unscaled with its norm (the
// operands of the undivided FP16 hop), the others as load_project forms them.
template <int P, int MU, int S>
__device__ __forceinline__ void pack_project(cx<typename Prec<P>::real> (&h0)[3], cx<typename Prec<P>::real> (&h1)[3],
                                             float& nrm, const void* in, long long Vh, int i)
{
    if constexpr (P == WL_F16) load_project_f16<MU, S>(h0, h1, nrm, in, Vh, i);
    else load_project<P, MU, S>(h0, h1, in, Vh, i);
}

// The spin-projected half spinors of the faces a neighbouring block needs.
template <int P, bool DAG>
__global__ void __launch_bounds__(kDDBlock) dd_pack_kernel(const DDPackArgs A)
{
    using T = typename Prec<P>::real;
    const int rhs = blockIdx.y, dom = blockIdx.z;
    const long long j = blockIdx.x * (long long)kDDBlock + threadIdx.x;
    if (j >= A.total) return;
    int k = 0;
    while (k + 1 < A.nseg && j >= A.seg[k + 1].start) ++k;
    const DDSeg& S = A.seg[k];
    const long long f = j - S.start;
    // face index -> half index at x_mu = 0 (side 0) or L_mu - 1 (side 1)
    const long long s_mu = S.mu == 1 ? A.g.sy : S.mu == 2 ? A.g.sz : A.g.st;
    const long long above = f / s_mu, below = f - above * s_mu;
    const long long xmu = S.side ? A.g.L[S.mu] - 1 : 0;
    const int i = (int)(below + xmu * s_mu + above * s_mu * A.g.L[S.mu]);
    const char* in = A.in[dom][S.pidx] + rhs * A.rs_in;
    cx<T> h0[3], h1[3];
    float nrm = 1.0f;
    const int d = 2 * S.mu + S.side;  // the hop of the receiving block
    if constexpr (P == WL_DF64) {
        cx<T> q[12];
        load_spinor_ro<P>(q, in, A.g.Vh, i);
        project_loop<P, DAG>(h0, h1, q, d);
    } else {
        constexpr int F = DAG ? +1 : -1;  // forward projector sign
        constexpr int B = -F;
        switch (d) {
            case 2: pack_project<P, 1, F>(h0, h1, nrm, in, A.g.Vh, i); break;
            case 3: pack_project<P, 1, B>(h0, h1, nrm, in, A.g.Vh, i); break;
            case 4: pack_project<P, 2, F>(h0, h1, nrm, in, A.g.Vh, i); break;
            case 5: pack_project<P, 2, B>(h0, h1, nrm, in, A.g.Vh, i); break;
            case 6: pack_project<P, 3, F>(h0, h1, nrm, in, A.g.Vh, i); break;
            default: pack_project<P, 3, B>(h0, h1, nrm, in, A.g.Vh, i); break;
        }
    }
    store_half<P>(A.dst[dom][S.mu][S.side] + A.hoff[S.pidx][S.mu][S.side] + rhs * halo_face_bytes(P, S.count),
                  S.count, f, h0, h1, nrm);
}

// Launchers of one link format and clover mode (LF = 1 exists for FP32 /
// FP16 only).
template <int LF, int CL>
struct DDKernels {
    static void hop(int prec, bool dagger, bool dot, bool bnd, const DDArgs& A, dim3 grid, cudaStream_t s);
};

// Blocks of a launch with a fused reduction: about four resident 128-thread
// blocks per SM, shared by the held blocks, at most one per 128 sites.
inline int dd_reducing_grid(long long sites, int ndom, int num_sms)
{
    const long long need = (sites + kDDBlock - 1) / kDDBlock;
    const long long g = std::max<long long>(1, 4LL * num_sms / std::max(1, ndom));
    return (int)std::max<long long>(1, std::min(need, g));
}

// The packed half spinor depends on neither (dd_hop.cu).
void dd_pack(int prec, bool dagger, const DDPackArgs& A, dim3 grid, cudaStream_t s);

template <int LF, int CL, int P, bool BND>
static void dd_hop_p(bool dagger, bool dot, const DDArgs& A, dim3 grid, cudaStream_t s)
{
    if (dagger) {
        if (dot) dd_hop_kernel<P, true, true, LF, BND, CL><<<grid, kDDBlock, 0, s>>>(A);
        else dd_hop_kernel<P, true, false, LF, BND, CL><<<grid, kDDBlock, 0, s>>>(A);
    } else {
        if (dot) dd_hop_kernel<P, false, true, LF, BND, CL><<<grid, kDDBlock, 0, s>>>(A);
        else dd_hop_kernel<P, false, false, LF, BND, CL><<<grid, kDDBlock, 0, s>>>(A);
    }
}

template <int LF, int CL, int P>
static void dd_hop_pb(bool dagger, bool dot, bool bnd, const DDArgs& A, dim3 grid, cudaStream_t s)
{
    if (bnd) dd_hop_p<LF, CL, P, true>(dagger, dot, A, grid, s);
    else dd_hop_p<LF, CL, P, false>(dagger, dot, A, grid, s);
}

template <int LF, int CL>
void DDKernels<LF, CL>::hop(int prec, bool dagger, bool dot, bool bnd, const DDArgs& A, dim3 grid, cudaStream_t s)
{
    if (prec == WL_F32) dd_hop_pb<LF, CL, WL_F32>(dagger, dot, bnd, A, grid, s);
    else if (prec == WL_F16) dd_hop_pb<LF, CL, WL_F16>(dagger, dot, bnd, A, grid, s);
    else if constexpr (LF == 0) {
        if (prec == WL_F64) dd_hop_pb<LF, CL, WL_F64>(dagger, dot, bnd, A, grid, s);
        else dd_hop_pb<LF, CL, WL_DF64>(dagger, dot, bnd, A, grid, s);
    }
}

}  // namespace wl
