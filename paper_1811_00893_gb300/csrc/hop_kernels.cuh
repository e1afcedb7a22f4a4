// The hopping kernels of Eq. 1 (and, through the epilogue's clover modes, of
// Eq. 2), as templates over precision P, dagger DAG, fused reduction DOT and
// clover mode CL.  dslash.cu instantiates the Wilson kernels (CL = 0),
// dslash_clover_x2.cu and dslash_clover_out.cu the clover ones, so the three
// compile in parallel.
//
// One thread per output site of one parity.  The eight neighbour spinors are
// spin-projected to half spinors (12 reals), multiplied by the link (folded
// with the boundary phase, backward links pre-daggered at set-up) and
// reconstructed into the four spin components.  Spinors and links live in
// structure-of-arrays planes, so consecutive threads read consecutive 16-byte
// words; the neighbour spinors' eightfold reuse is served by L1/L2 (the y, z,
// t neighbours are the same half index shifted by a row, plane or slab).
#pragma once

#include "hop.cuh"

namespace wl {

// One right-hand side per grid row, one output site per thread and step of a
// grid-stride loop over the output sites of both parities in the launch
// (plain launches cover every site in one step; launches with a fused
// reduction use a grid of resident blocks, so few partials are left).
// Resident 256-thread blocks per SM each kernel is compiled for: 2 caps the
// registers at 128 so that more warps hide latency -- memory latency for
// FP32/FP16, the long dependent FP32 chains of the double-float type (measured
// 6-15% faster than uncapped on GB300).  FP64 keeps all the registers it
// needs (capped, it spills without getting faster).
#ifndef WL_MINBLOCKS_F32
#define WL_MINBLOCKS_F32 2
#endif
#ifndef WL_MINBLOCKS_F16
#define WL_MINBLOCKS_F16 2
#endif
#ifndef WL_MINBLOCKS_F64
#define WL_MINBLOCKS_F64 1
#endif
#ifndef WL_MINBLOCKS_DF64
#define WL_MINBLOCKS_DF64 2
#endif
template <int P, bool DOT>
struct MinBlocks {
    static constexpr int base = P == WL_F64    ? WL_MINBLOCKS_F64
                                : P == WL_DF64 ? WL_MINBLOCKS_DF64
                                : P == WL_F32  ? WL_MINBLOCKS_F32
                                               : WL_MINBLOCKS_F16;
    static constexpr int value = DOT && base > 2 ? 2 : base;  // the reducing loop needs more
};

// Ask L2 for the site's epilogue operands (x1, x2, w) before the stencil
// starts, so that their loads after the eight hops do not wait on HBM.  A
// prefetch holds no register.  Measured: FP16 solve 149.8 -> 148.5 ms, but
// the FP32 hop 141 -> 151 us (its register budget tips into spills), so only
// the FP16 kernels prefetch.  WL_PREFETCH_EPILOGUE=0 builds without it.
#ifndef WL_PREFETCH_EPILOGUE
#define WL_PREFETCH_EPILOGUE 1
#endif
template <int P>
__device__ __forceinline__ void prefetch_spinor_l2(const char* base, long long Vh, long long i)
{
    constexpr int planes = (P == WL_F32) ? 6 : (P == WL_F16) ? 3 : 12;  // 16-byte planes
#pragma unroll
    for (int k = 0; k < planes; ++k)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (k * Vh + i) * 16));
    if (P == WL_F16) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + 3 * Vh * 16 + i * 4));
}

template <int P, bool DAG, bool DOT, int CL, int LF>
__device__ __forceinline__ void hop_kernel_site(const HopArgs& A, int rhs, int pidx, int i,
                                                typename Prec<P>::real (&part)[3])
{
    using T = typename Prec<P>::real;
    if (WL_PREFETCH_EPILOGUE && P == WL_F16) {
        if (A.x1[pidx]) prefetch_spinor_l2<P>(A.x1[pidx] + rhs * A.rs_x1, A.g.Vh, i);
        if (A.x2[pidx]) prefetch_spinor_l2<P>(A.x2[pidx] + rhs * A.rs_x2, A.g.Vh, i);
        if (DOT && A.w[pidx] && A.w[pidx] != A.x1[pidx])
            prefetch_spinor_l2<P>(A.w[pidx] + rhs * A.rs_w, A.g.Vh, i);
    }
    cx<T> acc[12];
    int nb[8];
    unsigned cross = 0;
    if constexpr (LF >= 1) neighbours(A.g, A.parity0 + pidx, i, nb, cross);
    else neighbours(A.g, A.parity0 + pidx, i, nb);
    hop_site<P, DAG, LF>(acc, nb, A.g.Vh, A.in[pidx] + rhs * A.rs_in, A.links[pidx], A.g.Vh, i, cross,
                         A.ph);
    T pt[3] = {0, 0, 0};
    epilogue<P, DOT, CL>(acc, A, pidx, rhs, i, pt);
    if (DOT)
        for (int k = 0; k < 3; ++k) part[k] += pt[k];
}

template <int P, bool DAG, bool DOT, int CL, int LF>
__global__ void __launch_bounds__(256, (MinBlocks<P, DOT>::value)) hop_kernel(const HopArgs A)
{
    const int rhs = blockIdx.y;
    if (A.active && A.active[rhs * A.active_stride] == 0) return;  // uniform per block
    using T = typename Prec<P>::real;
    const long long total = (long long)A.nparity * A.g.Vh;
    T tpart[3] = {0, 0, 0};  // this thread's sites, in the kernel's arithmetic
    if constexpr (!DOT) {  // one site per thread; the block's parity is fixed
        const int pidx = blockIdx.x / A.blocks_per_parity;
        const int i = (blockIdx.x - pidx * A.blocks_per_parity) * blockDim.x + threadIdx.x;
        if (i < A.g.Vh) hop_kernel_site<P, DAG, DOT, CL, LF>(A, rhs, pidx, i, tpart);
        (void)total;
    } else {
        for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total;
             j += (long long)gridDim.x * blockDim.x) {
            const int pidx = j >= A.g.Vh ? 1 : 0;
            hop_kernel_site<P, DAG, DOT, CL, LF>(A, rhs, pidx, (int)(j - pidx * A.g.Vh), tpart);
        }
        // warp totals in the arithmetic type (FP32 for the narrow types), FP64 from there
        typename RedType<T>::type wp[3] = {(typename RedType<T>::type)tpart[0],
                                           (typename RedType<T>::type)tpart[1],
                                           (typename RedType<T>::type)tpart[2]};
        warp_sum<3>(wp);
        double part[3] = {(double)wp[0], (double)wp[1], (double)wp[2]};
        __shared__ double sh[3 * 32];
        block_sum_warps<3>(part, sh);
        if (A.partials_only) {
            if (threadIdx.x == 0)
                for (int k = 0; k < 3; ++k)
                    A.red.partial[((long long)rhs * A.red.max_blocks + blockIdx.x) * 3 + k] = part[k];
            return;
        }
        double tot[3];
        if (grid_sum<3>(part, tot, A.red, rhs, gridDim.x, blockIdx.x, sh)) {
            double* o = A.dot_out + (long long)rhs * A.dot_stride;
            o[0] = tot[0];
            o[1] = tot[1];
            o[2] = tot[2];
        }
    }
}

template <int P, bool DAG, bool DOT, int CL, int LF>
__global__ void __launch_bounds__(256, (MinBlocks<P, DOT>::value)) hop_mrhs_kernel(const HopArgs A, int nrhs)
{
    using T = typename Prec<P>::real;
    extern __shared__ __align__(16) char smem[];
    const int pidx = blockIdx.x / A.blocks_per_parity;
    const int p = A.parity0 + pidx;
    const int base = (blockIdx.x - pidx * A.blocks_per_parity) * kTile;
    const int n = (int)min((long long)kTile, A.g.Vh - base);
    stage_links<P, LF>(smem, (const char*)A.links[pidx], A.g.Vh, base, n);
    double* bpart = (double*)(smem + LinkLayout<P, LF>::bytes * kTile);
    __syncthreads();
    const int lane = threadIdx.x, i = base + lane;
    const bool valid = lane < n;
    int nb[8];
    unsigned cross = 0;
    if (valid) {
        if constexpr (LF >= 1) neighbours(A.g, p, i, nb, cross);
        else neighbours(A.g, p, i, nb);
    }
    for (int r = threadIdx.y; r < nrhs; r += blockDim.y) {
        const bool act = !A.active || A.active[r * A.active_stride] != 0;  // warp-uniform
        T part[3] = {0, 0, 0};
        if (act && valid) {
            cx<T> acc[12];
            hop_site<P, DAG, LF>(acc, nb, A.g.Vh, A.in[pidx] + r * A.rs_in, smem, kTile, lane, cross, A.ph);
            epilogue<P, DOT, CL>(acc, A, pidx, r, i, part);
        }
        if (DOT) {  // 32 sites in FP32 (FP64 for the wide types), then FP64 from here on
            typename RedType<T>::type rp[3] = {(typename RedType<T>::type)part[0],
                                               (typename RedType<T>::type)part[1],
                                               (typename RedType<T>::type)part[2]};
            warp_sum<3>(rp);
            if (lane == 0)
                for (int k = 0; k < 3; ++k) bpart[3 * r + k] = (double)rp[k];
        }
    }
    if (!DOT) return;
    // every block leaves its per-rhs partials; a finishing launch (one block
    // per right-hand side) adds them up in block order
    __syncthreads();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int e = tid; e < 3 * nrhs; e += nt) {
        const int r = e / 3, k = e - 3 * r;
        A.red.partial[((long long)r * A.red.max_blocks + blockIdx.x) * 3 + k] = bpart[e];
    }
}

// Persistent, software-pipelined form of hop_mrhs_kernel for the narrow
// types: a grid of resident blocks walks the 32-site tiles round-robin
// (tile = blockIdx.x + k * gridDim.x, a fixed assignment, so the reduction
// order is deterministic); while its warps compute on one tile's links the
// block already copies the next tile's links into the other half of a
// double buffer with cp.async.  Partial sums are written per tile, as in
// hop_mrhs_kernel, and added up in tile order by the finishing launch.
template <int P, bool DAG, bool DOT, int CL, int LF>
__global__ void __launch_bounds__(256, 2) hop_mrhs_pipe_kernel(const HopArgs A, int nrhs, int ntiles)
{
    using T = typename Prec<P>::real;
    extern __shared__ __align__(16) char smem[];
    constexpr int kBuf = LinkLayout<P, LF>::bytes * kTile;
    double* bpart = (double*)(smem + 2 * kBuf);
    const int lane = threadIdx.x;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    auto tile_at = [&](int t, int& pidx, int& base, int& n) {
        pidx = t / A.blocks_per_parity;
        base = (t - pidx * A.blocks_per_parity) * kTile;
        n = (int)min((long long)kTile, A.g.Vh - base);
    };
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    {
        int pidx, base, n;
        tile_at(tile, pidx, base, n);
        stage_links_async<P, LF>(smem, (const char*)A.links[pidx], A.g.Vh, base, n);
        cp_async_commit();
    }
    for (int it = 0; tile < ntiles; ++it) {
        const int next = tile + gridDim.x;
        if (next < ntiles) {  // prefetch the next tile into the other buffer
            int pidx, base, n;
            tile_at(next, pidx, base, n);
            stage_links_async<P, LF>(smem + ((it + 1) & 1) * kBuf, (const char*)A.links[pidx], A.g.Vh,
                                 base, n);
        }
        cp_async_commit();  // (an empty group on the last tile)
        cp_async_wait<1>();  // this tile's copies have landed
        __syncthreads();
        const char* links = smem + (it & 1) * kBuf;
        int pidx, base, n;
        tile_at(tile, pidx, base, n);
        const int p = A.parity0 + pidx;
        const int i = base + lane;
        const bool valid = lane < n;
        int nb[8];
        unsigned cross = 0;
        if (valid) {
            if constexpr (LF >= 1) neighbours(A.g, p, i, nb, cross);
            else neighbours(A.g, p, i, nb);
        }
        for (int r = threadIdx.y; r < nrhs; r += blockDim.y) {
            const bool act = !A.active || A.active[r * A.active_stride] != 0;  // warp-uniform
            T part[3] = {0, 0, 0};
            if (act && valid) {
                cx<T> acc[12];
                hop_site<P, DAG, LF>(acc, nb, A.g.Vh, A.in[pidx] + r * A.rs_in, links, kTile, lane, cross,
                                     A.ph);
                epilogue<P, DOT, CL>(acc, A, pidx, r, i, part);
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
        if (DOT) {
            __syncthreads();
            for (int e = tid; e < 3 * nrhs; e += nt) {
                const int r = e / 3, k = e - 3 * r;
                A.red.partial[((long long)r * A.red.max_blocks + tile) * 3 + k] = bpart[e];
            }
        }
        __syncthreads();  // the buffer and bpart are reused by the tile after next
        tile = next;
    }
}

// FP64 hopping term for small lattices, where one thread per site leaves
// most SMs with less than a warp and the kernel's time is the latency of one
// thread's dependent FP64 chain: three threads per output site, one colour
// row a each (output components 3 s + a).  Each projects the full neighbour
// spinors (the three rows read them from L1) and applies row a of every link,
// a third of hop_kernel's chain per thread and no exchange between the three.
// Every output component sees hop_kernel's operations in the same order.
// Block: kRowSites sites x 3 rows (thread t: row t / kRowSites); a reducing
// launch leaves one partial per block for the finishing launch.  32 sites per
// block spread an 8^4 lattice's 2 x 2,048 sites over 128 SMs: on small lattices
// the FP64 pipes of the SMs a launch reaches are its limit.
static constexpr int kRowSites = 32;

template <int D, int MU, int S>
__device__ __forceinline__ void hop_row(cx<double> (&acc)[12], const char* in, long long Vh, int nb,
                                        const void* links, int i, int a)
{
    cx<double> h0[3], h1[3], w[3];
    load_project<WL_F64, MU, S>(h0, h1, in, Vh, nb);
    load_link_row<WL_F64>(w, links, Vh, D, i, a);
    reconstruct<MU, S>(acc, 0, dot3(w[0], w[1], w[2], h0), dot3(w[0], w[1], w[2], h1));
}

template <bool DAG, bool DOT>
__global__ void __launch_bounds__(3 * kRowSites) hop_rows_kernel(const HopArgs A)
{
    const int rhs = blockIdx.y;
    if (A.active && A.active[rhs * A.active_stride] == 0) return;  // uniform per block
    const int pidx = blockIdx.x / A.blocks_per_parity;
    const int a = threadIdx.x / kRowSites;
    const int i = (blockIdx.x - pidx * A.blocks_per_parity) * kRowSites + (threadIdx.x - a * kRowSites);
    const long long Vh = A.g.Vh;
    double part[3] = {0, 0, 0};
    if (i < Vh) {
        int nb[8];
        neighbours(A.g, A.parity0 + pidx, i, nb);
        const char* in = A.in[pidx] + rhs * A.rs_in;
        const void* links = A.links[pidx];
        cx<double> acc[12];  // the rows of colour a at 0, 3, 6, 9
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = {0.0, 0.0};
        constexpr int F = DAG ? +1 : -1;  // forward projector sign
        constexpr int B = -F;
        hop_row<0, 0, F>(acc, in, Vh, nb[0], links, i, a);
        hop_row<1, 0, B>(acc, in, Vh, nb[1], links, i, a);
        hop_row<2, 1, F>(acc, in, Vh, nb[2], links, i, a);
        hop_row<3, 1, B>(acc, in, Vh, nb[3], links, i, a);
        hop_row<4, 2, F>(acc, in, Vh, nb[4], links, i, a);
        hop_row<5, 2, B>(acc, in, Vh, nb[5], links, i, a);
        hop_row<6, 3, F>(acc, in, Vh, nb[6], links, i, a);
        hop_row<7, 3, B>(acc, in, Vh, nb[7], links, i, a);
        // epilogue (as epilogue_ptrs, on this thread's four components)
        auto at = [&](const char* q, long long rs) -> const double2* {
            return q ? (const double2*)(q + rhs * rs) : nullptr;
        };
        const double2* x1 = at(A.x1[pidx], A.rs_x1);
        const double2* x2 = at(A.x2[pidx], A.rs_x2);
        const double2* w = at(A.w[pidx], A.rs_w);
        double2* out = (double2*)(A.out[pidx] + rhs * A.rs_out);
        const double sa = A.a, b1 = A.b1;
        cx<double> v[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) v[s] = sa * acc[3 * s];
        if (x1)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const double2 t = x1[(3 * s + a) * Vh + i];
                v[s] = v[s] + cx<double>{t.x, t.y};
            }
        if (x2)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const double2 t = x2[(3 * s + a) * Vh + i];
                v[s] = v[s] + b1 * cx<double>{t.x, t.y};
            }
#pragma unroll
        for (int s = 0; s < 4; ++s) out[(3 * s + a) * Vh + i] = make_double2(v[s].re, v[s].im);
        if (DOT) {
            if (w)
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const double2 t = w[(3 * s + a) * Vh + i];
                    part[0] = fma(t.x, v[s].re, fma(t.y, v[s].im, part[0]));
                    part[1] = fma(t.x, v[s].im, fma(-t.y, v[s].re, part[1]));
                }
#pragma unroll
            for (int s = 0; s < 4; ++s) part[2] = fma(v[s].re, v[s].re, fma(v[s].im, v[s].im, part[2]));
        }
    }
    if constexpr (DOT) {
        warp_sum<3>(part);
        __shared__ double sh[3 * 32];
        block_sum_warps<3>(part, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) A.red.partial[((long long)rhs * A.red.max_blocks + blockIdx.x) * 3 + k] = part[k];
    }
}

// Host-side launchers of one clover mode and link format (LF = 1 exists for
// FP32 and FP16 only; other precisions are never requested with it).
template <int CL, int LF = 0>
struct HopKernels {
    static void single(int prec, bool dagger, bool dot, const HopArgs& A, dim3 grid, int block,
                       cudaStream_t s);
    static void multi(int prec, bool dagger, bool dot, const HopArgs& A, int nrhs, dim3 grid,
                      dim3 block, size_t smem, cudaStream_t s);
    // pipelined multi-RHS kernel (FP32 / FP16 only)
    static void pipe(int prec, bool dagger, bool dot, const HopArgs& A, int nrhs, int ntiles, dim3 grid,
                     dim3 block, size_t smem, cudaStream_t s);
    static const void* pipe_kernel(int prec, bool dagger, bool dot);
    // three threads per site (FP64, CL = 0, LF = 0 only), kRowSites sites per block
    static void rows(bool dagger, bool dot, const HopArgs& A, dim3 grid, cudaStream_t s);
    // the reducing single-RHS kernel (for occupancy queries)
    static const void* reducing(int prec, bool dagger);
};

template <int CL, int LF, int P>
static void hop_single_p(bool dagger, bool dot, const HopArgs& A, dim3 grid, int block, cudaStream_t s)
{
    if (dagger) {
        if (dot) hop_kernel<P, true, true, CL, LF><<<grid, block, 0, s>>>(A);
        else hop_kernel<P, true, false, CL, LF><<<grid, block, 0, s>>>(A);
    } else {
        if (dot) hop_kernel<P, false, true, CL, LF><<<grid, block, 0, s>>>(A);
        else hop_kernel<P, false, false, CL, LF><<<grid, block, 0, s>>>(A);
    }
}

template <int CL, int LF, int P>
static void hop_multi_p(bool dagger, bool dot, const HopArgs& A, int nrhs, dim3 grid, dim3 block,
                        size_t smem, cudaStream_t s)
{
    if (dagger) {
        if (dot) hop_mrhs_kernel<P, true, true, CL, LF><<<grid, block, smem, s>>>(A, nrhs);
        else hop_mrhs_kernel<P, true, false, CL, LF><<<grid, block, smem, s>>>(A, nrhs);
    } else {
        if (dot) hop_mrhs_kernel<P, false, true, CL, LF><<<grid, block, smem, s>>>(A, nrhs);
        else hop_mrhs_kernel<P, false, false, CL, LF><<<grid, block, smem, s>>>(A, nrhs);
    }
}

template <int CL, int LF, int P>
static void hop_pipe_p(bool dagger, bool dot, const HopArgs& A, int nrhs, int ntiles, dim3 grid,
                       dim3 block, size_t smem, cudaStream_t s)
{
    if (dagger) {
        if (dot) hop_mrhs_pipe_kernel<P, true, true, CL, LF><<<grid, block, smem, s>>>(A, nrhs, ntiles);
        else hop_mrhs_pipe_kernel<P, true, false, CL, LF><<<grid, block, smem, s>>>(A, nrhs, ntiles);
    } else {
        if (dot) hop_mrhs_pipe_kernel<P, false, true, CL, LF><<<grid, block, smem, s>>>(A, nrhs, ntiles);
        else hop_mrhs_pipe_kernel<P, false, false, CL, LF><<<grid, block, smem, s>>>(A, nrhs, ntiles);
    }
}

template <int CL, int LF, int P>
static const void* pipe_kernel_p(bool dagger, bool dot)
{
    if (dagger)
        return dot ? (const void*)hop_mrhs_pipe_kernel<P, true, true, CL, LF>
                   : (const void*)hop_mrhs_pipe_kernel<P, true, false, CL, LF>;
    return dot ? (const void*)hop_mrhs_pipe_kernel<P, false, true, CL, LF>
               : (const void*)hop_mrhs_pipe_kernel<P, false, false, CL, LF>;
}

// The eight-real link format (LF = 2) exists for FP32 single-RHS launches only.
template <int CL, int LF>
void HopKernels<CL, LF>::pipe(int prec, bool dagger, bool dot, const HopArgs& A, int nrhs, int ntiles,
                          dim3 grid, dim3 block, size_t smem, cudaStream_t s)
{
    if constexpr (LF < 2) {
        if (prec == WL_F32) hop_pipe_p<CL, LF, WL_F32>(dagger, dot, A, nrhs, ntiles, grid, block, smem, s);
        else hop_pipe_p<CL, LF, WL_F16>(dagger, dot, A, nrhs, ntiles, grid, block, smem, s);
    }
}

template <int CL, int LF>
const void* HopKernels<CL, LF>::pipe_kernel(int prec, bool dagger, bool dot)
{
    if constexpr (LF < 2)
        return prec == WL_F32 ? pipe_kernel_p<CL, LF, WL_F32>(dagger, dot) : pipe_kernel_p<CL, LF, WL_F16>(dagger, dot);
    return nullptr;
}

template <int CL, int LF>
void HopKernels<CL, LF>::single(int prec, bool dagger, bool dot, const HopArgs& A, dim3 grid, int block,
                            cudaStream_t s)
{
    if constexpr (LF == 2) {
        if (prec == WL_F32) hop_single_p<CL, LF, WL_F32>(dagger, dot, A, grid, block, s);
    } else {
        if (prec == WL_F32) hop_single_p<CL, LF, WL_F32>(dagger, dot, A, grid, block, s);
        else if (prec == WL_F16) hop_single_p<CL, LF, WL_F16>(dagger, dot, A, grid, block, s);
        else if constexpr (LF == 0) {
            if (prec == WL_F64) hop_single_p<CL, LF, WL_F64>(dagger, dot, A, grid, block, s);
            else hop_single_p<CL, LF, WL_DF64>(dagger, dot, A, grid, block, s);
        }
    }
}

template <int CL, int LF>
void HopKernels<CL, LF>::multi(int prec, bool dagger, bool dot, const HopArgs& A, int nrhs, dim3 grid,
                           dim3 block, size_t smem, cudaStream_t s)
{
    if constexpr (LF < 2) {
        if (prec == WL_F32) hop_multi_p<CL, LF, WL_F32>(dagger, dot, A, nrhs, grid, block, smem, s);
        else if (prec == WL_F16) hop_multi_p<CL, LF, WL_F16>(dagger, dot, A, nrhs, grid, block, smem, s);
        else if constexpr (LF == 0) {
            if (prec == WL_F64) hop_multi_p<CL, LF, WL_F64>(dagger, dot, A, nrhs, grid, block, smem, s);
            else hop_multi_p<CL, LF, WL_DF64>(dagger, dot, A, nrhs, grid, block, smem, s);
        }
    }
}

template <int CL, int LF>
void HopKernels<CL, LF>::rows(bool dagger, bool dot, const HopArgs& A, dim3 grid, cudaStream_t s)
{
    if constexpr (CL == kClNone && LF == 0) {
        const int block = 3 * kRowSites;
        if (dagger) {
            if (dot) hop_rows_kernel<true, true><<<grid, block, 0, s>>>(A);
            else hop_rows_kernel<true, false><<<grid, block, 0, s>>>(A);
        } else {
            if (dot) hop_rows_kernel<false, true><<<grid, block, 0, s>>>(A);
            else hop_rows_kernel<false, false><<<grid, block, 0, s>>>(A);
        }
    }
}

template <int CL, int LF>
const void* HopKernels<CL, LF>::reducing(int prec, bool dagger)
{
    if (prec == WL_F32)
        return dagger ? (const void*)hop_kernel<WL_F32, true, true, CL, LF> : (const void*)hop_kernel<WL_F32, false, true, CL, LF>;
    if constexpr (LF < 2) {
        if (prec == WL_F16)
            return dagger ? (const void*)hop_kernel<WL_F16, true, true, CL, LF> : (const void*)hop_kernel<WL_F16, false, true, CL, LF>;
        if constexpr (LF == 0) {
            if (prec == WL_F64)
                return dagger ? (const void*)hop_kernel<WL_F64, true, true, CL, LF> : (const void*)hop_kernel<WL_F64, false, true, CL, LF>;
            return dagger ? (const void*)hop_kernel<WL_DF64, true, true, CL, LF> : (const void*)hop_kernel<WL_DF64, false, true, CL, LF>;
        }
    }
    return nullptr;
}

}  // namespace wl
