// The even-odd hopping term of the Wilson matrix (Eq. 1) on sm_103a.
//
// One thread per output site of one parity.  The eight neighbour spinors are
// spin-projected to half spinors (12 reals), multiplied by the link (folded
// with the boundary phase, backward links pre-daggered at set-up) and
// reconstructed into the four spin components.  Spinors and links live in
// structure-of-arrays planes, so consecutive threads read consecutive 16-byte
// words; the neighbour spinors' eightfold reuse is served by L1/L2 (the y, z,
// t neighbours are the same half index shifted by a row, plane or slab).
// The epilogue optionally forms out = x1 + b1*x2 + a*H in and accumulates
// the complex dot (w, out) and ||out||^2 into a deterministic grid reduction,
// so the solver's matrix applies carry their reductions for free.
#include "internal.cuh"

namespace wl {

// (1 + S gamma_mu) projection / reconstruction in the chiral basis
// (gamma_5 = diag(1,1,-1,-1)); S = -1 is Eq. 1's forward projector
// (1 - gamma_mu), S = +1 the backward one.  With u0 = W h0, u1 = W h1 the
// four spin rows of (1 + S gamma_mu) W psi are (u0, u1, r2, r3):
//   mu=x: h0 = psi0 + S i psi3, h1 = psi1 + S i psi2, r2 = -S i u1, r3 = -S i u0
//   mu=y: h0 = psi0 - S psi3,   h1 = psi1 + S psi2,   r2 =  S u1,   r3 = -S u0
//   mu=z: h0 = psi0 + S i psi2, h1 = psi1 - S i psi3, r2 = -S i u0, r3 =  S i u1
//   mu=t: h0 = psi0 + S psi2,   h1 = psi1 + S psi3,   r2 =  S u0,   r3 =  S u1
template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate(cx<T> (&acc)[12], const cx<T> (&q)[12],
                                           const cx<T> (&W)[9])
{
    const T s = (T)S;
    cx<T> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<T> p0 = q[c], p1 = q[3 + c], p2 = q[6 + c], p3 = q[9 + c];
        if (MU == 0) {
            h0[c] = p0 + s * mul_i(p3);
            h1[c] = p1 + s * mul_i(p2);
        } else if (MU == 1) {
            h0[c] = p0 - s * p3;
            h1[c] = p1 + s * p2;
        } else if (MU == 2) {
            h0[c] = p0 + s * mul_i(p2);
            h1[c] = p1 - s * mul_i(p3);
        } else {
            h0[c] = p0 + s * p2;
            h1[c] = p1 + s * p3;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<T> u0 = W[3 * a] * h0[0];
        cmac(u0, W[3 * a + 1], h0[1]);
        cmac(u0, W[3 * a + 2], h0[2]);
        cx<T> u1 = W[3 * a] * h1[0];
        cmac(u1, W[3 * a + 1], h1[1]);
        cmac(u1, W[3 * a + 2], h1[2]);
        acc[a] = acc[a] + u0;
        acc[3 + a] = acc[3 + a] + u1;
        if (MU == 0) {
            acc[6 + a] = acc[6 + a] - s * mul_i(u1);
            acc[9 + a] = acc[9 + a] - s * mul_i(u0);
        } else if (MU == 1) {
            acc[6 + a] = acc[6 + a] + s * u1;
            acc[9 + a] = acc[9 + a] - s * u0;
        } else if (MU == 2) {
            acc[6 + a] = acc[6 + a] - s * mul_i(u0);
            acc[9 + a] = acc[9 + a] + s * mul_i(u1);
        } else {
            acc[6 + a] = acc[6 + a] + s * u0;
            acc[9 + a] = acc[9 + a] + s * u1;
        }
    }
}

// Half indices of the eight neighbours (order +x, -x, +y, -y, +z, -z, +t, -t)
// of output site i on parity p, with periodic wrap-around.
__device__ __forceinline__ void neighbours(const Geom& g, int p, int i, int (&nb)[8])
{
    const int xh = i % g.Lxh;
    int r = i / g.Lxh;
    const int y = r % g.L[1];
    r /= g.L[1];
    const int z = r % g.L[2];
    const int t = r / g.L[2];
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int row = i - xh;
    const int sy = (int)g.sy, sz = (int)g.sz, st = (int)g.st;
    nb[0] = row + ((x + 1 == g.L[0] ? 0 : x + 1) >> 1);
    nb[1] = row + ((x == 0 ? g.L[0] - 1 : x - 1) >> 1);
    nb[2] = (y == g.L[1] - 1) ? i - (g.L[1] - 1) * sy : i + sy;
    nb[3] = (y == 0) ? i + (g.L[1] - 1) * sy : i - sy;
    nb[4] = (z == g.L[2] - 1) ? i - (g.L[2] - 1) * sz : i + sz;
    nb[5] = (z == 0) ? i + (g.L[2] - 1) * sz : i - sz;
    nb[6] = (t == g.L[3] - 1) ? i - (g.L[3] - 1) * st : i + st;
    nb[7] = (t == 0) ? i + (g.L[3] - 1) * st : i - st;
}

template <int P, int D, int MU, int S>
__device__ __forceinline__ void hop_one(cx<typename Prec<P>::real> (&acc)[12], const void* in,
                                        long long Vh, int nb, const void* links, long long lVh,
                                        int li)
{
    using T = typename Prec<P>::real;
    cx<T> q[12], W[9];
    load_spinor<P>(q, in, Vh, nb);
    load_link<P>(W, links, lVh, D, li);
    accumulate<MU, S, T>(acc, q, W);
}

// acc = H_{p,1-p} in at the output site whose neighbours are nb.  The links
// are read from planes of stride lVh at index li (the global link field, or a
// tile of it staged in shared memory).  DAG flips the projector signs.
template <int P, bool DAG>
__device__ __forceinline__ void hop_site(cx<typename Prec<P>::real> (&acc)[12], const int (&nb)[8],
                                         long long Vh, const void* in, const void* links,
                                         long long lVh, int li)
{
    using T = typename Prec<P>::real;
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = {(T)0, (T)0};
    constexpr int F = DAG ? +1 : -1;  // forward projector sign
    constexpr int B = -F;             // backward projector sign
    hop_one<P, 0, 0, F>(acc, in, Vh, nb[0], links, lVh, li);
    hop_one<P, 1, 0, B>(acc, in, Vh, nb[1], links, lVh, li);
    hop_one<P, 2, 1, F>(acc, in, Vh, nb[2], links, lVh, li);
    hop_one<P, 3, 1, B>(acc, in, Vh, nb[3], links, lVh, li);
    hop_one<P, 4, 2, F>(acc, in, Vh, nb[4], links, lVh, li);
    hop_one<P, 5, 2, B>(acc, in, Vh, nb[5], links, lVh, li);
    hop_one<P, 6, 3, F>(acc, in, Vh, nb[6], links, lVh, li);
    hop_one<P, 7, 3, B>(acc, in, Vh, nb[7], links, lVh, li);
}

struct HopArgs {
    Geom g;
    const void* links[2];
    const char* in[2];
    char* out[2];
    const char* x1[2];
    const char* x2[2];
    const char* w[2];
    long long rs_in, rs_out, rs_x1, rs_x2, rs_w;
    double a, b1;
    int parity0, blocks_per_parity;
    double* dot_out;
    int dot_stride;
    const int* active;
    int active_stride;
    RedScratch red;
};

// out = x1 + b1 x2 + a acc at site i of right-hand side rhs; with DOT the
// thread's contributions to (w, out) and ||out||^2 go to part.
template <int P, bool DOT>
__device__ __forceinline__ void epilogue(cx<typename Prec<P>::real> (&acc)[12], const HopArgs& A,
                                         int pidx, int rhs, int i, double (&part)[3])
{
    using T = typename Prec<P>::real;
    const T a = (T)A.a;
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = a * acc[c];
    if (A.x1[pidx]) {
        cx<T> x[12];
        load_spinor<P>(x, A.x1[pidx] + rhs * A.rs_x1, A.g.Vh, i);
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = acc[c] + x[c];
    }
    if (A.x2[pidx]) {
        cx<T> x[12];
        const T b1 = (T)A.b1;
        load_spinor<P>(x, A.x2[pidx] + rhs * A.rs_x2, A.g.Vh, i);
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = acc[c] + b1 * x[c];
    }
    store_spinor<P>(A.out[pidx] + rhs * A.rs_out, A.g.Vh, i, acc);
    if (DOT) {
        T cr = 0, ci = 0, nn = 0;
        if (A.w[pidx]) {
            cx<T> w[12];
            load_spinor<P>(w, A.w[pidx] + rhs * A.rs_w, A.g.Vh, i);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                cr = fma(w[c].re, acc[c].re, fma(w[c].im, acc[c].im, cr));
                ci = fma(w[c].re, acc[c].im, fma(-w[c].im, acc[c].re, ci));
            }
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) nn = fma(acc[c].re, acc[c].re, fma(acc[c].im, acc[c].im, nn));
        part[0] = cr;
        part[1] = ci;
        part[2] = nn;
    }
}

// One right-hand side per grid row, one output site per thread.
template <int P, bool DAG, bool DOT>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs A)
{
    using T = typename Prec<P>::real;
    const int rhs = blockIdx.y;
    if (A.active && A.active[rhs * A.active_stride] == 0) return;  // uniform per block
    const int pidx = blockIdx.x / A.blocks_per_parity;
    const int p = A.parity0 + pidx;
    const int i = (blockIdx.x - pidx * A.blocks_per_parity) * blockDim.x + threadIdx.x;
    double part[3] = {0.0, 0.0, 0.0};
    if (i < A.g.Vh) {
        cx<T> acc[12];
        int nb[8];
        neighbours(A.g, p, i, nb);
        hop_site<P, DAG>(acc, nb, A.g.Vh, A.in[pidx] + rhs * A.rs_in, A.links[pidx], A.g.Vh, i);
        epilogue<P, DOT>(acc, A, pidx, rhs, i, part);
    }
    if (DOT) {
        __shared__ double sh[3 * 32];
        block_sum<3>(part, sh);
        double tot[3];
        if (grid_sum<3>(part, tot, A.red, rhs, gridDim.x, blockIdx.x, sh)) {
            double* o = A.dot_out + (long long)rhs * A.dot_stride;
            o[0] = tot[0];
            o[1] = tot[1];
            o[2] = tot[2];
        }
    }
}

// ---------------------------------------------------------------------------
// Many right-hand sides: a block owns kTile output sites of one parity.  It
// copies their links (all eight hops) into shared memory once, then its
// warps sweep the right-hand sides, lane = site, reading the links from
// shared memory: the links leave HBM once for all right-hand sides.
// ---------------------------------------------------------------------------

static constexpr int kTile = 32;
static constexpr int kMaxRhsLaunch = 32;

template <int P>
struct LinkPlanes;  // the link field as 16-byte planes plus narrower planes
template <>
struct LinkPlanes<WL_F64> {
    static constexpr int n16 = 72, nsmall = 0, small_bytes = 8;
};
template <>
struct LinkPlanes<WL_F32> {
    static constexpr int n16 = 32, nsmall = 8, small_bytes = 8;
};
template <>
struct LinkPlanes<WL_F16> {
    static constexpr int n16 = 16, nsmall = 8, small_bytes = 4;
};

// Copy the links of sites [base, base + n) into a kTile-stride tile.
template <int P>
__device__ __forceinline__ void stage_links(char* sm, const char* gl, long long Vh, int base, int n)
{
    using LP = LinkPlanes<P>;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int e = tid; e < LP::n16 * kTile; e += nt) {
        const int q = e / kTile, j = e - q * kTile;
        if (j < n) ((uint4*)sm)[q * kTile + j] = __ldg((const uint4*)gl + q * Vh + base + j);
    }
    if (LP::nsmall) {
        const char* gs = gl + (size_t)LP::n16 * 16 * Vh;
        char* ss = sm + LP::n16 * 16 * kTile;
        for (int e = tid; e < LP::nsmall * kTile; e += nt) {
            const int q = e / kTile, j = e - q * kTile;
            if (j >= n) continue;
            if (LP::small_bytes == 8)
                ((uint2*)ss)[q * kTile + j] = __ldg((const uint2*)gs + q * Vh + base + j);
            else
                ((unsigned*)ss)[q * kTile + j] = __ldg((const unsigned*)gs + q * Vh + base + j);
        }
    }
}

template <int P, bool DAG, bool DOT>
__global__ void __launch_bounds__(256) hop_mrhs_kernel(const HopArgs A, int nrhs)
{
    using T = typename Prec<P>::real;
    extern __shared__ __align__(16) char smem[];
    const int pidx = blockIdx.x / A.blocks_per_parity;
    const int p = A.parity0 + pidx;
    const int base = (blockIdx.x - pidx * A.blocks_per_parity) * kTile;
    const int n = (int)min((long long)kTile, A.g.Vh - base);
    stage_links<P>(smem, (const char*)A.links[pidx], A.g.Vh, base, n);
    double* bpart = (double*)(smem + Prec<P>::link_bytes * kTile);
    __syncthreads();
    const int lane = threadIdx.x, i = base + lane;
    const bool valid = lane < n;
    int nb[8];
    if (valid) neighbours(A.g, p, i, nb);
    for (int r = threadIdx.y; r < nrhs; r += blockDim.y) {
        const bool act = !A.active || A.active[r * A.active_stride] != 0;  // warp-uniform
        double part[3] = {0.0, 0.0, 0.0};
        if (act && valid) {
            cx<T> acc[12];
            hop_site<P, DAG>(acc, nb, A.g.Vh, A.in[pidx] + r * A.rs_in, smem, kTile, lane);
            epilogue<P, DOT>(acc, A, pidx, r, i, part);
        }
        if (DOT) {
            warp_sum<3>(part);
            if (lane == 0)
                for (int k = 0; k < 3; ++k) bpart[3 * r + k] = part[k];
        }
    }
    if (!DOT) return;
    // every block leaves its per-rhs partials; the last block to finish adds
    // them up in block order (one ticket for all right-hand sides)
    __syncthreads();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int e = tid; e < 3 * nrhs; e += nt) {
        const int r = e / 3, k = e - 3 * r;
        A.red.partial[((long long)r * A.red.max_blocks + blockIdx.x) * 3 + k] = bpart[e];
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (tid == 0) last = atomicAdd(&A.red.ticket[0], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int wid = tid >> 5, nw = nt >> 5;
    for (int r = wid; r < nrhs; r += nw) {
        double v[3] = {0.0, 0.0, 0.0};
        const double* pr = A.red.partial + (long long)r * A.red.max_blocks * 3;
        for (int b = lane; b < (int)gridDim.x; b += 32)
            for (int k = 0; k < 3; ++k) v[k] += __ldcg(&pr[(long long)b * 3 + k]);
        warp_sum<3>(v);
        const bool act = !A.active || A.active[r * A.active_stride] != 0;
        if (lane == 0 && act) {
            double* o = A.dot_out + (long long)r * A.dot_stride;
            o[0] = v[0];
            o[1] = v[1];
            o[2] = v[2];
        }
    }
    if (tid == 0) A.red.ticket[0] = 0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static const int kHopBlock = 128;

template <int P>
static void launch_mrhs_t(const HopLaunch& h, const HopArgs& A, int nrhs, dim3 grid, dim3 block,
                          size_t smem, cudaStream_t s)
{
    if (h.dagger) {
        if (h.dot) hop_mrhs_kernel<P, true, true><<<grid, block, smem, s>>>(A, nrhs);
        else hop_mrhs_kernel<P, true, false><<<grid, block, smem, s>>>(A, nrhs);
    } else {
        if (h.dot) hop_mrhs_kernel<P, false, true><<<grid, block, smem, s>>>(A, nrhs);
        else hop_mrhs_kernel<P, false, false><<<grid, block, smem, s>>>(A, nrhs);
    }
}

template <int P>
static void launch_hop_t(const HopLaunch& h, const HopArgs& A, dim3 grid, int block, cudaStream_t s)
{
    if (h.dagger) {
        if (h.dot) hop_kernel<P, true, true><<<grid, block, 0, s>>>(A);
        else hop_kernel<P, true, false><<<grid, block, 0, s>>>(A);
    } else {
        if (h.dot) hop_kernel<P, false, true><<<grid, block, 0, s>>>(A);
        else hop_kernel<P, false, false><<<grid, block, 0, s>>>(A);
    }
}

static int launch_hop_chunk(wl_gauge g, const HopLaunch& h, HopArgs A, int nrhs, cudaStream_t s)
{
    const bool multi = nrhs > 1;
    const int tile = multi ? kTile : kHopBlock;
    const long long bpp = (g->geo.Vh + tile - 1) / tile;
    A.blocks_per_parity = (int)bpp;
    const unsigned gx = (unsigned)(bpp * h.nparity);
    if (h.dot) WL_TRY(ensure_red(g, nrhs, (long long)gx));
    A.red = g->red;
    // algorithmic bytes: links once for all rhs; in, out and epilogue fields per rhs
    const int extra = (h.x1[0] ? 1 : 0) + (h.x2[0] ? 1 : 0) + (h.w[0] ? 1 : 0);
    const double bytes = (double)g->geo.Vh * h.nparity *
                         (link_field_bytes(h.prec, 1) +
                          (double)nrhs * (2 + extra) * spinor_field_bytes(h.prec, 1));
    int slot = -1;
    timing_begin(g, s, bytes, h.prec, &slot);
    if (!multi) {
        const dim3 grid(gx, 1);
        switch (h.prec) {
            case WL_F64: launch_hop_t<WL_F64>(h, A, grid, kHopBlock, s); break;
            case WL_F32: launch_hop_t<WL_F32>(h, A, grid, kHopBlock, s); break;
            default: launch_hop_t<WL_F16>(h, A, grid, kHopBlock, s); break;
        }
    } else {
        const int lanes = nrhs < 8 ? nrhs : 8;
        const dim3 block(kTile, lanes);
        const size_t smem = link_field_bytes(h.prec, kTile) + sizeof(double) * 3 * nrhs;
        switch (h.prec) {
            case WL_F64: launch_mrhs_t<WL_F64>(h, A, nrhs, dim3(gx), block, smem, s); break;
            case WL_F32: launch_mrhs_t<WL_F32>(h, A, nrhs, dim3(gx), block, smem, s); break;
            default: launch_mrhs_t<WL_F16>(h, A, nrhs, dim3(gx), block, smem, s); break;
        }
    }
    WL_CHECK_LAUNCH(bytes);
    timing_end(g, s, slot);
    return WL_OK;
}

int launch_hop(wl_gauge g, const HopLaunch& h, cudaStream_t s)
{
    if (!g->links[h.prec][0])
        return set_error(WL_ERR_STATE, "gauge object has no links in the requested precision");
    HopArgs A;
    A.g = g->geo;
    for (int k = 0; k < 2; ++k) {
        const int p = h.parity0 + (k < h.nparity ? k : 0);
        A.links[k] = g->links[h.prec][p];
    }
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
        WL_TRY(launch_hop_chunk(g, h, A, n, s));
    }
    return WL_OK;
}

}  // namespace wl

using namespace wl;

static int check_common(wl_gauge g, const void* out, const void* in, wl_prec prec, int nrhs)
{
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (prec < WL_F64 || prec > WL_F16) return set_error(WL_ERR_ARG, "unknown precision");
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
        h.x1[0] = in;
        h.x1[1] = (const char*)in + fb;
        h.rs_in = h.rs_out = h.rs_x1 = (long long)(2 * fb);
        h.a = -kappa;
        return launch_hop(g, h, s);
    }
    // M_ee = 1 - kappa^2 H_eo H_oe on even half fields
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
    WL_TRY(launch_hop(g, h1, s));
    HopLaunch h2 = h1;
    h2.parity0 = 0;
    h2.in[0] = g->tmp[prec];
    h2.out[0] = out;
    h2.x1[0] = in;
    h2.rs_x1 = (long long)fb;
    h2.a = -kappa * kappa;
    return launch_hop(g, h2, s);
}
