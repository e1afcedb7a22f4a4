// Gauge objects: validation, the internal link layouts, layout conversion of
// fermion fields, workspace growth and per-launch timing.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace wl {

std::atomic<long long> g_launches{0};
std::atomic<long long> g_bytes{0};

static thread_local std::string t_last_error;

int set_error(int code, const std::string& msg)
{
    t_last_error = msg;
    return code;
}

Geom make_geom(const int* dims)
{
    Geom g;
    for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
    g.Lxh = dims[0] / 2;
    g.Vh = (long long)dims[0] * dims[1] * dims[2] * dims[3] / 2;
    g.sy = g.Lxh;
    g.sz = g.sy * dims[1];
    g.st = g.sz * dims[2];
    // Round-up reciprocals (Granlund-Montgomery): with l = ceil(log2 d) and
    // m = floor(2^(31+l) / d) + 1 < 2^32, floor(n m / 2^(31+l)) = n / d
    // exactly for 0 <= n < 2^31, since m d - 2^(31+l) <= d <= 2^l.
    const int div[3] = {g.Lxh, dims[1], dims[2]};
    for (int k = 0; k < 3; ++k) fast_div_magic(div[k], &g.dm[k], &g.ds[k]);
    return g;
}

void fast_div_magic(int divisor, unsigned* m, int* shift)
{
    const unsigned long long d = (unsigned long long)divisor;
    if (d <= 1) {  // m = 0 marks "divide by one"
        *m = 0;
        *shift = 0;
        return;
    }
    int l = 0;
    while ((1ull << l) < d) ++l;
    *m = (unsigned)((1ull << (31 + l)) / d + 1);
    *shift = l - 1;
}

bool is_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// ---------------------------------------------------------------------------
// links: W_d(x) for the 8 hops of each output site, phases folded in,
// backward links daggered.
// ---------------------------------------------------------------------------

template <int P>
__device__ __forceinline__ void store_link(void* base, long long Vh, int d, long long i,
                                           const cx<double> (&w)[9]);

template <>
__device__ __forceinline__ void store_link<WL_F64>(void* base, long long Vh, int d, long long i,
                                                   const cx<double> (&w)[9])
{
    double2* p = (double2*)base + (long long)d * 9 * Vh;
    for (int k = 0; k < 9; ++k) p[k * Vh + i] = make_double2(w[k].re, w[k].im);
}
template <>
__device__ __forceinline__ void store_link<WL_F32>(void* base, long long Vh, int d, long long i,
                                                   const cx<double> (&w)[9])
{
    float4* p = (float4*)base + (long long)d * 4 * Vh;
    for (int k = 0; k < 4; ++k)
        p[k * Vh + i] = make_float4((float)w[2 * k].re, (float)w[2 * k].im, (float)w[2 * k + 1].re,
                                    (float)w[2 * k + 1].im);
    float2* q = (float2*)((float4*)base + 8 * 4 * Vh) + (long long)d * Vh;
    q[i] = make_float2((float)w[8].re, (float)w[8].im);
}
template <>
__device__ __forceinline__ void store_link<WL_DF64>(void* base, long long Vh, int d, long long i,
                                                    const cx<double> (&w)[9])
{
    float4* p = (float4*)base + (long long)d * 9 * Vh;
    for (int k = 0; k < 9; ++k) {
        const df64 re(w[k].re), im(w[k].im);
        p[k * Vh + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}
template <>
__device__ __forceinline__ void store_link<WL_F16>(void* base, long long Vh, int d, long long i,
                                                   const cx<double> (&w)[9])
{
    // |entries| <= 1 for unitary links, so FP16 needs no scale
    uint4* p = (uint4*)base + (long long)d * 2 * Vh;
    for (int k = 0; k < 2; ++k) {
        uint4 t;
        t.x = f2h((float)w[4 * k].re, (float)w[4 * k].im);
        t.y = f2h((float)w[4 * k + 1].re, (float)w[4 * k + 1].im);
        t.z = f2h((float)w[4 * k + 2].re, (float)w[4 * k + 2].im);
        t.w = f2h((float)w[4 * k + 3].re, (float)w[4 * k + 3].im);
        p[k * Vh + i] = t;
    }
    unsigned* q = (unsigned*)((uint4*)base + 8 * 2 * Vh) + (long long)d * Vh;
    q[i] = f2h((float)w[8].re, (float)w[8].im);
}

struct BC {
    double re[4], im[4];
};

// Where a gauge object's sites sit in the lattice its links come from: the
// whole lattice (origin 0, gl = the object's own geometry), or one block of a
// domain decomposition (gl = the global lattice, origin = the block's first
// site).  Links are read from the global field at global coordinates, so the
// hop matrices of a block's face sites are those of the undivided lattice:
// neighbours across a cut face and boundary phases come from the global
// geometry.
struct Place {
    Geom gl;
    int o[4];
};

// Global site index of half site i (parity p of the local lattice) and its
// global coordinates.
__device__ __forceinline__ long long global_site(const Geom& g, const Place& pl, int p, long long i,
                                                 int (&c)[4])
{
    long long r = site_of_half(g, p, i);
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(r % g.L[mu]) + pl.o[mu];
        r /= g.L[mu];
    }
    return c[0] + (long long)pl.gl.L[0] * (c[1] + (long long)pl.gl.L[1] * (c[2] + (long long)pl.gl.L[2] * c[3]));
}

template <int P>
__global__ void build_links_kernel(void* out, const double* __restrict__ U, Geom g, Place pl, BC bc, int p)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    int c[4];
    const long long s = global_site(g, pl, p, i, c);
    const Geom& G = pl.gl;
    const long long stride[4] = {1, G.L[0], (long long)G.L[0] * G.L[1],
                                 (long long)G.L[0] * G.L[1] * G.L[2]};
    for (int mu = 0; mu < 4; ++mu) {
        cx<double> w[9];
        // forward: phi^[x_mu = L-1] U_mu(x)
        const double* u = U + (s * 4 + mu) * 18;
        double pr = 1.0, pi = 0.0;
        if (c[mu] == G.L[mu] - 1) { pr = bc.re[mu]; pi = bc.im[mu]; }
        for (int k = 0; k < 9; ++k) {
            const double a = u[2 * k], b = u[2 * k + 1];
            w[k] = {pr * a - pi * b, pr * b + pi * a};
        }
        store_link<P>(out, g.Vh, 2 * mu, i, w);
        // backward: conj(phi)^[x_mu = 0] U_mu(x - mu)^dag
        const long long n = (c[mu] == 0) ? s + (G.L[mu] - 1) * stride[mu] : s - stride[mu];
        const double* v = U + (n * 4 + mu) * 18;
        pr = 1.0;
        pi = 0.0;
        if (c[mu] == 0) { pr = bc.re[mu]; pi = -bc.im[mu]; }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double re = v[2 * (b * 3 + a)], im = -v[2 * (b * 3 + a) + 1];
                w[a * 3 + b] = {pr * re - pi * im, pr * im + pi * re};
            }
        store_link<P>(out, g.Vh, 2 * mu + 1, i, w);
    }
}

// Compressed links (LF = 1 of the hopping kernels): rows 0 and 1 of the
// hop matrices U_mu(x) and U_mu(x - mu)^dag without the boundary phase; the
// kernels rebuild row 2 from unitarity.  Set-up checks that every link is in
// SU(3) to 1e-6 (max |U U^dag - 1| and |det U - 1|) and raises *flag if not.
template <int P>
__device__ __forceinline__ void store_link_r12(void* base, long long Vh, int d, long long i,
                                               const cx<double> (&w)[9]);
template <>
__device__ __forceinline__ void store_link_r12<WL_F32>(void* base, long long Vh, int d, long long i,
                                                       const cx<double> (&w)[9])
{
    float4* p = (float4*)base + (long long)d * 3 * Vh;
    for (int k = 0; k < 3; ++k)
        p[k * Vh + i] = make_float4((float)w[2 * k].re, (float)w[2 * k].im, (float)w[2 * k + 1].re,
                                    (float)w[2 * k + 1].im);
}
template <>
__device__ __forceinline__ void store_link_r12<WL_F16>(void* base, long long Vh, int d, long long i,
                                                       const cx<double> (&w)[9])
{
    uint4 t;
    t.x = f2h((float)w[0].re, (float)w[0].im);
    t.y = f2h((float)w[1].re, (float)w[1].im);
    t.z = f2h((float)w[2].re, (float)w[2].im);
    t.w = f2h((float)w[3].re, (float)w[3].im);
    ((uint4*)base)[(long long)d * Vh + i] = t;
    uint2 u;
    u.x = f2h((float)w[4].re, (float)w[4].im);
    u.y = f2h((float)w[5].re, (float)w[5].im);
    ((uint2*)((uint4*)base + 8 * Vh))[(long long)d * Vh + i] = u;
}

// max |U U^dag - 1| and |det U - 1| of a 3x3 complex matrix
__device__ double su3_deviation(const double* u)
{
    auto at = [&](int a, int b) { return cx<double>{u[2 * (3 * a + b)], u[2 * (3 * a + b) + 1]}; };
    double dev = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cx<double> sum = {a == b ? -1.0 : 0.0, 0.0};
            for (int k = 0; k < 3; ++k) sum = sum + at(a, k) * conj(at(b, k));
            dev = fmax(dev, hypot(sum.re, sum.im));
        }
    const cx<double> det = at(0, 0) * (at(1, 1) * at(2, 2) - at(1, 2) * at(2, 1)) -
                           at(0, 1) * (at(1, 0) * at(2, 2) - at(1, 2) * at(2, 0)) +
                           at(0, 2) * (at(1, 0) * at(2, 1) - at(1, 1) * at(2, 0));
    return fmax(dev, hypot(det.re - 1.0, det.im));
}

// The eight reals of an SU(3) matrix w that load_link_r8 (hop.cuh) decodes:
// rows taken in the cyclic order that puts the smaller of |w_00|, |w_10| first
// (shifted: (W1, W2, W0)), then a2, a3, b1, tan(arg(a1) / 4) (+ 3 when shifted)
// and tan(arg(c1) / 4), computed in FP64 and rounded to FP32.
__device__ void store_link_r8(void* base, long long Vh, int d, long long i, const cx<double> (&w)[9])
{
    auto mag2 = [](cx<double> z) { return z.re * z.re + z.im * z.im; };
    const bool shift = mag2(w[0]) > mag2(w[3]);
    const cx<double>* a = shift ? w + 3 : w;
    const cx<double>* b = shift ? w + 6 : w + 3;
    const cx<double>* c = shift ? w : w + 6;
    const double ta = tan(0.25 * atan2(a[0].im, a[0].re)), tc = tan(0.25 * atan2(c[0].im, c[0].re));
    float4* p = (float4*)base + (long long)d * 2 * Vh;
    p[i] = make_float4((float)a[1].re, (float)a[1].im, (float)a[2].re, (float)a[2].im);
    p[Vh + i] = make_float4((float)b[0].re, (float)b[0].im, (float)(ta + (shift ? 3.0 : 0.0)), (float)tc);
}

template <int P>
__global__ void build_links_r12_kernel(void* out, const double* __restrict__ U, Geom g, Place pl, int p,
                                       int* flag)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    int c[4];
    const long long s = global_site(g, pl, p, i, c);
    const Geom& G = pl.gl;
    const long long stride[4] = {1, G.L[0], (long long)G.L[0] * G.L[1],
                                 (long long)G.L[0] * G.L[1] * G.L[2]};
    for (int mu = 0; mu < 4; ++mu) {
        cx<double> w[9];
        const double* u = U + (s * 4 + mu) * 18;
        if (su3_deviation(u) > 1e-6) atomicOr(flag, 1);
        for (int k = 0; k < 9; ++k) w[k] = {u[2 * k], u[2 * k + 1]};
        store_link_r12<P>(out, g.Vh, 2 * mu, i, w);
        const long long n = (c[mu] == 0) ? s + (G.L[mu] - 1) * stride[mu] : s - stride[mu];
        const double* v = U + (n * 4 + mu) * 18;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) w[a * 3 + b] = {v[2 * (b * 3 + a)], -v[2 * (b * 3 + a) + 1]};
        store_link_r12<P>(out, g.Vh, 2 * mu + 1, i, w);
    }
}

// Eight-real FP32 links of parity p (hop d = 2 mu: U_mu(x); 2 mu + 1: the
// daggered backward link), no boundary phase; flag set on a non-SU(3) link.
__global__ void build_links_r8_kernel(void* out, const double* __restrict__ U, Geom g, Place pl, int p, int* flag)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.Vh) return;
    int c[4];
    const long long s = global_site(g, pl, p, i, c);
    const Geom& G = pl.gl;
    const long long stride[4] = {1, G.L[0], (long long)G.L[0] * G.L[1],
                                 (long long)G.L[0] * G.L[1] * G.L[2]};
    for (int mu = 0; mu < 4; ++mu) {
        cx<double> w[9];
        const double* u = U + (s * 4 + mu) * 18;
        if (su3_deviation(u) > 1e-6) atomicOr(flag, 1);
        for (int k = 0; k < 9; ++k) w[k] = {u[2 * k], u[2 * k + 1]};
        store_link_r8(out, g.Vh, 2 * mu, i, w);
        const long long n = (c[mu] == 0) ? s + (G.L[mu] - 1) * stride[mu] : s - stride[mu];
        const double* v = U + (n * 4 + mu) * 18;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) w[a * 3 + b] = {v[2 * (b * 3 + a)], -v[2 * (b * 3 + a) + 1]};
        store_link_r8(out, g.Vh, 2 * mu + 1, i, w);
    }
}

// ---------------------------------------------------------------------------
// fermion layout conversion
// ---------------------------------------------------------------------------

template <int P>
__global__ void to_internal_kernel(char* out, const double* __restrict__ in, Geom g, int p,
                                   size_t fb, long long V)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.Vh) return;
    const long long s = site_of_half(g, p, i);
    const double* q = in + ((long long)rhs * V + s) * 24;
    cx<typename Prec<P>::real> v[12];
    for (int c = 0; c < 12; ++c)
        v[c] = {(typename Prec<P>::real)q[2 * c], (typename Prec<P>::real)q[2 * c + 1]};
    store_spinor<P>(out + rhs * fb, g.Vh, i, v);
}

template <int P>
__global__ void to_canonical_kernel(double* out, const char* in, Geom g, int p, size_t fb,
                                    long long V)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.Vh) return;
    const long long s = site_of_half(g, p, i);
    double* q = out + ((long long)rhs * V + s) * 24;
    cx<typename Prec<P>::real> v[12];
    load_spinor<P>(v, in + rhs * fb, g.Vh, i);
    for (int c = 0; c < 12; ++c) {
        q[2 * c] = (double)v[c].re;
        q[2 * c + 1] = (double)v[c].im;
    }
}

// ---------------------------------------------------------------------------
// workspace growth
// ---------------------------------------------------------------------------

int ensure_red(wl_gauge g, int slots, long long blocks)
{
    if (slots <= g->red_slots && blocks <= g->red.max_blocks) return WL_OK;
    const int ns = slots > g->red_slots ? slots : g->red_slots;
    const long long nb = blocks > g->red.max_blocks ? blocks : g->red.max_blocks;
    WL_CUDA(cudaDeviceSynchronize());
    if (g->red.partial) cudaFree(g->red.partial);
    if (g->red.ticket) cudaFree(g->red.ticket);
    g->red.partial = nullptr;
    g->red.ticket = nullptr;
    WL_CUDA(cudaMalloc(&g->red.partial, sizeof(double) * 4 * (size_t)ns * (size_t)nb));
    WL_CUDA(cudaMalloc(&g->red.ticket, sizeof(unsigned) * (size_t)ns));
    WL_CUDA(cudaMemset(g->red.ticket, 0, sizeof(unsigned) * (size_t)ns));
    g->red.max_blocks = (int)nb;
    g->red_slots = ns;
    g->red_gen++;
    return WL_OK;
}

int ensure_tmp(wl_gauge g, int prec, size_t bytes)
{
    if (g->tmp_bytes[prec] >= bytes) return WL_OK;
    WL_CUDA(cudaDeviceSynchronize());
    if (g->tmp[prec]) cudaFree(g->tmp[prec]);
    g->tmp[prec] = nullptr;
    WL_CUDA(cudaMalloc(&g->tmp[prec], bytes));
    g->tmp_bytes[prec] = bytes;
    return WL_OK;
}

// ---------------------------------------------------------------------------
// timing
// ---------------------------------------------------------------------------

static const size_t kTimingPool = 1 << 14;
static const size_t kCapturePool = 256;  // timed launches in one solver graph

void timing_begin(wl_gauge g, cudaStream_t s, double bytes, int prec, int* slot)
{
    *slot = -1;
    Timing& t = g->timing;
    if (!t.on) return;
    if (is_capturing(s)) {  // a capture slot (slot = -2 - index), or dropped outside solver graphs
        if (!t.capturing || t.cused >= t.cstart.size()) {
            t.dropped++;
            return;
        }
        const size_t c = t.cused++;
        t.cbytes[c] = bytes;
        t.cprec[c] = prec;
        *slot = -2 - (int)c;
        // an event-record node of the graph (a plain record would only mark a
        // dependency inside the capture)
        cudaEventRecordWithFlags(t.cstart[c], s, cudaEventRecordExternal);
        return;
    }
    if (t.used >= t.start.size()) {
        t.dropped++;
        return;
    }
    *slot = (int)t.used++;
    t.bytes[*slot] = bytes;
    t.prec[*slot] = prec;
    t.fixed[*slot] = -1.f;
    cudaEventRecord(t.start[*slot], s);
}

void timing_end(wl_gauge g, cudaStream_t s, int slot)
{
    if (slot >= 0) cudaEventRecord(g->timing.stop[slot], s);
    else if (slot <= -2) cudaEventRecordWithFlags(g->timing.cstop[-2 - slot], s, cudaEventRecordExternal);
}

void timing_capture_begin(wl_gauge g)
{
    Timing& t = g->timing;
    timing_harvest(g);  // the capture slots are about to be recorded by another graph
    t.cused = 0;
    t.capturing = t.on;
}

size_t timing_capture_end(wl_gauge g)
{
    Timing& t = g->timing;
    const size_t n = t.capturing ? t.cused : 0;
    t.capturing = false;
    return n;
}

void timing_replayed(wl_gauge g, size_t nslots)
{
    Timing& t = g->timing;
    if (!t.on) return;
    for (size_t c = 0; c < nslots; ++c) {
        if (t.used >= t.start.size()) {
            t.dropped++;
            continue;
        }
        const size_t q = t.used++;
        t.bytes[q] = t.cbytes[c];
        t.prec[q] = t.cprec[c];
        t.fixed[q] = -1.f;
        t.pending.push_back({q, c});
    }
}

int timing_harvest(wl_gauge g)
{
    Timing& t = g->timing;
    for (const auto& pc : t.pending) {
        float e = 0.f;
        if (cudaEventSynchronize(t.cstop[pc.second]) != cudaSuccess ||
            cudaEventElapsedTime(&e, t.cstart[pc.second], t.cstop[pc.second]) != cudaSuccess) {
            cudaGetLastError();  // timing is a diagnostic: leave the record out, not the solve
            t.bytes[pc.first] = -1.0;
            t.dropped++;
            continue;
        }
        t.fixed[pc.first] = e;
    }
    t.pending.clear();
    return WL_OK;
}

}  // namespace wl

using namespace wl;

namespace wl {

// Create a gauge object for the local lattice `local` whose links are read
// from the canonical field U of the lattice `global` (equal to `local` for an
// undivided lattice) at the block starting at `origin`.
int gauge_create(wl_gauge* out, const wl_lattice* local, const wl_lattice* global, const int* origin,
                 const double* U, int prec_mask, cudaStream_t s)
{
    *out = nullptr;
    if (!U) return set_error(WL_ERR_ARG, "NULL gauge field");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, U) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return set_error(WL_ERR_ARG, "gauge field must be device memory");
    }
    auto g = new wl_gauge_s();
    g->geo = make_geom(local->dims);
    g->kappa = local->kappa;
    for (int k = 0; k < 4; ++k) {
        g->bc_re[k] = local->bc_re[k];
        g->bc_im[k] = local->bc_im[k];
    }
    Place pl;
    pl.gl = make_geom(global->dims);
    for (int k = 0; k < 4; ++k) pl.o[k] = origin ? origin[k] : 0;
    g->prec_mask = (prec_mask & WL_PREC_ALL) | WL_PREC_MASK(WL_F64);
    // the outer residual corrections of mixed-precision solves run in df64
    if (g->prec_mask & (WL_PREC_MASK(WL_F32) | WL_PREC_MASK(WL_F16)))
        g->prec_mask |= WL_PREC_MASK(WL_DF64);
    int rc = WL_OK;
    do {
        if (cudaGetDevice(&g->device) != cudaSuccess) { rc = set_error(WL_ERR_CUDA, "cudaGetDevice"); break; }
        cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
        BC bc;
        for (int k = 0; k < 4; ++k) {
            bc.re[k] = global->bc_re[k];
            bc.im[k] = global->bc_im[k];
        }
        const int block = 128;
        const unsigned grid = (unsigned)((g->geo.Vh + block - 1) / block);
        for (int prec = 0; prec < 4 && rc == WL_OK; ++prec) {
            if (!(g->prec_mask & WL_PREC_MASK(prec))) continue;
            for (int p = 0; p < 2; ++p) {
                cudaError_t e = cudaMalloc(&g->links[prec][p], link_field_bytes(prec, g->geo.Vh));
                if (e != cudaSuccess) {
                    rc = set_error(WL_ERR_CUDA, std::string("cudaMalloc links: ") + cudaGetErrorString(e));
                    break;
                }
                if (prec == WL_F64) build_links_kernel<WL_F64><<<grid, block, 0, s>>>(g->links[prec][p], U, g->geo, pl, bc, p);
                else if (prec == WL_F32) build_links_kernel<WL_F32><<<grid, block, 0, s>>>(g->links[prec][p], U, g->geo, pl, bc, p);
                else if (prec == WL_F16) build_links_kernel<WL_F16><<<grid, block, 0, s>>>(g->links[prec][p], U, g->geo, pl, bc, p);
                else build_links_kernel<WL_DF64><<<grid, block, 0, s>>>(g->links[prec][p], U, g->geo, pl, bc, p);
                e = cudaGetLastError();
                if (e != cudaSuccess) {
                    rc = set_error(WL_ERR_CUDA, std::string("link build launch: ") + cudaGetErrorString(e));
                    break;
                }
                count_launch(1, (double)g->geo.Vh * (8 * 144.0 + link_field_bytes(prec, 1)));
            }
        }
        if (rc != WL_OK) break;
        if (prec_mask & WL_LINKS_R12) {  // compressed FP32 / FP16 copies
            int* flag = nullptr;
            if (cudaMalloc((void**)&flag, sizeof(int)) != cudaSuccess ||
                cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) {
                cudaGetLastError();
                if (flag) cudaFree(flag);
                rc = set_error(WL_ERR_CUDA, "cudaMalloc for the SU(3) check");
                break;
            }
            for (int prec : {(int)WL_F32, (int)WL_F16}) {
                if (!(g->prec_mask & WL_PREC_MASK(prec)) || rc != WL_OK) continue;
                for (int p = 0; p < 2 && rc == WL_OK; ++p) {
                    const size_t bytes = (prec == WL_F32 ? 384 : 192) * (size_t)g->geo.Vh;
                    if (cudaMalloc(&g->links_r12[prec][p], bytes) != cudaSuccess) {
                        cudaGetLastError();
                        rc = set_error(WL_ERR_CUDA, "cudaMalloc compressed links");
                        break;
                    }
                    if (prec == WL_F32) build_links_r12_kernel<WL_F32><<<grid, block, 0, s>>>(g->links_r12[prec][p], U, g->geo, pl, p, flag);
                    else build_links_r12_kernel<WL_F16><<<grid, block, 0, s>>>(g->links_r12[prec][p], U, g->geo, pl, p, flag);
                    if (cudaGetLastError() != cudaSuccess) rc = set_error(WL_ERR_CUDA, "compressed link build launch");
                    count_launch(1, (double)g->geo.Vh * (8 * 144.0 + bytes / g->geo.Vh));
                }
            }
            int hflag = 0;
            if (rc == WL_OK && (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                                cudaStreamSynchronize(s) != cudaSuccess))
                rc = set_error(WL_ERR_CUDA, "compressed link build failed");
            cudaFree(flag);
            if (rc == WL_OK && hflag)
                rc = set_error(WL_ERR_ARG, "WL_LINKS_R12 needs SU(3) links (unitary, det 1, to 1e-6)");
            if (rc != WL_OK) break;
        }
        if ((prec_mask & WL_LINKS_R8) && (g->prec_mask & WL_PREC_MASK(WL_F32))) {  // eight-real FP32 copies
            int* flag = nullptr;
            if (cudaMalloc((void**)&flag, sizeof(int)) != cudaSuccess ||
                cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) {
                cudaGetLastError();
                if (flag) cudaFree(flag);
                rc = set_error(WL_ERR_CUDA, "cudaMalloc for the SU(3) check");
                break;
            }
            for (int p = 0; p < 2 && rc == WL_OK; ++p) {
                const size_t bytes = 256 * (size_t)g->geo.Vh;
                if (cudaMalloc(&g->links_r8[WL_F32][p], bytes) != cudaSuccess) {
                    cudaGetLastError();
                    rc = set_error(WL_ERR_CUDA, "cudaMalloc eight-real links");
                    break;
                }
                build_links_r8_kernel<<<grid, block, 0, s>>>(g->links_r8[WL_F32][p], U, g->geo, pl, p, flag);
                if (cudaGetLastError() != cudaSuccess) rc = set_error(WL_ERR_CUDA, "eight-real link build launch");
                count_launch(1, (double)g->geo.Vh * (8 * 144.0 + 256.0));
            }
            int hflag = 0;
            if (rc == WL_OK && (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                                cudaStreamSynchronize(s) != cudaSuccess))
                rc = set_error(WL_ERR_CUDA, "eight-real link build failed");
            cudaFree(flag);
            if (rc == WL_OK && hflag)
                rc = set_error(WL_ERR_ARG, "WL_LINKS_R8 needs SU(3) links (unitary, det 1, to 1e-6)");
            if (rc != WL_OK) break;
        }
        // the link build reads U: finish before returning so U may be freed
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = set_error(WL_ERR_CUDA, "link build failed"); break; }
    } while (0);
    if (rc != WL_OK) {
        wl_gauge_destroy(g);
        return rc;
    }
    *out = g;
    return WL_OK;
}

int validate_lattice(const wl_lattice* lat)
{
    if (!lat) return set_error(WL_ERR_ARG, "NULL lattice");
    long long V = 1;
    for (int k = 0; k < 4; ++k) {
        if (lat->dims[k] < 2 || lat->dims[k] % 2)
            return set_error(WL_ERR_ARG, "lattice extents must be even and >= 2");
        V *= lat->dims[k];
    }
    if (V / 2 > 0x7fffffffLL / 16)
        return set_error(WL_ERR_ARG, "lattice too large for 32-bit half-index arithmetic");
    for (int k = 0; k < 4; ++k) {
        const double m = std::hypot(lat->bc_re[k], lat->bc_im[k]);
        if (std::fabs(m - 1.0) > 1e-12) return set_error(WL_ERR_ARG, "boundary phases must have |phi| = 1");
    }
    if (!std::isfinite(lat->kappa)) return set_error(WL_ERR_ARG, "kappa must be finite");
    return WL_OK;
}

}  // namespace wl

extern "C" int wl_gauge_create(wl_gauge* out, const wl_lattice* lat, const double* U, int prec_mask,
                               void* stream)
{
    WL_ENTRY();
    if (!out) return set_error(WL_ERR_ARG, "NULL output handle");
    *out = nullptr;
    WL_TRY(validate_lattice(lat));
    return gauge_create(out, lat, lat, nullptr, U, prec_mask, (cudaStream_t)stream);
}

void free_workspace(wl_gauge g);  // solver.cu
void batch_forget(wl_gauge g);    // batch.cu

extern "C" int wl_gauge_destroy(wl_gauge g)
{
    if (!g) return WL_OK;
    cudaDeviceSynchronize();
    batch_forget(g);
    free_workspace(g);
    free_clover(g);
    for (int prec = 0; prec < 4; ++prec) {
        for (int p = 0; p < 2; ++p) {
            if (g->links[prec][p]) cudaFree(g->links[prec][p]);
            if (g->links_r12[prec][p]) cudaFree(g->links_r12[prec][p]);
            if (g->links_r8[prec][p]) cudaFree(g->links_r8[prec][p]);
        }
        if (g->tmp[prec]) cudaFree(g->tmp[prec]);
    }
    if (g->red.partial) cudaFree(g->red.partial);
    if (g->red.ticket) cudaFree(g->red.ticket);
    for (auto e : g->timing.start) cudaEventDestroy(e);
    for (auto e : g->timing.stop) cudaEventDestroy(e);
    for (auto e : g->timing.cstart) cudaEventDestroy(e);
    for (auto e : g->timing.cstop) cudaEventDestroy(e);
    delete g;
    return WL_OK;
}

extern "C" long long wl_half_volume(wl_gauge g) { return g ? g->geo.Vh : 0; }

extern "C" size_t wl_field_bytes(wl_gauge g, wl_prec prec, int nrhs)
{
    if (!g || prec < WL_F64 || prec > WL_DF64 || nrhs < 0) return 0;
    return spinor_field_bytes(prec, g->geo.Vh) * (size_t)nrhs;
}

static int conv_check(wl_gauge g, const void* a, const void* b, int parity, wl_prec prec, int nrhs)
{
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    if (!a || !b) return set_error(WL_ERR_ARG, "NULL field pointer");
    if (parity != 0 && parity != 1) return set_error(WL_ERR_ARG, "parity must be 0 or 1");
    if (prec < WL_F64 || prec > WL_DF64) return set_error(WL_ERR_ARG, "unknown precision");
    if (nrhs < 1 || nrhs > 65535) return set_error(WL_ERR_ARG, "nrhs must be in 1..65535");
    return WL_OK;
}

namespace wl {

int field_to_internal(wl_gauge g, void* out, const double* in, int parity, int prec, int nrhs,
                      cudaStream_t s, long long out_rs)
{
    const int block = 128;
    dim3 grid((unsigned)((g->geo.Vh + block - 1) / block), (unsigned)nrhs);
    const size_t fb = out_rs > 0 ? (size_t)out_rs : spinor_field_bytes(prec, g->geo.Vh);
    const long long V = 2 * g->geo.Vh;
    switch (prec) {
        case WL_F64: to_internal_kernel<WL_F64><<<grid, block, 0, s>>>((char*)out, in, g->geo, parity, fb, V); break;
        case WL_F32: to_internal_kernel<WL_F32><<<grid, block, 0, s>>>((char*)out, in, g->geo, parity, fb, V); break;
        case WL_F16: to_internal_kernel<WL_F16><<<grid, block, 0, s>>>((char*)out, in, g->geo, parity, fb, V); break;
        default: to_internal_kernel<WL_DF64><<<grid, block, 0, s>>>((char*)out, in, g->geo, parity, fb, V); break;
    }
    WL_CHECK_LAUNCH((double)nrhs * g->geo.Vh * (192.0 + (double)spinor_field_bytes(prec, 1)));
    return WL_OK;
}

int field_to_canonical(wl_gauge g, double* out, const void* in, int parity, int prec, int nrhs,
                       cudaStream_t s, long long in_rs)
{
    const int block = 128;
    dim3 grid((unsigned)((g->geo.Vh + block - 1) / block), (unsigned)nrhs);
    const size_t fb = in_rs > 0 ? (size_t)in_rs : spinor_field_bytes(prec, g->geo.Vh);
    const long long V = 2 * g->geo.Vh;
    switch (prec) {
        case WL_F64: to_canonical_kernel<WL_F64><<<grid, block, 0, s>>>(out, (const char*)in, g->geo, parity, fb, V); break;
        case WL_F32: to_canonical_kernel<WL_F32><<<grid, block, 0, s>>>(out, (const char*)in, g->geo, parity, fb, V); break;
        case WL_F16: to_canonical_kernel<WL_F16><<<grid, block, 0, s>>>(out, (const char*)in, g->geo, parity, fb, V); break;
        default: to_canonical_kernel<WL_DF64><<<grid, block, 0, s>>>(out, (const char*)in, g->geo, parity, fb, V); break;
    }
    WL_CHECK_LAUNCH((double)nrhs * g->geo.Vh * (192.0 + (double)spinor_field_bytes(prec, 1)));
    return WL_OK;
}

}  // namespace wl

extern "C" int wl_field_to_internal(wl_gauge g, void* out, const double* in, int parity, wl_prec prec,
                                    int nrhs, void* stream)
{
    WL_ENTRY();
    WL_TRY(conv_check(g, out, in, parity, prec, nrhs));
    return field_to_internal(g, out, in, parity, prec, nrhs, (cudaStream_t)stream);
}

extern "C" int wl_field_to_canonical(wl_gauge g, double* out, const void* in, int parity, wl_prec prec,
                                     int nrhs, void* stream)
{
    WL_ENTRY();
    WL_TRY(conv_check(g, out, in, parity, prec, nrhs));
    return field_to_canonical(g, out, in, parity, prec, nrhs, (cudaStream_t)stream);
}

extern "C" const char* wl_last_error(void) { return wl::t_last_error.c_str(); }

extern "C" int wl_spinor16_format(void) { return WL_SPINOR16_FIXED ? 1 : 0; }

extern "C" long long wl_launch_count(void) { return wl::g_launches.load(); }

extern "C" double wl_algorithmic_bytes(void) { return (double)wl::g_bytes.load(); }

extern "C" int wl_timing(wl_gauge g, int enable)
{
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    Timing& t = g->timing;
    if (enable) {
        if (t.start.empty()) {
            t.start.resize(kTimingPool);
            t.stop.resize(kTimingPool);
            t.bytes.resize(kTimingPool);
            t.prec.resize(kTimingPool);
            t.fixed.resize(kTimingPool);
            for (size_t k = 0; k < kTimingPool; ++k) {
                WL_CUDA(cudaEventCreate(&t.start[k]));
                WL_CUDA(cudaEventCreate(&t.stop[k]));
            }
            t.cstart.resize(kCapturePool);
            t.cstop.resize(kCapturePool);
            t.cbytes.resize(kCapturePool);
            t.cprec.resize(kCapturePool);
            for (size_t k = 0; k < kCapturePool; ++k) {
                WL_CUDA(cudaEventCreate(&t.cstart[k]));
                WL_CUDA(cudaEventCreate(&t.cstop[k]));
            }
        }
        t.pending.clear();
        t.used = 0;
        t.dropped = 0;
    }
    t.on = enable != 0;
    return WL_OK;
}

extern "C" int wl_timing_read(wl_gauge g, int prec, double* ms, long long* launches, double* bytes)
{
    if (!g) return set_error(WL_ERR_ARG, "NULL gauge object");
    Timing& t = g->timing;
    WL_TRY(timing_harvest(g));
    double total = 0.0, b = 0.0;
    long long n = 0;
    for (size_t k = 0; k < t.used; ++k) {
        if (prec >= 0 && t.prec[k] != prec) continue;
        if (t.bytes[k] < 0.0) continue;  // a launch that found no work (solver chunk tail)
        ++n;
        float e = t.fixed[k];
        if (e < 0.f) {
            WL_CUDA(cudaEventSynchronize(t.stop[k]));
            WL_CUDA(cudaEventElapsedTime(&e, t.start[k], t.stop[k]));
        }
        total += e;
        b += t.bytes[k];
    }
    if (ms) *ms = total;
    if (launches) *launches = n;
    if (bytes) *bytes = b;
    return WL_OK;
}
