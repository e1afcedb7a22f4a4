// Host-side internals shared by the library's translation units: the gauge
// object, lattice geometry, kernel-launch helpers and solver workspace.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"

namespace wl {

// Lattice geometry in half-lattice (checkerboard) index units.
struct Geom {
    int L[4];      // Lx, Ly, Lz, Lt
    int Lxh;       // Lx / 2
    long long Vh;  // half volume
    long long sy, sz, st;  // half-index strides of y, z, t
    // division by Lxh, Ly, Lz by multiply-high and shift (set by make_geom):
    // n / d = umulhi(n, dm) >> ds for 0 <= n < 2^31 (dm = 0: d = 1)
    unsigned dm[3];
    int ds[3];
};

// Per-launch event timing of hopping kernels (see wl_timing).
struct Timing {
    bool on = false;
    std::vector<cudaEvent_t> start, stop;
    std::vector<double> bytes;
    std::vector<int> prec;
    std::vector<float> fixed;  // ms of a slot read from a graph replay; < 0: read the slot's events
    size_t used = 0;
    long long dropped = 0;
    // Launches inside a captured solver graph ("capture slots"): their event
    // records are graph nodes, recorded again by every replay.
    std::vector<cudaEvent_t> cstart, cstop;
    std::vector<double> cbytes;
    std::vector<int> cprec;
    size_t cused = 0;
    bool capturing = false;
    std::vector<std::pair<size_t, size_t>> pending;  // (slot, capture slot) of the last replay
};

struct Workspace;  // solver.cu

// Tuned launch shape of one kernel configuration (autotuner cache entry).
struct Tuned {
    int block = 0;     // threads per block
    int rhs_tile = 1;  // right-hand sides per thread block (multi-RHS hop)
};

}  // namespace wl

struct wl_gauge_s {
    wl::Geom geo;
    double kappa;
    double bc_re[4], bc_im[4];
    int prec_mask;
    int device;
    int num_sms;
    // [prec][out parity]; prec 3 is the internal df64 copy used by the outer corrections
    void* links[4][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    // compressed (two-row) copies of the FP32 / FP16 links, when requested (WL_LINKS_R12)
    void* links_r12[4][2] = {};
    void* links_r8[4][2] = {};  // eight-real links (FP32 only), see hop.cuh load_link_r8
    // grid-reduction scratch
    wl::RedScratch red = {nullptr, nullptr, 0};
    int red_slots = 0;
    int red_gen = 0;  // bumped whenever the scratch moves (captured graphs hold its address)
    // odd-parity temporaries for wilson_mult (eo = 1), per precision
    void* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t tmp_bytes[4] = {0, 0, 0, 0};
    wl::Timing timing;
    wl::Workspace* ws = nullptr;  // solver workspace, owned (solver.cu)
    // clover term (clover.cu): [prec][parity][0: A = 1 + F, 1: A^-1]
    void* clov[4][2][2] = {};
    bool has_clover = false;
    std::map<std::string, wl::Tuned> tuned;
    // set for a block of a domain decomposition (wl_dd): its links see the
    // neighbouring blocks across the cut faces, so only the _dd calls apply it
    int dd_part = 0;
};

namespace wl {

Geom make_geom(const int* dims);
int validate_lattice(const wl_lattice* lat);
// Gauge object of the lattice `local`, its links read from the canonical field
// U of the lattice `global` at the block that starts at `origin` (nullptr:
// the undivided lattice, global = local).
int gauge_create(wl_gauge* out, const wl_lattice* local, const wl_lattice* global, const int* origin,
                 const double* U, int prec_mask, cudaStream_t s);

// Canonical (x-fastest) site index of half-site i of parity p: the half
// index runs over x/2 fastest, then y, z, t; the site's parity fixes x's
// lowest bit.
__device__ __forceinline__ long long site_of_half(const Geom& g, int p, long long i)
{
    const long long row = i / g.Lxh;  // (y, z, t) row
    const int y = (int)(row % g.L[1]);
    const int z = (int)((row / g.L[1]) % g.L[2]);
    const int t = (int)(row / ((long long)g.L[1] * g.L[2]));
    return 2 * i + ((p + y + z + t) & 1);
}

// Make sure the reduction scratch holds `slots` slots of `blocks` blocks.
int ensure_red(wl_gauge g, int slots, long long blocks);
// Make sure g->tmp[prec] holds at least `bytes`.
int ensure_tmp(wl_gauge g, int prec, size_t bytes);

// Clover term (clover.cu): release its storage; out = A in or A^-1 in on
// half fields of one parity (strides in bytes between right-hand sides, 0:
// contiguous).
void free_clover(wl_gauge g);
int launch_clover_apply(wl_gauge g, int prec, void* out, const void* in, int parity, int inverse,
                        int nrhs, cudaStream_t s, long long rs_out, long long rs_in);

// Hopping kernel launch description.  Fields are per output parity where an
// array of two is given; strides are bytes between right-hand sides.
struct HopLaunch {
    int prec = WL_F32;
    int dagger = 0;
    int parity0 = 0;   // first output parity
    int nparity = 1;   // 1 or 2 (both parities in one launch: the full D)
    int nrhs = 1;
    const void* in[2] = {nullptr, nullptr};
    void* out[2] = {nullptr, nullptr};
    const void* x1[2] = {nullptr, nullptr};  // out = x1 + b1 * x2 + a * H in
    const void* x2[2] = {nullptr, nullptr};
    const void* w[2] = {nullptr, nullptr};   // fused (w, out) and ||out||^2
    long long rs_in = 0, rs_out = 0, rs_x1 = 0, rs_x2 = 0, rs_w = 0;
    double a = 1.0, b1 = 0.0;
    bool dot = false;
    double* dot_out = nullptr;  // 3 doubles per rhs, stride dot_stride doubles
    int dot_stride = 3;
    const int* active = nullptr;  // skip right-hand sides whose flag is 0
    int active_stride = 1;
    // clover term (Eq. 2): 0 none; 1 out = x1 + b1 C x2 + a H in;
    // 2 out = C (x1 + b1 x2 + a H in); C = clov[k] per output parity
    int cl_mode = 0;
    const void* clov[2] = {nullptr, nullptr};
};

int launch_hop(wl_gauge g, const HopLaunch& h, cudaStream_t s);

// record-or-not helpers for per-launch timing
// Attach the clover field F (canonical FP64, device; NULL detaches) to g:
// wl_clover_set without its entry checks.
int clover_set(wl_gauge g, const double* F, cudaStream_t s);
void timing_begin(wl_gauge g, cudaStream_t s, double bytes, int prec, int* slot);
void timing_end(wl_gauge g, cudaStream_t s, int slot);
// Solver graphs: launches captured between timing_capture_begin and
// timing_capture_end are timed by capture slots; after each replay,
// timing_replayed appends one record per capture slot, and timing_harvest
// reads the replay's times (before the next replay records them again).
void timing_capture_begin(wl_gauge g);
size_t timing_capture_end(wl_gauge g);
void timing_replayed(wl_gauge g, size_t nslots);
int timing_harvest(wl_gauge g);

// BLAS-1 / reductions (blas.cu).  Vectors are `nhalf` half fields per rhs
// back to back; rhs stride = nhalf * spinor_field_bytes(prec, Vh).
// A stride argument of 0 selects the default (nhalf half fields per rhs).
int launch_cdot(wl_gauge g, int prec, const void* a, const void* b, int nhalf, int nrhs,
                double* out, int out_stride, const int* mask, cudaStream_t s, long long rs = 0);
int launch_convert(wl_gauge g, int pdst, void* dst, int psrc, const void* src, int nhalf, int nrhs,
                   const int* mask, cudaStream_t s, long long dst_rs = 0, long long src_rs = 0);
int launch_zero(wl_gauge g, int prec, void* dst, int nhalf, int nrhs, const int* mask,
                cudaStream_t s);
// x_hi (precision phi: FP64 or df64) += x_lo (precision plo)
int launch_accum_hi(wl_gauge g, int phi, void* xhi, int plo, const void* xlo, int nhalf, int nrhs,
                    const int* mask, cudaStream_t s, long long hi_rs = 0);

bool is_capturing(cudaStream_t s);

// Layout conversion for any storage precision (including the internal df64).
// out_rs / in_rs: bytes between right-hand sides of the internal field (0:
// contiguous half fields).
int field_to_internal(wl_gauge g, void* out, const double* in, int parity, int prec, int nrhs,
                      cudaStream_t s, long long out_rs = 0);
int field_to_canonical(wl_gauge g, double* out, const void* in, int parity, int prec, int nrhs,
                       cudaStream_t s, long long in_rs = 0);

// Blocks of `kernel` (block threads, dynamic smem bytes) that fit on the whole
// GPU at once: the grid of a grid-stride kernel whose reduction should have
// few partials.
// Round-up reciprocal (m, shift) with floor(n m / 2^(32 + shift)) = n / divisor
// for 0 <= n < 2^31 (m = 0: the divisor is 1); see make_geom.
void fast_div_magic(int divisor, unsigned* m, int* shift);
int resident_grid(const void* kernel, int block, size_t smem);

// Second stage of a multi-slot reduction: one block per slot sums
// partial[slot * stride + b] (3 doubles each, b < nblocks) in block order and
// writes out[slot * out_stride + 0..2] for slots whose active flag is set.
int launch_finish_slots(const double* partial, long long stride, int nblocks, int nslots,
                        double* out, int out_stride, const int* active, int active_stride,
                        cudaStream_t s);

}  // namespace wl
