/*
 * wilson.h -- C ABI of the GB300 Wilson-matrix library.
 *
 * The library applies the Wilson fermion matrix of lattice QCD,
 *     D(x,y) = delta_{x,y} - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                                           + (1 + gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} ]
 * (Eq. 1, Sec. 2 "Wilson Fermion Matrix"), and solves D x = b with BiCGStab
 * (Sec. 2, the paragraph after Table 1), in FP64, FP32 and FP16 storage, with
 * FP64 defect correction or reliable updates (the "mixed precision solver"
 * that the same paragraph names), for many right-hand sides at once.
 *
 * Conventions
 *   Lattice   extents Lx, Ly, Lz, Lt, all even and >= 2; site index
 *             s = x + Lx*(y + Ly*(z + Lz*t)) (x fastest, as in Sec. 4.1).
 *             V = Lx*Ly*Lz*Lt, Vh = V/2.  Parity of a site = (x+y+z+t) mod 2;
 *             the half index of site s is s/2.
 *   Gamma     the paper fixes no basis; the library uses the Hermitian chiral
 *             (DeGrand-Rossi) basis, gamma_5 = diag(1, 1, -1, -1).
 *   Boundary  Sec. 2 allows periodic or antiperiodic conditions.  A hop across
 *             the lattice edge in direction mu is multiplied by the unit phase
 *             phi_mu (forward) or conj(phi_mu) (backward).
 *   Canonical FP64 layouts (what callers hand in):
 *             gauge field  U[V][4][3][3] complex double (re, im interleaved)
 *             fermion      psi[nrhs][V][4][3] complex double (spin, colour)
 *   Internal  half-lattice fields in the library's own structure-of-arrays
 *             layout (one per parity and right-hand side); their size comes
 *             from wl_field_bytes() and they are produced and read back with
 *             wl_field_to_internal() / wl_field_to_canonical().
 *
 * Ownership and streams
 *   The caller owns every field buffer (x, b, in, out) and the CUDA stream;
 *   `stream` is a cudaStream_t (NULL = legacy default stream).  A wl_gauge
 *   owns its internal link copies and solver workspace and frees them in
 *   wl_gauge_destroy().  All calls except the solves are asynchronous on
 *   `stream`; the solves synchronise `stream` before returning.
 *
 * Errors
 *   Every call returns 0 (WL_OK) or a negative WL_ERR_* code; the message of
 *   the last error on the calling thread is returned by wl_last_error().
 *   Arguments are validated on the host before any launch.
 */
#ifndef WILSON_H
#define WILSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage precisions.  WL_DF64 stores each real as an unevaluated sum of two
 * FP32 numbers (hi + lo, a 48-bit significand) in FP64-sized fields and
 * computes with FP32 instructions (~2^-44 relative rounding per operation);
 * mixed-precision solves use it for their intermediate outer residuals,
 * because GB300 executes FP32 many times faster than FP64.  The final
 * convergence check of every solve is IEEE FP64. */
typedef enum { WL_F64 = 0, WL_F32 = 1, WL_F16 = 2, WL_DF64 = 3 } wl_prec;

#define WL_PREC_MASK(p) (1 << (p))
#define WL_PREC_ALL 15

/* Flag for wl_gauge_create's prec_mask: also keep the FP32 / FP16 links in a
 * compressed form -- the first two rows of each SU(3) matrix, the third
 * rebuilt in the kernel as the complex conjugate of their cross product, the
 * boundary phase applied on the fly -- and use it in the hopping kernels of
 * those precisions: 384 instead of 576 bytes of links per site in FP32 (192
 * instead of 288 in FP16), a bandwidth reduction of the Table 1 traffic.
 * Requires SU(3) links (unitary with det 1 to 1e-6; checked, WL_ERR_ARG
 * otherwise).  The uneven-batch solver keeps using the full links. */
#define WL_LINKS_R12 (1 << 8)

/* Flag for wl_gauge_create's prec_mask: also keep the FP32 links in an
 * eight-real form and use it in single-RHS FP32 hopping launches without a
 * clover term (256 instead of 576 bytes of links per site).  Per hop matrix:
 * with its rows taken in the cyclic order that puts the smaller of |U_00|,
 * |U_10| first, rows (a, b, c), the stored reals are a2, a3, b1 and the
 * quarter-angle tangents of the phases of a1 and c1 (the first carrying +3
 * when the order is shifted); the kernel rebuilds the rest from unitarity and
 * det 1, the boundary phase applied on the fly as for WL_LINKS_R12.  Entries
 * near zero come back with an absolute error of about the square root of the
 * FP32 rounding (2.4e-4), the others to FP32 rounding.  Requires SU(3) links
 * (checked as for WL_LINKS_R12).  Multi-RHS, clover, decomposed and batch
 * launches keep the other link forms.  On a GB300 the decode costs more than
 * the bytes it saves (32^3 x 64 FP32 hopping term 127 us, against 96 us with
 * WL_LINKS_R12 and 119 us with full links), so it is an option, not a default. */
#define WL_LINKS_R8 (1 << 9)

enum {
    WL_OK = 0,
    WL_ERR_ARG = -1,            /* invalid argument (message says which) */
    WL_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    WL_ERR_NOT_CONVERGED = -3,  /* maxiter reached; x holds the best iterate */
    WL_ERR_BREAKDOWN = -4,      /* BiCGStab broke down more often than it may restart */
    WL_ERR_NAN = -5,            /* a reduction produced NaN or Inf */
    /* -6 is unused: no kernel of the library waits on another */
    WL_ERR_STATE = -7           /* the gauge object lacks what the call needs */
};

typedef struct {
    int dims[4];       /* Lx, Ly, Lz, Lt: even, >= 2 */
    double kappa;      /* hopping parameter, kappa = 1/(8 + 2 m0) (Eq. 1); |kappa| < 1/8
                          guarantees that D is invertible */
    double bc_re[4];   /* boundary phase phi_mu = bc_re + i bc_im per direction, |phi| = 1 */
    double bc_im[4];
} wl_lattice;

typedef struct wl_gauge_s* wl_gauge;

/* Create a gauge object from the canonical FP64 gauge field U (device memory,
 * V*4*9 complex, Sec. 2 "link variable").  prec_mask selects which internal
 * link copies to build (WL_PREC_MASK(WL_F32) | ...); FP64 links are always
 * built because the final residual of every solve is FP64, and df64 links
 * whenever FP32 or FP16 is requested (the outer corrections use them).  Returns
 * WL_ERR_ARG for odd or small extents, |phi| != 1 or a NULL pointer.  U is
 * only read during the call (stream-ordered) and may be freed afterwards. */
int wl_gauge_create(wl_gauge* g, const wl_lattice* lat, const double* U, int prec_mask,
                    void* stream);
int wl_gauge_destroy(wl_gauge g);

/* Vh of the gauge object's lattice. */
long long wl_half_volume(wl_gauge g);

/* Bytes of `nrhs` internal half-lattice fields of precision `prec`, stored
 * back to back (right-hand side r starts at r * wl_field_bytes(g, prec, 1)).
 * A full-lattice internal field is two half fields, even then odd. */
size_t wl_field_bytes(wl_gauge g, wl_prec prec, int nrhs);

/* Copy the parity-`parity` sites of nrhs canonical FP64 fields `in` (device,
 * nrhs*V*12 complex) into internal half fields `out` of precision `prec`
 * (FP16 stores each site scaled by its largest |real component|, kept as a
 * per-site FP32 norm).  Asynchronous. */
int wl_field_to_internal(wl_gauge g, void* out, const double* in, int parity, wl_prec prec,
                         int nrhs, void* stream);

/* Inverse of wl_field_to_internal: write the parity-`parity` sites of the
 * canonical fields `out`; the other parity's sites are left untouched. */
int wl_field_to_canonical(wl_gauge g, double* out, const void* in, int parity, wl_prec prec,
                          int nrhs, void* stream);

/* Hopping term (the Dslash) between checkerboards, Eq. 1's bracketed sum:
 *     out_p = H_{p,1-p} in_{1-p},   p = out_parity,
 * for nrhs right-hand sides (half fields back to back).  dagger = 1 applies
 * the hopping term of D^dag (gamma_mu -> -gamma_mu).  No kappa.  `out` and
 * `in` must not overlap.  Flop count: 1320 per output site per right-hand
 * side. */
int wilson_dslash(wl_gauge g, void* out, const void* in, int out_parity, int dagger,
                  wl_prec prec, int nrhs, void* stream);

/* Matrix apply:
 *   eo = 0: out = D in on full-lattice internal fields (Eq. 1; 1368 flop/site);
 *   eo = 1: out = M_ee in = in - kappa^2 H_eo H_oe in on even half fields
 *           (the Schur complement of D on the even sites).
 * With a clover term attached (wl_clover_set), D is D_clov of Eq. 2 and
 *   eo = 0: out_p = A_pp in_p - kappa H_{p,1-p} in_{1-p},  A = 1 + F;
 *   eo = 1: out = M_ee in = A_ee in - kappa^2 H_eo A_oo^-1 H_oe in.
 * dagger = 1 applies D^dag / M_ee^dag (F is Hermitian, so A is unchanged).
 * `out` and `in` must not overlap.  eo = 1 uses an odd-parity temporary from
 * the gauge object's workspace. */
int wilson_mult(wl_gauge g, void* out, const void* in, int eo, int dagger, wl_prec prec,
                int nrhs, void* stream);

/* Clover term (Eq. 2, Sec. 2 "Clover Fermion Matrix"):
 *     D_clov(x,y) = D(x,y) + F(x) delta_{x,y},
 * F(x) a 12x12 Hermitian matrix, block diagonal in the chiral basis with two
 * 6x6 Hermitian blocks: block b acts on spins {2b, 2b+1}.  The paper takes F
 * as given (its construction is outside the cost model); so does the library.
 *
 * wl_clover_set attaches F to the gauge object: from then on wilson_mult,
 * wilson_solve and wilson_solve_batch use D_clov; wilson_dslash stays the
 * hopping term.  F is device memory, FP64, F[V][2][6][6] complex (re, im
 * interleaved; row/column index = local spin * 3 + colour, local spin =
 * spin - 2b), canonical site order.  F must be Hermitian: an input whose
 * blocks depart from it by more than 1e-10 of their largest entry returns
 * WL_ERR_ARG, as does a site where A = 1 + F is singular (pivot below 1e-13
 * of the block's largest entry) or, for a gauge object holding FP16, an entry
 * of A or A^-1 beyond 6e4.  The library computes A and A^-1 per site in FP64
 * and keeps both for each parity in every precision the gauge object holds
 * (72 reals per site each: 576 B FP64/df64, 288 B FP32, 144 B FP16).  Returns
 * after the set-up has finished (F may be freed).  F = NULL detaches the term.
 * On error no clover term is attached. */
int wl_clover_set(wl_gauge g, const double* F, void* stream);

/* Site-diagonal part of D_clov on half fields of parity `parity`:
 *     out = A in (inverse = 0)   or   out = A^-1 in (inverse = 1),
 * nrhs fields back to back.  WL_ERR_STATE without a clover term.  `out` may
 * equal `in`.  Asynchronous. */
int wl_clover_apply(wl_gauge g, void* out, const void* in, int parity, int inverse,
                    wl_prec prec, int nrhs, void* stream);

/* Per-right-hand-side complex dot products and norms of internal half
 * fields (the global reductions of BiCGStab, Sec. 2):
 *     out[3r+0] + i out[3r+1] = sum conj(a_r) b_r,   out[3r+2] = ||b_r||^2.
 * `out` is device memory (3*nrhs doubles); accumulation is FP64 from the
 * warp level up.  Uses partial sums in the gauge object's workspace. */
int wl_cdot(wl_gauge g, double* out, const void* a, const void* b, wl_prec prec, int nrhs,
            void* stream);

/* Limits of wl_cdot_noalloc's built-in scratch. */
#define WL_NOALLOC_MAX_RHS 64
#define WL_NOALLOC_BLOCKS 512

/* wl_cdot without any device allocation.  The paper has no counterpart: this
 * is a library facility for callers that cannot allocate device memory --
 * code running inside another framework's memory pool that must not call
 * cudaMalloc behind it, latency-critical loops in which cudaMalloc/cudaFree
 * would synchronise the device, and callers holding raw field pointers but no
 * gauge object (wl_cdot keeps its scratch in the gauge object's workspace).
 * Same results as wl_cdot (up to summation order), in every precision
 * including WL_DF64, for nrhs half fields of Vh sites, stored back to back
 * with stride wl_field_bytes(g, prec, 1); `out` is device memory for 3*nrhs
 * doubles.  WL_F16 needs Vh divisible by 4 (a field takes 52 Vh bytes and the
 * next one must start on a 16-byte boundary; every lattice with even extents
 * has Vh divisible by 8); WL_ERR_ARG otherwise.  Scratch is one fixed
 * __device__ array of WL_NOALLOC_MAX_RHS x WL_NOALLOC_BLOCKS x 3 doubles
 * (768 KiB) that every GPU loading the library holds until the process exits;
 * nrhs above WL_NOALLOC_MAX_RHS returns WL_ERR_ARG.  Every call looks up the
 * array's device address in the current context (cudaGetSymbolAddress, a
 * host-side query), so it stays valid after the context is reset; the first
 * call on a device may load the library's device code, so make it before any
 * stream capture.  All calls share the array and each call overwrites what
 * the previous one left: calls that overlap on the GPU race.  Never calls
 * cudaMalloc, cudaFree or any allocating routine.  Asynchronous. */
int wl_cdot_noalloc(double* out, const void* a, const void* b, long long Vh, wl_prec prec,
                    int nrhs, void* stream);

typedef struct {
    double tol;        /* stop when ||b - D x||_2 / ||b||_2 <= tol (full D, FP64), per RHS */
    int maxiter;       /* bound on inner iterations, per RHS */
    int eo;            /* 1: solve the even-odd Schur system M_ee x_e = b_e + kappa H_eo b_o */
    wl_prec inner;     /* precision of the Krylov iteration; WL_F64 = plain FP64 BiCGStab */
    double inner_tol;  /* defect correction: relative tolerance of each inner solve (0: default,
                          3e-6 for an FP32 inner solve, 1e-3 for FP16) */
    double delta;      /* > 0: reliable updates (recompute the FP64 residual when the iterated
                          residual drops below delta times its maximum since the last update)
                          instead of restarted defect correction */
    int use_x0;        /* 1: x holds the initial guess */
    int graph_iters;   /* > 0: capture this many iterations per CUDA-graph replay (the host
                          checks convergence after each replay); 0: the same with 4; < 0:
                          eager launches with a host check every -graph_iters iterations.
                          A chunk the solver predicts shorter than this runs eagerly. */
} wl_solve_params;

typedef struct {
    int iters;          /* inner iterations */
    int outer;          /* FP64 residual recomputations (defect corrections / reliable updates) */
    int restarts;       /* breakdown restarts */
    int status;         /* WL_OK or WL_ERR_* for this right-hand side */
    double true_resid;  /* final ||b - D x|| / ||b||, FP64 on the GPU */
    double secs;        /* wall time of the whole call */
} wl_solve_info;

/* Solve D x_r = b_r (D_clov with a clover term attached; its even-odd system
 * is A_ee - kappa^2 H_eo A_oo^-1 H_oe with b' = b_e + kappa H_eo A_oo^-1 b_o
 * and x_o = A_oo^-1 (b_o + kappa H_oe x_e)) for nrhs right-hand sides
 * (canonical FP64, nrhs*V*12 complex each).  x and b may be device or host memory (host buffers are
 * staged through the gauge object's workspace).  info has nrhs entries.
 * Returns WL_OK when every right-hand side reached tol, else the first
 * failing status; x always holds the best iterate. */
int wilson_solve(wl_gauge g, double* x, const double* b, int nrhs, const wl_solve_params* p,
                 wl_solve_info* info, void* stream);

/* Solve nlat independent systems of different lattices together (the
 * batched form of wilson_solve): gauge object gs[l] with nrhs[l] right-hand
 * sides x[l], b[l] (canonical; device or host memory, host buffers staged
 * through each gauge object's workspace).  Each inner BiCGStab operator
 * is one persistent hopping launch over 32-site tiles of all lattices (tiles
 * of lattices whose systems have all stopped are skipped), each vector update
 * one launch over all systems.  The outer work (set-up, FP64 residuals, final
 * check, host copies) runs per lattice on each gauge object's own stream, so
 * that the lattices' steps overlap; the call returns when all are done.  Limits:
 * 1 <= nlat <= 64, 1 <= nrhs[l] <= 32, even-odd systems only (p->eo = 1),
 * each gauge object at most once; WL_ERR_ARG otherwise.  A gauge object
 * with a clover term contributes D_clov.  info receives sum(nrhs) entries,
 * lattice by lattice.  The device description of a batch is cached for the
 * set of gauge objects (the 8 most recent sets), so callers alternating
 * between batches do not rebuild it; a gauge object's destruction drops the
 * descriptions that include it.  Calls must not overlap on the same gauge
 * objects (as for wilson_solve).  Synchronises the stream. */
int wilson_solve_batch(int nlat, const wl_gauge* gs, double* const* x, const double* const* b,
                       const int* nrhs, const wl_solve_params* p, wl_solve_info* info,
                       void* stream);

/* ------------------------------------------------------------------------
 * Domain decomposition (Sec. 4.4 "Thread Task Assignment"; the multi-node
 * setting of Sec. 5.2.3 and Sec. 6).
 *
 * The lattice is cut into grid[1] x grid[2] x grid[3] equal blocks along y, z
 * and t (grid[0] must be 1: x is never cut, as in Sec. 4.1); block extents
 * must be even and >= 2.  Block k has coordinates (0, k % g1, (k / g1) % g2,
 * k / (g1 g2)) and holds the sites whose global coordinates lie in
 * [coord_mu * L_mu / grid_mu, (coord_mu + 1) * L_mu / grid_mu).  Each block is
 * a gauge object (wl_dd_block) with its own link copies; its fields are the
 * library's internal half fields of the block lattice (wl_field_bytes,
 * wl_field_to_internal / wl_field_to_canonical on the block's gauge object,
 * with block-local canonical fields).  The hopping term of a block reads the
 * neighbouring blocks' spinors through halo buffers: each application packs
 * the spin-projected half spinors of the cut faces (12 reals per face site),
 * moves them to the neighbours' halos (a copy kernel, or, in the direct mode,
 * the pack kernel writes them there itself) and computes the boundary sites,
 * all on a second stream while the interior sites are computed on `stream`.
 * Global sums are formed per block and added over the blocks in block order.
 * Every output site is computed with the undivided kernel's operations, so
 * the hopping term is bit for bit that of the undivided lattice; sums differ
 * by their summation order.
 *
 * All blocks live on the calling thread's current GPU.  The calls are
 * asynchronous on `stream` except wl_dd_create, wl_dd_destroy,
 * wl_dd_set_exchange, wl_dd_clover_set and wilson_solve_dd.  Block gauge
 * objects belong to the decomposition: wilson_dslash, wilson_mult,
 * wilson_solve(_batch) and wl_clover_set refuse them (WL_ERR_STATE); the
 * clover term of the decomposed operator is attached with wl_dd_clover_set.
 * ---------------------------------------------------------------------- */
typedef struct wl_dd_s* wl_dd;

/* Create a decomposition of the lattice `lat` into grid[0..3] blocks (at most
 * 16), all held by this process, its links from the canonical FP64 gauge
 * field U of the whole lattice (device memory, read during the call).
 * prec_mask as for wl_gauge_create. */
int wl_dd_create(wl_dd* dd, const wl_lattice* lat, const int grid[4], const double* U, int prec_mask,
                 void* stream);

/* One face message of a halo exchange (the "communication" step of Sec. 4.4):
 * a packed face that one block sends to a neighbouring block, seen from one
 * end.  Faces are the spin-projected half spinors of a block's x_mu = 0
 * (side 0, sent to the backward neighbour) or x_mu = L_mu - 1 (side 1, sent
 * to the forward neighbour) sites, 6 complex per face site in the
 * arithmetic precision (FP64 / df64: 96 B, FP32: 48 B per site; FP16
 * storage: 48 B of the projection of the stored 16-bit values, not yet
 * multiplied by the site's norm, then the FP32 norms of the face sites, padded
 * to a multiple of 16 B), all right-hand sides back to back.  Layout of one
 * right-hand side's face in FP64: 6 planes of one complex double per face site, plane 3 s + c
 * holding spin row s (0 or 1) and colour c of (1 - gamma_mu) psi (side 0) or
 * (1 + gamma_mu) psi (side 1) at that site (the dagger flips the signs); the
 * two rows determine the other two.  Face sites are ordered by their half
 * index with the mu coordinate dropped (x / 2 fastest, then the remaining
 * directions in the order y, z, t). */
typedef struct {
    int send;       /* 1: send `bytes` at `buf` to block `peer`; 0: receive them from `peer` into `buf` */
    int block;      /* the block of this process the message belongs to */
    int peer;       /* the block at the other end */
    int tag;        /* equal at both ends: 12 * (receiving block) + segment, segment =
                       6 * launch parity + 2 * (mu - 1) + side */
    size_t offset;  /* byte offset of the face in the block's send (send = 1) or halo region */
    size_t bytes;
    void* buf;      /* device address (NULL from wl_dd_plan) */
} wl_dd_msg;

/* How faces and global sums reach blocks held by other processes.  Both
 * callbacks return 0 or a negative code (which the calling entry point
 * returns as WL_ERR_CUDA); `stream` is the cudaStream_t whose earlier work
 * produced the data, and work issued on it after the call must see the
 * result (e.g. NCCL calls on that stream, or a synchronisation of it before
 * host-side transfers that complete before returning).
 *   exchange   perform every message of msgs (sends and receives);
 *   allreduce  sum n doubles at buf (device) over all processes, in place;
 *   all        nonzero: route faces between blocks of this process through
 *              exchange too (otherwise they are device copies). */
typedef struct {
    void* ctx;
    int (*exchange)(void* ctx, int nmsg, const wl_dd_msg* msgs, void* stream);
    int (*allreduce)(void* ctx, double* buf, int n, void* stream);
    int all;
} wl_dd_transport;

/* A decomposition of which this process holds blocks first .. first+count-1
 * (at most 16); faces of other blocks and the global sums go through `tr`
 * (required when count is below the number of blocks, optional otherwise;
 * copied, and used until wl_dd_destroy).  U is the whole lattice's canonical
 * gauge field on this device (its held blocks and their faces are read). */
int wl_dd_create_part(wl_dd* dd, const wl_lattice* lat, const int grid[4], int first, int count,
                      const double* U, int prec_mask, const wl_dd_transport* tr, void* stream);

/* The face messages of block `block` of a decomposition of the lattice dims
 * into grid blocks, for one hopping application of precision prec, nrhs
 * right-hand sides and nparity (1 or 2) output parities: every message,
 * local or not, with buf = NULL.  Host code only (no GPU needed).  Returns
 * the number of messages (at most 24), or a negative code; writes at most
 * max_msgs entries. */
int wl_dd_plan(const int dims[4], const int grid[4], int block, wl_prec prec, int nrhs, int nparity,
               wl_dd_msg* msgs, int max_msgs);
int wl_dd_destroy(wl_dd dd);
/* Number of blocks this process holds (0 for NULL). */
int wl_dd_blocks(wl_dd dd);
/* Gauge object and grid coordinates of the k-th block held here (either
 * output may be NULL).  Arrays of block fields below are in this order. */
int wl_dd_block(wl_dd dd, int k, wl_gauge* g, int coord[4]);
/* Exchange of the packed faces between blocks of this process: 0 = the pack
 * kernel writes each block's own send buffer and one copy kernel moves every
 * face to the neighbour's halo (the default; the step a transport takes over
 * for blocks held elsewhere); 1 = the pack kernel writes straight into the
 * neighbours' halos.  Both run on a second stream, overlapping the interior
 * sweep.  Synchronises the device. */
int wl_dd_set_exchange(wl_dd dd, int mode);

/* Clover term of the decomposed operator (Eq. 2): F as for wl_clover_set,
 * for the whole lattice (device, canonical order, read during the call); each
 * block held here takes its sites' matrices.  From then on wilson_mult_dd and
 * wilson_solve_dd use D_clov (the fused clover epilogues of the undivided
 * operator, so the result is again bit for bit the undivided one);
 * wilson_dslash_dd stays the hopping term.  F = NULL detaches the term.  Errors
 * as wl_clover_set; on error no block keeps a term.  Synchronises the stream. */
int wl_dd_clover_set(wl_dd dd, const double* F, void* stream);

/* Copy nrhs canonical FP64 fields of the whole lattice (`global`, device,
 * nrhs*V*12 complex) to block-local canonical fields of the held blocks
 * (local[k], device, nrhs*V_block*12 complex), and back (gather writes the
 * held blocks' sites only).  Asynchronous. */
int wl_dd_scatter(wl_dd dd, double* const* local, const double* global, int nrhs, void* stream);
int wl_dd_gather(wl_dd dd, double* global, const double* const* local, int nrhs, void* stream);

/* wilson_dslash on the decomposed lattice: out[k] = H_{p,1-p} in[k] for every
 * block k (internal half fields of the block lattice, nrhs back to back). */
int wilson_dslash_dd(wl_dd dd, void* const* out, const void* const* in, int out_parity, int dagger,
                     wl_prec prec, int nrhs, void* stream);
/* wilson_mult on the decomposed lattice (eo = 0: full D on [even | odd]
 * block fields; eo = 1: M_ee on even block fields). */
int wilson_mult_dd(wl_dd dd, void* const* out, const void* const* in, int eo, int dagger, wl_prec prec,
                   int nrhs, void* stream);
/* wl_cdot over the whole lattice: each block's local sums, then their total
 * (the allreduce) in out (device, 3*nrhs doubles). */
int wl_cdot_dd(wl_dd dd, double* out, const void* const* a, const void* const* b, wl_prec prec, int nrhs,
               void* stream);
/* wilson_solve on the decomposed lattice: every inner iteration applies the
 * decomposed M_ee (two halo exchanges) and sums its dot products over the
 * blocks (one allreduce per reduction).  x[k], b[k]: block-local canonical
 * FP64 fields (device), nrhs each.  Even-odd systems only (p->eo = 1), eager
 * launches (|graph_iters| is read as the host-check interval, 4 when 0).  info has nrhs
 * entries.  Synchronises the stream. */
int wilson_solve_dd(wl_dd dd, double* const* x, const double* const* b, int nrhs, const wl_solve_params* p,
                    wl_solve_info* info, void* stream);

/* Encoding of the 16-bit words of WL_F16 spinors in this build.  Both forms
 * store each value divided by its site's max |component| (the FP32 norm kept
 * beside the site), so that it lies in [-1, 1]:
 *   0  IEEE binary16, round to nearest even (the default build);
 *   1  int16 fixed point: round(32767 v), stored biased by 32768 (a build
 *      with -DWL_SPINOR16_FIXED=1).
 * Links and clover matrices of WL_F16 are binary16 in both builds. */
int wl_spinor16_format(void);

/* Message of the last failed call on this thread ("" if none). */
const char* wl_last_error(void);

/* Kernels the library has launched so far in this process (a CUDA-graph
 * replay counts every kernel node it runs). */
long long wl_launch_count(void);

/* Algorithmic bytes of those launches: each kernel counts the fields it must
 * read and write once (links once per hopping launch for all right-hand
 * sides, every spinor operand once), not the traffic the hardware saw.
 * Iterations a solver chunk launched after every right-hand side had
 * stopped (whose kernels exit at once) are taken out again. */
double wl_algorithmic_bytes(void);

/* Per-launch CUDA-event timing of the hopping kernels launched by this gauge
 * object: eager launches, and the launches of wilson_solve's graph replays
 * (each replay adds one record per hopping launch of the graph, read from
 * event-record nodes once the replay has run); launches in other captured
 * graphs are not timed.  enable = 1 clears and starts recording, enable = 0
 * stops.  wl_timing_read
 * returns, for hopping launches of precision `prec` (-1: all), the summed
 * kernel time in ms, the number of timed launches and their summed
 * algorithmic bytes, leaving out launches that found no work (a solver
 * chunk's iterations after every right-hand side had stopped).  It waits for
 * the recorded events. */
int wl_timing(wl_gauge g, int enable);
int wl_timing_read(wl_gauge g, int prec, double* ms, long long* launches, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* WILSON_H */
