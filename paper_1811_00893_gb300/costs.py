"""Per-site cost model: flops and algorithmic HBM bytes.

Sec. 2, Table 1 counts, per lattice site of the Wilson matrix in single
precision, 1368 flops and 1536 bytes moved with no cache reuse; with ideal
reuse (each link used twice, each spinor nine times) the traffic drops to a
byte/flop ratio of 0.351.  The functions below reproduce those figures and
extend them to the even-odd hopping kernels this library runs, whose
algorithmic bytes count every input spinor once, every link once per hopping
application and every output once.
"""
from __future__ import annotations

NC, NS = 3, 4
SPINOR_REALS = 2 * NC * NS          # 24
LINK_REALS = 2 * NC * NC            # 18
HALF_SPINOR_REALS = SPINOR_REALS // 2

# flops of one hopping application per output site: per direction a spin
# projection (12), two SU(3) x colour-vector products (2 x 66) and the
# accumulation into four spin components (24), less the first accumulation.
FLOPS_PROJECT = 2 * NC * 2          # 6 complex adds = 12
FLOPS_SU3_VEC = 9 * 6 + 6 * 2       # 9 complex mul + 6 complex add = 66
FLOPS_HOP_SITE = 8 * (FLOPS_PROJECT + 2 * FLOPS_SU3_VEC + SPINOR_REALS) - SPINOR_REALS  # 1320
FLOPS_D_SITE = FLOPS_HOP_SITE + 2 * SPINOR_REALS  # kappa * h and the subtraction: 1368


def paper_bytes_per_site(word: int = 4, ideal_reuse: bool = False) -> int:
    """Table 1's traffic per site of D: eight neighbour spinors, the site's own
    spinor, eight links and the output (no reuse), or one spinor in, one out
    and four links (ideal reuse: links twice, spinors nine times)."""
    if ideal_reuse:
        return word * (4 * LINK_REALS + 2 * SPINOR_REALS)
    return word * (9 * SPINOR_REALS + 8 * LINK_REALS + SPINOR_REALS)


def paper_byte_per_flop(ideal_reuse: bool = False) -> float:
    return paper_bytes_per_site(4, ideal_reuse) / FLOPS_D_SITE


def roofline_gflops(bandwidth_gbs: float, ideal_reuse: bool = False) -> float:
    """Bandwidth-bound flop rate, as in Table 1's roofline columns."""
    return bandwidth_gbs / paper_byte_per_flop(ideal_reuse)


# ---- this library's kernels -------------------------------------------------

#: bytes per real, per storage precision
WORD = {"f64": 8, "f32": 4, "f16": 2}
#: per-site norm bytes that ride along with an FP16 spinor
NORM_BYTES = {"f64": 0, "f32": 0, "f16": 4}


def spinor_bytes(prec: str) -> int:
    return SPINOR_REALS * WORD[prec] + NORM_BYTES[prec]


def link_bytes(prec: str, r12: bool = False) -> int:
    """Bytes of one stored link: 18 reals, or 12 with two-row compression
    (the third row rebuilt from unitarity)."""
    return (12 if r12 else LINK_REALS) * WORD[prec]


#: reals of the clover term per site (Eq. 2): two Hermitian 6x6 blocks = 2 x 36
CLOVER_REALS = 72


def clover_bytes(prec: str) -> int:
    """Bytes of the packed clover matrix (A = 1 + F or its inverse) per site;
    288 in single precision, Table 1's clover surplus over the Wilson matrix."""
    return CLOVER_REALS * WORD[prec]


def hop_bytes_per_site(prec: str, nrhs: int = 1, extra_in: int = 0, extra_out: int = 0,
                       clover: bool = False, r12: bool = False) -> int:
    """Algorithmic bytes per output site of one even-odd hopping kernel:
    eight links (and, with the clover term fused, one clover matrix) read
    once for all right-hand sides, one input spinor and one output spinor per
    right-hand side, plus `extra_in` / `extra_out` fused epilogue fields per
    right-hand side."""
    return (8 * link_bytes(prec, r12) + (clover_bytes(prec) if clover else 0) +
            nrhs * (1 + extra_in + 1 + extra_out) * spinor_bytes(prec))


def bicgstab_iteration_bytes(prec: str, xprec: str, eo: bool = True, clover: bool = False) -> int:
    """Algorithmic bytes per site of one BiCGStab iteration as this library
    schedules it (per half-lattice site for eo, per lattice site for the full
    D).  Matrix applies: M_ee is two hopping launches, the first writing an
    odd temporary (links, in, out) and the second fusing the xpay and the dot
    (links, in, out, x1, w); the full D is one launch per apply that fuses
    both (links, in, out, x1, w).  Vector passes: p update 4 fields, s update
    3, x/r update 5 plus reading and writing x.  With the clover term each
    hopping launch also reads one clover matrix per output site (A_oo^-1,
    then A_ee for M_ee; A for the full D)."""
    sp, lk, xb = spinor_bytes(prec), 8 * link_bytes(prec), spinor_bytes(xprec)
    if clover:
        lk += clover_bytes(prec)
    if eo:
        applies = 2 * ((lk + 2 * sp) + (lk + 4 * sp))
    else:
        applies = 2 * (lk + 4 * sp)
    return applies + (4 + 3 + 5) * sp + 2 * xb
