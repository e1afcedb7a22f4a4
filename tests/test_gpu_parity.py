"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Small lattices span several thread blocks with a ragged tail (Vh not a
multiple of the block size) and the L = 2 case where the +mu and -mu
neighbours coincide.  Tolerances (relative L2 against the FP64 oracle):
FP64 1e-12, FP32 1e-5, FP16 storage 7e-4 (twice the worst error measured by
test_fp16_error_margins; gpu_helpers.TOL).
Solves must reach a true residual ||b - D x|| / ||b|| <= 1e-10, evaluated by
the oracle's own D on the GPU's solution.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import PRECS, TOL, Case, rel
from paper_1811_00893_gb300 import wilson

pytestmark = pytest.mark.gpu

SMALL = [((4, 4, 4, 4), (1, 1, 1, -1)),          # Vh = 128: exactly one block
         ((6, 4, 2, 8), (1, np.exp(0.3j), 1, -1)),  # Vh = 192: ragged tail, L = 2, twisted phase
         ((8, 6, 4, 10), (1, 1, 1, -1)),          # Vh = 960: several blocks + tail
         ((2, 2, 2, 2), (1, 1, 1, -1)),           # L = 2 in every direction
         ((6, 2, 2, 6), (-1, 1, np.exp(1.1j), -1))]  # Vh = 72: ragged 32-site tiles and blocks


@pytest.fixture(scope="module", params=SMALL, ids=lambda c: "x".join(map(str, c[0])))
def case(request):
    dims, bc = request.param
    c = Case(dims, kappa=0.124, kind="haar", seed=7, bc=bc)
    yield c
    c.close()


def full_internal(c, psi, prec):
    nrhs = psi.shape[0]
    fb = wilson.wl_field_bytes(c.g.handle, PRECS[prec], 1)
    out = torch.empty(2 * fb * nrhs, dtype=torch.uint8, device="cuda")
    for r in range(nrhs):
        for p in (0, 1):
            seg = out[(2 * r + p) * fb:(2 * r + p + 1) * fb]
            wilson.wl_field_to_internal(c.g.handle, seg, psi[r:r + 1], p, PRECS[prec], 1)
    return out


def full_canonical(c, internal, prec, nrhs):
    fb = wilson.wl_field_bytes(c.g.handle, PRECS[prec], 1)
    out = torch.zeros((nrhs, c.V, 4, 3), dtype=torch.complex128, device="cuda")
    for r in range(nrhs):
        for p in (0, 1):
            seg = internal[(2 * r + p) * fb:(2 * r + p + 1) * fb]
            wilson.wl_field_to_canonical(c.g.handle, out[r:r + 1], seg, p, PRECS[prec], 1)
    return out


# ----------------------------------------------------------------------------
# a1: layout conversion
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
def test_conversion_round_trip(case, prec):
    psi = case.source(nrhs=2, seed=11)
    for p in (0, 1):
        internal = case.to_internal(psi, p, prec)
        back = case.to_canonical(internal, p, prec, nrhs=2)
        want = psi.clone()
        sites = torch.from_numpy(np.nonzero(
            (np.indices(case.dims[::-1]).sum(0).reshape(-1) % 2) == p)[0]).cuda()
        other = torch.ones(case.V, dtype=torch.bool, device="cuda")
        other[sites] = False
        assert torch.all(back[:, other] == 0), "conversion wrote the other parity"
        err = rel(back[:, sites].cpu().numpy(), want[:, sites].cpu().numpy())
        if prec == "f64":
            assert err == 0.0
        else:
            assert err < {"f32": 1e-7, "f16": 1.3e-3, "df64": 1e-14}[prec], err


def _df64_test_values(n, rng):
    """Doubles over the whole binary32 range, with the edge cases of the
    double-float split: both ends of its integer-arithmetic range (biased
    exponents 949 and 1149) and the exponents just outside, exact ties of the
    24-bit rounding with an odd and an even kept bit, carries into the
    exponent, signed zeros, binary32 subnormals and values below them."""
    e = rng.integers(1023 - 152, 1023 + 128, n).astype(np.uint64)  # biased exponents
    frac = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    sign = rng.integers(0, 2, n).astype(np.uint64) << np.uint64(63)
    k = n // 8
    e[:k] = rng.choice([947, 948, 949, 950, 1148, 1149, 1150], k).astype(np.uint64)
    half = np.uint64(1 << 28)
    kept = rng.integers(0, 1 << 23, 2 * k, dtype=np.uint64) << np.uint64(29)
    frac[k:3 * k] = kept | half  # ties: kept bit odd or even
    frac[3 * k:3 * k + 8] = np.uint64((1 << 52) - 1)  # rounds up into the exponent
    e[3 * k + 4:3 * k + 8] = 1149
    bits = sign | (e << np.uint64(52)) | frac
    bits[-4:] = [0, 1 << 63, 0, 1 << 63]  # signed zeros
    return bits.view(np.float64)


def test_df64_conversion_bits():
    """FP64 -> df64 -> FP64 through the layout conversions is, bit for bit,
    hi = RN32(v), lo = RN32(v - hi) and hi + lo with numpy's IEEE 754
    conversions and sum (for these values hi + lo is exact in binary64 or
    rounds the same way on both sides), on every component of both parities."""
    c = Case((4, 2, 2, 4), kappa=0.12, kind="haar", seed=3)
    try:
        rng = np.random.default_rng(17)
        v = _df64_test_values(c.V * 24, rng)
        psi = torch.from_numpy(v.copy()).view(torch.complex128).reshape(1, c.V, 4, 3).cuda()
        back = torch.zeros_like(psi)
        odd = torch.from_numpy(np.indices(c.dims[::-1]).sum(0).reshape(-1) % 2 == 1).cuda()
        for p in (0, 1):
            internal = c.to_internal(psi, p, "df64")
            part = c.to_canonical(internal, p, "df64", nrhs=1)
            sites = odd if p else ~odd
            back[:, sites] = part[:, sites]  # (a copy keeps the sign of zeros)
        hi = v.astype(np.float32)
        lo = (v - hi.astype(np.float64)).astype(np.float32)
        want = hi.astype(np.float64) + lo.astype(np.float64)
        got = torch.view_as_real(back).reshape(-1).cpu().numpy()
        bad = np.nonzero(got.view(np.uint64) != want.view(np.uint64))[0]
        assert bad.size == 0, [(v[j], got[j], want[j]) for j in bad[:5]]
    finally:
        c.close()


def test_f16_spinor_codec_error_bound(case):
    """Each component of a stored WL_F16 spinor is within the rounding of the
    build's 16-bit encoding (wl_spinor16_format) of the exact value.  With m the
    site's max |component|, binary16 rounds v/m to 11 significant bits (2^-11
    relative; 2^-25 absolute in the subnormal range), and int16 fixed point
    rounds it to the nearest multiple of 1/32767.  The FP64 -> FP32 input
    rounding, the FP32 scale 1/m and the product with m on the way back add a
    few units of 2^-24 m.  The source spans eight decades within each site, so
    it reaches binary16's subnormal range and the fixed-point format's
    small-value end."""
    psi = case.source(nrhs=1, seed=13)
    g = torch.Generator().manual_seed(5)
    psi = psi * torch.pow(10.0, -8.0 * torch.rand(psi.shape, generator=g, dtype=torch.float64)).cuda()
    fmt = wilson.wl_spinor16_format()
    assert fmt in (0, 1)
    for p in (0, 1):
        back = case.to_canonical(case.to_internal(psi, p, "f16"), p, "f16", nrhs=1)
        w = case.half(psi, p).reshape(-1, 12).view(np.float64).reshape(-1, 24)
        got = case.half(back, p).reshape(-1, 12).view(np.float64).reshape(-1, 24)
        m = np.abs(w).max(axis=1, keepdims=True)
        if fmt == 0:
            bound = 2.0 ** -11 * np.abs(w) * (1 + 2.0 ** -20) + 2.0 ** -25 * m + 5 * 2.0 ** -24 * m
        else:
            bound = (0.5 / 32767 + 6 * 2.0 ** -24) * m
        err = np.abs(got - w)
        assert np.all(err <= bound), (fmt, p, float((err / bound).max()))


# ----------------------------------------------------------------------------
# a2: hopping term
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_dslash_matches_oracle(case, prec, dagger):
    nrhs = 2
    psi = case.source(nrhs=nrhs, seed=21)
    for out_parity in (0, 1):
        inp = case.to_internal(psi, 1 - out_parity, prec)
        out = case.g.field(prec, nrhs)
        wilson.wilson_dslash(case.g.handle, out, inp, out_parity, dagger, PRECS[prec], nrhs)
        got = case.to_canonical(out, out_parity, prec, nrhs=nrhs)
        for r in range(nrhs):
            want = oracle.hop_eo(case.U, case.half(psi, 1 - out_parity, r), case.dims, case.bc,
                                 out_parity, dagger=bool(dagger))
            err = rel(case.half(got, out_parity, r), want)
            assert err < TOL[prec], (prec, out_parity, r, err)


def test_dslash_rejects_overlap_and_bad_args(case):
    psi = case.source(nrhs=1, seed=3)
    inp = case.to_internal(psi, 1, "f32")
    with pytest.raises(wilson.WilsonError) as e:
        wilson.wilson_dslash(case.g.handle, inp, inp, 0, 0, wilson.WL_F32, 1)
    assert e.value.code == wilson.WL_ERR_ARG
    out = case.g.field("f32", 1)
    with pytest.raises(wilson.WilsonError):
        wilson.wilson_dslash(case.g.handle, out, inp, 2, 0, wilson.WL_F32, 1)
    with pytest.raises(wilson.WilsonError):
        wilson.wilson_dslash(case.g.handle, out, inp, 0, 0, wilson.WL_F32, 0)


# ----------------------------------------------------------------------------
# a3: matrix applies
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_full_D_matches_oracle(case, prec, dagger):
    nrhs = 2
    psi = case.source(nrhs=nrhs, seed=31)
    inp = full_internal(case, psi, prec)
    out = torch.empty_like(inp)
    wilson.wilson_mult(case.g.handle, out, inp, 0, dagger, PRECS[prec], nrhs)
    got = full_canonical(case, out, prec, nrhs).cpu().numpy()
    for r in range(nrhs):
        want = oracle.D_full(case.U, psi[r].cpu().numpy(), case.dims, case.bc, case.kappa,
                             dagger=bool(dagger))
        assert rel(got[r], want) < TOL[prec], (prec, r)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_Mee_matches_oracle(case, prec, dagger):
    nrhs = 3
    psi = case.source(nrhs=nrhs, seed=41)
    inp = case.to_internal(psi, 0, prec)
    out = case.g.field(prec, nrhs)
    wilson.wilson_mult(case.g.handle, out, inp, 1, dagger, PRECS[prec], nrhs)
    got = case.to_canonical(out, 0, prec, nrhs=nrhs)
    for r in range(nrhs):
        want = oracle.Mee(case.U, case.half(psi, 0, r), case.dims, case.bc, case.kappa,
                          dagger=bool(dagger))
        assert rel(case.half(got, 0, r), want) < TOL[prec], (prec, r)


# ----------------------------------------------------------------------------
# a5: reductions
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
def test_cdot_matches_oracle(case, prec):
    nrhs = 3
    a = case.source(nrhs=nrhs, seed=51)
    b = case.source(nrhs=nrhs, seed=61)
    ia, ib = case.to_internal(a, 0, prec), case.to_internal(b, 0, prec)
    out = torch.zeros(3 * nrhs, dtype=torch.float64, device="cuda")
    wilson.wl_cdot(case.g.handle, out, ia, ib, PRECS[prec], nrhs)
    got = out.cpu().numpy().reshape(nrhs, 3)
    # the oracle reduces the fields as the library stores them
    ca = case.to_canonical(ia, 0, prec, nrhs)
    cb = case.to_canonical(ib, 0, prec, nrhs)
    tol = {"f64": 1e-13, "f32": 1e-6, "f16": 1e-6, "df64": 1e-13}[prec]
    for r in range(nrhs):
        ha, hb = case.half(ca, 0, r), case.half(cb, 0, r)
        d = oracle.cdot(ha, hb)
        n = oracle.cdot(hb, hb).real
        scale = np.sqrt(oracle.cdot(ha, ha).real * n)
        assert abs(complex(got[r, 0], got[r, 1]) - d) < tol * scale
        assert abs(got[r, 2] - n) < tol * n
    # deterministic: a second launch gives identical bits
    out2 = torch.zeros_like(out)
    wilson.wl_cdot(case.g.handle, out2, ia, ib, PRECS[prec], nrhs)
    assert torch.equal(out, out2)


@pytest.mark.parametrize("shape", [1, 3, 18, 20, 21, 3064, 3256])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_multi_rhs_shapes_match_oracle(monkeypatch, prec, shape):
    """Every multi-RHS launch shape the autotuner may pick (warps per block of
    the staged kernel; 16 + warps for the pipelined persistent kernel; 3000 +
    block size for one single-RHS grid row per right-hand side) gives the
    oracle's hopping term and reductions, on a lattice whose last 32-site
    tile is half empty (Vh = 144).  The solve also runs its FP64 and
    double-float multi-RHS launches in the forced shape."""
    monkeypatch.setenv("WL_MRHS_SHAPE", str(shape))
    c = Case((6, 4, 2, 6), kappa=0.124, kind="haar", seed=9, bc=(1, np.exp(0.3j), 1, -1))
    try:
        nrhs = 5
        psi = c.source(nrhs=nrhs, seed=71)
        for dagger in (0, 1):
            inp = c.to_internal(psi, 1, prec)
            out = c.g.field(prec, nrhs)
            wilson.wilson_dslash(c.g.handle, out, inp, 0, dagger, PRECS[prec], nrhs)
            got = c.to_canonical(out, 0, prec, nrhs=nrhs)
            for r in range(nrhs):
                want = oracle.hop_eo(c.U, c.half(psi, 1, r), c.dims, c.bc, 0, dagger=bool(dagger))
                assert rel(c.half(got, 0, r), want) < TOL[prec], (shape, dagger, r)
        # the reducing variant inside a multi-RHS solve
        b = c.source(nrhs=nrhs, seed=72)
        x = torch.zeros_like(b)
        p = wilson.solve_params(tol=1e-10, eo=True, inner=PRECS[prec], delta=0.1 if prec == "f16" else 0.0)
        rc, info = wilson.wilson_solve(c.g.handle, x, b, nrhs, p)
        bn, xn = b.cpu().numpy(), x.cpu().numpy()
        for r in range(nrhs):
            assert oracle.true_residual(c.U, bn[r], xn[r], c.dims, c.bc, c.kappa) <= 1e-10
    finally:
        c.close()


@pytest.mark.parametrize("shape", [2, 3064, 3128, 3256])
@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_wide_multi_rhs_shapes_match_oracle(monkeypatch, prec, shape):
    """The FP64 and double-float multi-RHS hopping term in the staged kernel
    and in one single-RHS grid row per right-hand side (the shapes the
    autotuner chooses among for the wide types) equals the oracle's, with and
    without dagger, on a lattice with a ragged last tile and a twisted phase."""
    monkeypatch.setenv("WL_MRHS_SHAPE", str(shape))
    c = Case((6, 4, 2, 6), kappa=0.124, kind="haar", seed=9, bc=(1, np.exp(0.3j), 1, -1))
    try:
        nrhs = 3
        psi = c.source(nrhs=nrhs, seed=73)
        for dagger in (0, 1):
            inp = c.to_internal(psi, 1, prec)
            out = c.g.field(prec, nrhs)
            wilson.wilson_dslash(c.g.handle, out, inp, 0, dagger, PRECS[prec], nrhs)
            got = c.to_canonical(out, 0, prec, nrhs=nrhs)
            for r in range(nrhs):
                want = oracle.hop_eo(c.U, c.half(psi, 1, r), c.dims, c.bc, 0, dagger=bool(dagger))
                assert rel(c.half(got, 0, r), want) < TOL[prec], (shape, dagger, r)
    finally:
        c.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_rhs_beyond_one_launch_chunk(prec):
    """33 right-hand sides: two launch chunks of the multi-RHS kernel (32 + 1)."""
    c = Case((4, 2, 4, 6), kappa=0.12, kind="haar", seed=23, bc=(1, 1, 1, -1))
    try:
        nrhs = 33
        psi = c.source(nrhs=nrhs, seed=81)
        inp = c.to_internal(psi, 1, prec)
        out = c.g.field(prec, nrhs)
        wilson.wilson_dslash(c.g.handle, out, inp, 0, 0, PRECS[prec], nrhs)
        got = c.to_canonical(out, 0, prec, nrhs=nrhs)
        for r in (0, 31, 32):
            want = oracle.hop_eo(c.U, c.half(psi, 1, r), c.dims, c.bc, 0)
            assert rel(c.half(got, 0, r), want) < TOL[prec], r
        a = torch.zeros(3 * nrhs, dtype=torch.float64, device="cuda")
        wilson.wl_cdot(c.g.handle, a, out, out, PRECS[prec], nrhs)
        n = a.cpu().numpy().reshape(nrhs, 3)[:, 2]
        for r in (0, 32):
            h = c.half(got, 0, r)
            assert abs(n[r] - oracle.cdot(h, h).real) < 1e-5 * n[r]
    finally:
        c.close()


@pytest.mark.parametrize("shape", [32, 64, 256, 1032, 1064, 1128])
def test_reducing_hop_shapes_in_solve(monkeypatch, shape):
    """Both forms of the reducing single-RHS hop (grid of resident blocks with
    a last-block sum; full grid with a finishing launch, shapes 1000 + block),
    down to the 32-thread blocks of small lattices, drive a solve to the true
    residual."""
    monkeypatch.setenv("WL_HOP_BLOCK", str(shape))
    c = Case((6, 2, 2, 6), kappa=0.124, kind="haar", seed=29, bc=(1, 1, 1, -1))
    try:
        b = c.source(nrhs=1, seed=91)
        for inner in (wilson.WL_F32, wilson.WL_F64):
            x = torch.zeros_like(b)
            rc, info = wilson.wilson_solve(c.g.handle, x, b, 1,
                                           wilson.solve_params(tol=1e-10, eo=True, inner=inner))
            tr = oracle.true_residual(c.U, b[0].cpu().numpy(), x[0].cpu().numpy(), c.dims, c.bc,
                                      c.kappa)
            assert tr <= 1e-10 and abs(info[0]["true_resid"] - tr) <= 0.05 * tr + 1e-15, (shape, inner)
    finally:
        c.close()


# ----------------------------------------------------------------------------
# FP64 on small lattices: three threads per site (launch shape 2000)
# ----------------------------------------------------------------------------

def _fp64_ops(monkeypatch, shape, dims, bc):
    """Hopping term (both parities and signs), D and M_ee (both signs) in FP64
    on a fresh gauge object whose hopping launches take `shape`."""
    monkeypatch.setenv("WL_HOP_BLOCK", str(shape))
    c = Case(dims, kappa=0.124, kind="haar", seed=41, bc=bc)
    try:
        psi = c.source(nrhs=1, seed=43)
        outs = []
        for dagger in (0, 1):
            for p in (0, 1):
                inp = c.to_internal(psi, 1 - p, "f64")
                out = c.g.field("f64", 1)
                wilson.wilson_dslash(c.g.handle, out, inp, p, dagger, wilson.WL_F64, 1)
                outs.append(("dslash", p, dagger, out.clone()))
            inp = full_internal(c, psi, "f64")
            out = torch.empty_like(inp)
            wilson.wilson_mult(c.g.handle, out, inp, 0, dagger, wilson.WL_F64, 1)
            outs.append(("D", 0, dagger, out.clone()))
            inp = c.to_internal(psi, 0, "f64")
            out = c.g.field("f64", 1)
            wilson.wilson_mult(c.g.handle, out, inp, 1, dagger, wilson.WL_F64, 1)
            outs.append(("Mee", 0, dagger, out.clone()))
        torch.cuda.synchronize()
        return c, psi, outs
    except Exception:
        c.close()
        raise


# Vh = 144 (ragged: 4.5 blocks of 32 sites), 288 and 128
@pytest.mark.parametrize("dims", [(6, 4, 2, 6), (6, 4, 4, 6), (4, 4, 4, 4)])
def test_fp64_rows_kernel_equals_one_thread_per_site(monkeypatch, dims):
    """The three-threads-per-site FP64 hop gives the one-thread-per-site
    kernel's result bit for bit (same operations per output component), and
    both match the oracle; so does the one-thread-per-site kernel in 32-thread
    blocks."""
    bc = (1, 1, 1, -1)
    c0, _, small = _fp64_ops(monkeypatch, 32, dims, bc)
    c0.close()
    c1, psi, ref = _fp64_ops(monkeypatch, 128, dims, bc)
    for (name, p, dagger, a), (_, _, _, b) in zip(ref, small):
        assert torch.equal(a, b), (name, p, dagger, "32-thread blocks")
    c1.close()
    c2, _, got = _fp64_ops(monkeypatch, 2000, dims, bc)
    try:
        for (name, p, dagger, a), (_, _, _, b) in zip(ref, got):
            assert torch.equal(a, b), (name, p, dagger)
        # and the oracle, for the hopping term of each parity
        for name, p, dagger, out in got:
            if name != "dslash":
                continue
            have = c2.half(c2.to_canonical(out, p, "f64"), p)
            want = oracle.hop_eo(c2.U, c2.half(psi, 1 - p), dims, bc, p, dagger=bool(dagger))
            assert rel(have, want) < TOL["f64"], (p, dagger)
    finally:
        c2.close()


def test_fp64_rows_kernel_in_solves(monkeypatch):
    """The reducing form of the three-threads-per-site hop drives the FP64
    full-D and even-odd solves to the oracle's true residual."""
    monkeypatch.setenv("WL_HOP_BLOCK", "2000")
    c = Case((6, 4, 4, 6), kappa=0.124, kind="haar", seed=47, bc=(1, 1, 1, -1))
    try:
        b = c.source(nrhs=1, seed=48)
        for eo in (False, True):
            x = torch.zeros_like(b)
            rc, info = wilson.wilson_solve(c.g.handle, x, b, 1,
                                           wilson.solve_params(tol=1e-10, eo=eo, inner=wilson.WL_F64))
            tr = oracle.true_residual(c.U, b[0].cpu().numpy(), x[0].cpu().numpy(), c.dims, c.bc, c.kappa)
            assert tr <= 1e-10 and abs(info[0]["true_resid"] - tr) <= 0.05 * tr + 1e-15, eo
    finally:
        c.close()


# ----------------------------------------------------------------------------
# FP16 error margins: the measured relative errors of every FP16 operator on
# every parity lattice, printed (pytest -s) and held against TOL["f16"]
# ----------------------------------------------------------------------------

def test_fp16_error_margins():
    """The largest FP16 relative error over the parity lattices, for the
    hopping term (both parities, both signs), D and M_ee, with Gaussian and
    with smooth links.  TOL["f16"] is set from these at a stated factor."""
    rows = []
    for (dims, bc) in SMALL + [((16, 16, 16, 16), (1, 1, 1, -1))]:
        for kind in ("haar", "smooth"):
            c = Case(dims, kappa=0.124, kind=kind, seed=7, bc=bc)
            try:
                psi = c.source(nrhs=2, seed=21)
                errs = {"dslash": 0.0, "D": 0.0, "Mee": 0.0}
                for dagger in (0, 1):
                    for p in (0, 1):
                        inp = c.to_internal(psi, 1 - p, "f16")
                        out = c.g.field("f16", 2)
                        wilson.wilson_dslash(c.g.handle, out, inp, p, dagger, wilson.WL_F16, 2)
                        got = c.to_canonical(out, p, "f16", nrhs=2)
                        for r in range(2):
                            want = oracle.hop_eo(c.U, c.half(psi, 1 - p, r), dims, bc, p, dagger=bool(dagger))
                            errs["dslash"] = max(errs["dslash"], rel(c.half(got, p, r), want))
                    inp = full_internal(c, psi, "f16")
                    out = torch.empty_like(inp)
                    wilson.wilson_mult(c.g.handle, out, inp, 0, dagger, wilson.WL_F16, 2)
                    got = full_canonical(c, out, "f16", 2).cpu().numpy()
                    for r in range(2):
                        want = oracle.D_full(c.U, psi[r].cpu().numpy(), dims, bc, c.kappa, dagger=bool(dagger))
                        errs["D"] = max(errs["D"], rel(got[r], want))
                    inp = c.to_internal(psi, 0, "f16")
                    out = c.g.field("f16", 2)
                    wilson.wilson_mult(c.g.handle, out, inp, 1, dagger, wilson.WL_F16, 2)
                    got = c.to_canonical(out, 0, "f16", nrhs=2)
                    for r in range(2):
                        want = oracle.Mee(c.U, c.half(psi, 0, r), dims, bc, c.kappa, dagger=bool(dagger))
                        errs["Mee"] = max(errs["Mee"], rel(c.half(got, 0, r), want))
                rows.append((dims, kind, errs))
            finally:
                c.close()
    print("\nFP16 relative L2 errors against the FP64 oracle (max over parities, signs, 2 RHS):")
    for dims, kind, e in rows:
        print(f"  {'x'.join(map(str, dims)):>12} {kind:>6}: dslash {e['dslash']:.3e}  D {e['D']:.3e}  "
              f"M_ee {e['Mee']:.3e}")
    worst = max(max(e.values()) for _, _, e in rows)
    print(f"  worst {worst:.3e}; TOL['f16'] = {TOL['f16']:.1e} ({TOL['f16'] / worst:.2f}x the worst)")
    assert worst <= TOL["f16"]
