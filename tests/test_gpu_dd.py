"""GPU parity of the domain-decomposed operator and solve (Sec. 4.4: pack the
spin-projected faces, exchange them, interior sweep while they move, then the
boundary) against the FP64 oracle on the undivided lattice.

Cuts along t, t x z and y x z x t; a block extent of 2 along the cut (every
site is a boundary site, and both faces of a block are one site apart); three
blocks along t (distinct forward and backward neighbours); a twisted boundary
phase on the cut direction.  Tolerances are those of the undivided operator
(gpu_helpers.TOL); solves must reach an oracle true residual <= 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import PRECS, TOL, rel
from paper_1811_00893_gb300 import fields, wilson

pytestmark = pytest.mark.gpu

TW = np.exp(0.7j)
CASES = [((4, 4, 4, 8), (1, 1, 1, 2), (1, 1, 1, -1)),       # t cut, 2 blocks
         ((6, 4, 4, 4), (1, 1, 1, 2), (1, 1, 1, TW)),       # block extent 2 on the cut, twisted t phase
         ((4, 4, 8, 8), (1, 1, 2, 2), (1, np.exp(0.2j), 1, -1)),  # t x z
         ((4, 4, 4, 8), (1, 2, 2, 2), (1, 1, TW, -1)),      # 8 blocks, y x z x t, extent 2 in y, z
         ((8, 4, 4, 12), (1, 1, 1, 3), (1, 1, 1, -1))]      # 3 blocks along t


class DDCase:
    def __init__(self, dims, grid, bc, kappa=0.124, seed=3, precs=("f64", "f32", "f16"), r12=False):
        self.dims, self.grid, self.bc, self.kappa = tuple(dims), tuple(grid), bc, kappa
        U = fields.gauge_field(dims, "haar", seed)
        self.U = U.numpy()
        self.U_dev = U.cuda().contiguous()
        self.dd = wilson.Decomposition(dims, kappa, self.U_dev, grid, precs=precs, bc=bc, r12=r12)
        self.V = int(np.prod(dims))

    def to_blocks(self, psi_dev, parity, prec):
        """Global canonical fields -> one internal half field per block."""
        nrhs = psi_dev.shape[0]
        loc = self.dd.canonical(nrhs)
        wilson.wl_dd_scatter(self.dd.handle, loc, psi_dev, nrhs)
        out = self.dd.field(prec, nrhs)
        for k, (g, _) in enumerate(self.dd.blocks):
            wilson.wl_field_to_internal(g, out[k], loc[k], parity, PRECS[prec], nrhs)
        return out

    def to_blocks_full(self, psi_dev, prec):
        """Global canonical fields -> one [even | odd] internal field per block."""
        nrhs = psi_dev.shape[0]
        loc = self.dd.canonical(nrhs)
        wilson.wl_dd_scatter(self.dd.handle, loc, psi_dev, nrhs)
        g0 = self.dd.blocks[0][0]
        fb = wilson.wl_field_bytes(g0, PRECS[prec], 1)
        out = self.dd.field(prec, nrhs, nhalf=2)
        for k, (g, _) in enumerate(self.dd.blocks):
            for r in range(nrhs):
                for p in (0, 1):
                    seg = out[k][(2 * r + p) * fb:(2 * r + p + 1) * fb]
                    wilson.wl_field_to_internal(g, seg, loc[k][r:r + 1], p, PRECS[prec], 1)
        return out

    def from_blocks(self, fields_, parity, prec, nrhs):
        loc = self.dd.canonical(nrhs)
        for k, (g, _) in enumerate(self.dd.blocks):
            wilson.wl_field_to_canonical(g, loc[k], fields_[k], parity, PRECS[prec], nrhs)
        out = torch.zeros((nrhs, self.V, 4, 3), dtype=torch.complex128, device="cuda")
        wilson.wl_dd_gather(self.dd.handle, out, loc, nrhs)
        return out

    def from_blocks_full(self, fields_, prec, nrhs):
        g0 = self.dd.blocks[0][0]
        fb = wilson.wl_field_bytes(g0, PRECS[prec], 1)
        loc = self.dd.canonical(nrhs)
        for k, (g, _) in enumerate(self.dd.blocks):
            for r in range(nrhs):
                for p in (0, 1):
                    seg = fields_[k][(2 * r + p) * fb:(2 * r + p + 1) * fb]
                    wilson.wl_field_to_canonical(g, loc[k][r:r + 1], seg, p, PRECS[prec], 1)
        out = torch.zeros((nrhs, self.V, 4, 3), dtype=torch.complex128, device="cuda")
        wilson.wl_dd_gather(self.dd.handle, out, loc, nrhs)
        return out

    def half(self, canon, parity, r=0):
        e, o = oracle.split(canon[r].cpu().numpy(), self.dims)
        return e if parity == 0 else o

    def close(self):
        self.dd.close()


@pytest.fixture(scope="module", params=CASES,
                ids=lambda c: "x".join(map(str, c[0])) + "-g" + "".join(map(str, c[1])))
def ddc(request):
    dims, grid, bc = request.param
    c = DDCase(dims, grid, bc)
    yield c
    c.close()


def test_scatter_gather_round_trip(ddc):
    psi = fields.gaussian_fermion(ddc.dims, 2, 5).cuda()
    loc = ddc.dd.canonical(2)
    wilson.wl_dd_scatter(ddc.dd.handle, loc, psi, 2)
    back = torch.zeros_like(psi)
    wilson.wl_dd_gather(ddc.dd.handle, back, loc, 2)
    torch.cuda.synchronize()
    assert torch.equal(back, psi)
    # block 0 holds the sites of the first block of the grid
    L = ddc.dd.local_dims
    want = psi[0].reshape(ddc.dims[::-1] + (4, 3))[:L[3], :L[2], :L[1], :L[0]].reshape(-1, 4, 3)
    assert torch.equal(loc[0][0], want)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_dslash_dd_matches_oracle(ddc, prec, dagger):
    nrhs = 2
    psi = fields.gaussian_fermion(ddc.dims, nrhs, 21).cuda()
    for out_parity in (0, 1):
        inp = ddc.to_blocks(psi, 1 - out_parity, prec)
        out = ddc.dd.field(prec, nrhs)
        wilson.wilson_dslash_dd(ddc.dd.handle, out, inp, out_parity, dagger, PRECS[prec], nrhs)
        got = ddc.from_blocks(out, out_parity, prec, nrhs)
        for r in range(nrhs):
            want = oracle.hop_eo(ddc.U, ddc.half(psi, 1 - out_parity, r), ddc.dims, ddc.bc, out_parity,
                                 dagger=bool(dagger))
            err = rel(ddc.half(got, out_parity, r), want)
            assert err <= TOL[prec], (prec, dagger, out_parity, r, err)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
def test_dslash_dd_equals_undivided(ddc, prec):
    """Every site is computed once with the operations of the undivided
    kernel and the halo carries exactly the half spinor that kernel forms, so
    the decomposed result is bit for bit the undivided one."""
    nrhs = 1
    psi = fields.gaussian_fermion(ddc.dims, nrhs, 23).cuda()
    g = wilson.Gauge(ddc.dims, ddc.kappa, ddc.U_dev, precs=("f64", "f32", "f16"), bc=ddc.bc)
    try:
        inp = g.field(prec, nrhs)
        wilson.wl_field_to_internal(g.handle, inp, psi, 1, PRECS[prec], nrhs)
        out = g.field(prec, nrhs)
        wilson.wilson_dslash(g.handle, out, inp, 0, 0, PRECS[prec], nrhs)
        ref = torch.zeros((nrhs, ddc.V, 4, 3), dtype=torch.complex128, device="cuda")
        wilson.wl_field_to_canonical(g.handle, ref, out, 0, PRECS[prec], nrhs)
        dout = ddc.dd.field(prec, nrhs)
        wilson.wilson_dslash_dd(ddc.dd.handle, dout, ddc.to_blocks(psi, 1, prec), 0, 0, PRECS[prec], nrhs)
        got = ddc.from_blocks(dout, 0, prec, nrhs)
        assert torch.equal(got, ref), rel(ddc.half(got, 0), ddc.half(ref, 0))
    finally:
        g.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_mult_dd_matches_oracle(ddc, prec, dagger):
    nrhs = 2
    psi = fields.gaussian_fermion(ddc.dims, nrhs, 31).cuda()
    # eo = 1: M_ee on even half fields
    inp = ddc.to_blocks(psi, 0, prec)
    out = ddc.dd.field(prec, nrhs)
    wilson.wilson_mult_dd(ddc.dd.handle, out, inp, 1, dagger, PRECS[prec], nrhs)
    got = ddc.from_blocks(out, 0, prec, nrhs)
    for r in range(nrhs):
        want = oracle.Mee(ddc.U, ddc.half(psi, 0, r), ddc.dims, ddc.bc, ddc.kappa, dagger=bool(dagger))
        err = rel(ddc.half(got, 0, r), want)
        assert err <= TOL[prec], ("Mee", prec, dagger, r, err)
    # eo = 0: full D on [even | odd] fields
    inp = ddc.to_blocks_full(psi, prec)
    out = ddc.dd.field(prec, nrhs, nhalf=2)
    wilson.wilson_mult_dd(ddc.dd.handle, out, inp, 0, dagger, PRECS[prec], nrhs)
    got = ddc.from_blocks_full(out, prec, nrhs)
    for r in range(nrhs):
        want = oracle.D_full(ddc.U, psi[r].cpu().numpy(), ddc.dims, ddc.bc, ddc.kappa, dagger=bool(dagger))
        err = rel(got[r].cpu().numpy(), want)
        assert err <= TOL[prec], ("D", prec, dagger, r, err)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cdot_dd_is_the_global_sum(ddc, prec):
    nrhs = 3
    a = fields.gaussian_fermion(ddc.dims, nrhs, 41).cuda()
    b = fields.gaussian_fermion(ddc.dims, nrhs, 42).cuda()
    ia, ib = ddc.to_blocks(a, 0, prec), ddc.to_blocks(b, 0, prec)
    out = torch.zeros(3 * nrhs, dtype=torch.float64, device="cuda")
    wilson.wl_cdot_dd(ddc.dd.handle, out, ia, ib, PRECS[prec], nrhs)
    # the oracle on the stored (rounded) fields gathered back
    ga, gb = ddc.from_blocks(ia, 0, prec, nrhs), ddc.from_blocks(ib, 0, prec, nrhs)
    o = out.view(nrhs, 3).cpu().numpy()
    # per-site products in the storage type's arithmetic (2^-24 relative per
    # term in FP32), sums in FP64
    tol = {"f64": 1e-12, "f32": 1e-6}[prec]
    for r in range(nrhs):
        ea, eb = ddc.half(ga, 0, r), ddc.half(gb, 0, r)
        c = oracle.cdot(ea, eb)
        n2 = oracle.cdot(eb, eb).real
        scale = np.sqrt(n2 * oracle.cdot(ea, ea).real)
        assert abs(o[r, 0] - c.real) <= tol * scale
        assert abs(o[r, 1] - c.imag) <= tol * scale
        assert abs(o[r, 2] - n2) <= tol * n2


@pytest.mark.parametrize("inner,delta", [("f32", 0.0), ("f64", 0.0), ("f16", 0.003)],
                         ids=["f32-defect-correction", "f64", "f16-reliable"])
def test_solve_dd_reaches_oracle_residual(ddc, inner, delta):
    nrhs = 2
    b = fields.gaussian_fermion(ddc.dims, nrhs, 51).cuda()
    bl = ddc.dd.canonical(nrhs)
    wilson.wl_dd_scatter(ddc.dd.handle, bl, b, nrhs)
    xl = ddc.dd.canonical(nrhs)
    prm = wilson.solve_params(tol=1e-10, eo=True, inner=PRECS[inner], delta=delta)
    rc, info = wilson.wilson_solve_dd(ddc.dd.handle, xl, bl, nrhs, prm)
    x = torch.zeros_like(b)
    wilson.wl_dd_gather(ddc.dd.handle, x, xl, nrhs)
    for r in range(nrhs):
        tr = oracle.true_residual(ddc.U, b[r].cpu().numpy(), x[r].cpu().numpy(), ddc.dims, ddc.bc, ddc.kappa)
        assert tr <= 1e-10, (inner, r, tr, info[r])
        assert info[r]["status"] == 0 and info[r]["true_resid"] <= 1e-10


def test_solve_dd_iterations_match_undivided():
    """The decomposed FP64 solve takes the undivided solve's iterations (the
    same Krylov sequence up to the summation order of the global sums)."""
    c = DDCase((4, 4, 4, 8), (1, 1, 1, 2), (1, 1, 1, -1))
    g = wilson.Gauge(c.dims, c.kappa, c.U_dev, precs=("f64",), bc=c.bc)
    try:
        b = fields.gaussian_fermion(c.dims, 1, 61).cuda()
        prm = wilson.solve_params(tol=1e-10, eo=True, inner=wilson.WL_F64)
        x = torch.zeros_like(b)
        _, ref = wilson.wilson_solve(g.handle, x, b, 1, prm)
        bl = c.dd.canonical(1)
        wilson.wl_dd_scatter(c.dd.handle, bl, b, 1)
        xl = c.dd.canonical(1)
        _, got = wilson.wilson_solve_dd(c.dd.handle, xl, bl, 1, prm)
        assert abs(got[0]["iters"] - ref[0]["iters"]) <= 1, (got, ref)
    finally:
        g.close()
        c.close()


@pytest.mark.parametrize("mode", [0, 1], ids=["copy", "direct"])
def test_exchange_modes_agree(mode):
    c = DDCase((4, 4, 8, 8), (1, 1, 2, 2), (1, 1, 1, -1))
    try:
        wilson.wl_dd_set_exchange(c.dd.handle, mode)
        psi = fields.gaussian_fermion(c.dims, 1, 71).cuda()
        inp = c.to_blocks(psi, 0, "f32")
        out = c.dd.field("f32", 1)
        wilson.wilson_mult_dd(c.dd.handle, out, inp, 1, 0, wilson.WL_F32, 1)
        got = c.from_blocks(out, 0, "f32", 1)
        want = oracle.Mee(c.U, c.half(psi, 0), c.dims, c.bc, c.kappa)
        assert rel(c.half(got, 0), want) <= TOL["f32"]
    finally:
        c.close()


def test_dd_compressed_links():
    c = DDCase((6, 4, 4, 8), (1, 1, 2, 2), (1, 1, np.exp(0.4j), TW), precs=("f64", "f32", "f16"), r12=True)
    try:
        psi = fields.gaussian_fermion(c.dims, 1, 81).cuda()
        for prec in ("f32", "f16"):
            for dagger in (0, 1):
                inp = c.to_blocks(psi, 1, prec)
                out = c.dd.field(prec, 1)
                wilson.wilson_dslash_dd(c.dd.handle, out, inp, 0, dagger, PRECS[prec], 1)
                got = c.from_blocks(out, 0, prec, 1)
                want = oracle.hop_eo(c.U, c.half(psi, 1), c.dims, c.bc, 0, dagger=bool(dagger))
                assert rel(c.half(got, 0), want) <= TOL[prec], (prec, dagger)
    finally:
        c.close()


def test_dd_errors():
    U = fields.gauge_field((4, 4, 4, 8), "haar", 1).cuda()
    lat = wilson.lattice((4, 4, 4, 8), 0.12)
    for grid in [(2, 1, 1, 1), (1, 1, 1, 3), (1, 1, 1, 8), (1, 4, 4, 1)]:
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wl_dd_create(lat, grid, U, wilson.prec_mask("f64"))
        assert e.value.code == wilson.WL_ERR_ARG, grid
    with wilson.Decomposition((4, 4, 4, 8), 0.12, U, (1, 1, 1, 2), precs=("f64",)) as dd:
        g = dd.blocks[0][0]
        f = dd.field("f64", 1)
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wilson_dslash(g, f[0], f[1], 0, 0, wilson.WL_F64, 1)
        assert e.value.code == wilson.WL_ERR_STATE
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wilson_dslash_dd(dd.handle, f, f, 0, 0, wilson.WL_F32, 1)
        assert e.value.code == wilson.WL_ERR_STATE  # no FP32 links


# ----------------------------------------------------------------------------
# the clover term (Eq. 2) on the decomposed lattice
# ----------------------------------------------------------------------------

CLOVER_CASES = [((4, 4, 4, 8), (1, 1, 1, 2), (1, 1, 1, -1)),
                ((4, 4, 8, 8), (1, 1, 2, 2), (1, np.exp(0.2j), 1, TW))]


@pytest.fixture(scope="module", params=CLOVER_CASES,
                ids=lambda c: "x".join(map(str, c[0])) + "-g" + "".join(map(str, c[1])))
def cdd(request):
    dims, grid, bc = request.param
    c = DDCase(dims, grid, bc)
    c.F = fields.clover_field(dims, 57).numpy()
    c.F_dev = torch.from_numpy(c.F).cuda().contiguous()
    wilson.wl_dd_clover_set(c.dd.handle, c.F_dev)
    c.g = wilson.Gauge(dims, c.kappa, c.U_dev, precs=("f64", "f32", "f16"), bc=bc)
    wilson.wl_clover_set(c.g.handle, c.F_dev)
    yield c
    c.g.close()
    c.close()


def _full_internal(g, psi, prec):
    nrhs = psi.shape[0]
    fb = wilson.wl_field_bytes(g.handle, PRECS[prec], 1)
    out = torch.empty(2 * fb * nrhs, dtype=torch.uint8, device="cuda")
    for r in range(nrhs):
        for p in (0, 1):
            wilson.wl_field_to_internal(g.handle, out[(2 * r + p) * fb:(2 * r + p + 1) * fb], psi[r:r + 1], p,
                                        PRECS[prec], 1)
    return out, fb


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_clover_mult_dd_equals_undivided(cdd, prec, dagger):
    """M_ee = A_ee - kappa^2 H_eo A_oo^-1 H_oe and D_clov on the decomposed
    lattice run the undivided operator's fused clover epilogues on every
    site: bit for bit the undivided results (which the clover tests hold
    against the oracle); M_ee also against the oracle here."""
    nrhs = 1
    psi = fields.gaussian_fermion(cdd.dims, nrhs, 33).cuda()
    g = cdd.g
    inp = g.field(prec, nrhs)
    wilson.wl_field_to_internal(g.handle, inp, psi, 0, PRECS[prec], nrhs)
    out = g.field(prec, nrhs)
    wilson.wilson_mult(g.handle, out, inp, 1, dagger, PRECS[prec], nrhs)
    ref = torch.zeros((nrhs, cdd.V, 4, 3), dtype=torch.complex128, device="cuda")
    wilson.wl_field_to_canonical(g.handle, ref, out, 0, PRECS[prec], nrhs)
    dout = cdd.dd.field(prec, nrhs)
    wilson.wilson_mult_dd(cdd.dd.handle, dout, cdd.to_blocks(psi, 0, prec), 1, dagger, PRECS[prec], nrhs)
    got = cdd.from_blocks(dout, 0, prec, nrhs)
    assert torch.equal(got, ref), ("Mee", rel(cdd.half(got, 0), cdd.half(ref, 0)))
    if dagger == 0:
        want = oracle.clover_Mee(cdd.U, cdd.F, cdd.half(psi, 0), cdd.dims, cdd.bc, cdd.kappa)
        assert rel(cdd.half(got, 0), want) <= TOL[prec]
    # eo = 0: D_clov on [even | odd] fields
    inp, fb = _full_internal(g, psi, prec)
    out = torch.empty_like(inp)
    wilson.wilson_mult(g.handle, out, inp, 0, dagger, PRECS[prec], nrhs)
    ref = torch.zeros((nrhs, cdd.V, 4, 3), dtype=torch.complex128, device="cuda")
    for p in (0, 1):
        wilson.wl_field_to_canonical(g.handle, ref, out[p * fb:(p + 1) * fb], p, PRECS[prec], 1)
    dout = cdd.dd.field(prec, nrhs, nhalf=2)
    wilson.wilson_mult_dd(cdd.dd.handle, dout, cdd.to_blocks_full(psi, prec), 0, dagger, PRECS[prec], nrhs)
    got = cdd.from_blocks_full(dout, prec, nrhs)
    assert torch.equal(got, ref), ("D", rel(got[0].cpu().numpy(), ref[0].cpu().numpy()))


@pytest.mark.parametrize("inner,delta", [("f32", 0.0), ("f64", 0.0), ("f16", 0.003)],
                         ids=["f32-defect-correction", "f64", "f16-reliable"])
def test_clover_solve_dd_reaches_oracle_residual(cdd, inner, delta):
    nrhs = 2
    b = fields.gaussian_fermion(cdd.dims, nrhs, 53).cuda()
    bl = cdd.dd.canonical(nrhs)
    wilson.wl_dd_scatter(cdd.dd.handle, bl, b, nrhs)
    xl = cdd.dd.canonical(nrhs)
    prm = wilson.solve_params(tol=1e-10, eo=True, inner=PRECS[inner], delta=delta)
    rc, info = wilson.wilson_solve_dd(cdd.dd.handle, xl, bl, nrhs, prm)
    x = torch.zeros_like(b)
    wilson.wl_dd_gather(cdd.dd.handle, x, xl, nrhs)
    for r in range(nrhs):
        tr = oracle.clover_true_residual(cdd.U, cdd.F, b[r].cpu().numpy(), x[r].cpu().numpy(), cdd.dims, cdd.bc,
                                         cdd.kappa)
        assert tr <= 1e-10, (inner, r, tr, info[r])
        assert info[r]["status"] == 0 and info[r]["true_resid"] <= 1e-10


def test_clover_set_dd_errors_leave_no_term():
    c = DDCase((4, 4, 4, 8), (1, 1, 1, 2), (1, 1, 1, -1))
    try:
        F = fields.clover_field(c.dims, 5).numpy()
        F[3, 0, 1, 2] += 0.5  # no longer Hermitian
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wl_dd_clover_set(c.dd.handle, torch.from_numpy(F).cuda().contiguous())
        assert e.value.code == wilson.WL_ERR_ARG
        psi = fields.gaussian_fermion(c.dims, 1, 7).cuda()
        got = _mee_blocks(c, psi, "f64")  # the Wilson operator: no block kept a term
        want = oracle.Mee(c.U, c.half(psi, 0), c.dims, c.bc, c.kappa)
        assert rel(c.half(got, 0), want) <= TOL["f64"]
        g = c.dd.blocks[0][0]
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wl_clover_set(g, torch.from_numpy(F).cuda().contiguous())
        assert e.value.code == wilson.WL_ERR_STATE  # blocks take the term through the decomposition
        # a valid term, then detached again: back to the Wilson operator
        Fok = fields.clover_field(c.dims, 6).cuda().contiguous()
        wilson.wl_dd_clover_set(c.dd.handle, Fok)
        with_term = _mee_blocks(c, psi, "f64")
        want_c = oracle.clover_Mee(c.U, Fok.cpu().numpy(), c.half(psi, 0), c.dims, c.bc, c.kappa)
        assert rel(c.half(with_term, 0), want_c) <= TOL["f64"]
        wilson.wl_dd_clover_set(c.dd.handle, None)
        got = _mee_blocks(c, psi, "f64")
        assert rel(c.half(got, 0), want) <= TOL["f64"]
    finally:
        c.close()


# ----------------------------------------------------------------------------
# the transport path: faces and sums through wl_dd_transport callbacks
# ----------------------------------------------------------------------------

def _mee_blocks(c, psi, prec="f32"):
    inp = c.to_blocks(psi, 0, prec)
    out = c.dd.field(prec, psi.shape[0])
    wilson.wilson_mult_dd(c.dd.handle, out, inp, 1, 0, PRECS[prec], psi.shape[0])
    return c.from_blocks(out, 0, prec, psi.shape[0])


def test_transport_callbacks_match_device_copies():
    """Every face of a one-process decomposition routed through the Python
    transport gives the built-in copies' results bit for bit."""
    from paper_1811_00893_gb300 import dd_transport
    dims, grid, bc = (4, 4, 8, 8), (1, 1, 2, 2), (1, 1, 1, -1)
    ref = DDCase(dims, grid, bc)
    tr = dd_transport.TorchTransport(rank_of=lambda b: 0, rank=0, route_all=True)
    c = DDCase(dims, grid, bc)
    c.dd.close()
    c.dd = wilson.Decomposition(dims, c.kappa, c.U_dev, grid, bc=bc, transport=tr)
    try:
        psi = fields.gaussian_fermion(dims, 2, 91).cuda()
        for prec in ("f64", "f32", "f16"):
            assert torch.equal(_mee_blocks(c, psi, prec), _mee_blocks(ref, psi, prec)), prec
        assert tr.calls["exchange"] >= 6
        b = fields.gaussian_fermion(dims, 1, 92).cuda()
        bl = c.dd.canonical(1)
        wilson.wl_dd_scatter(c.dd.handle, bl, b, 1)
        xl = c.dd.canonical(1)
        rc, info = wilson.wilson_solve_dd(c.dd.handle, xl, bl, 1, wilson.solve_params(tol=1e-10, inner=wilson.WL_F32))
        x = torch.zeros_like(b)
        wilson.wl_dd_gather(c.dd.handle, x, xl, 1)
        assert oracle.true_residual(c.U, b[0].cpu().numpy(), x[0].cpu().numpy(), dims, bc, c.kappa) <= 1e-10
        assert tr.calls["allreduce"] > 0
    finally:
        c.close()
        ref.close()


class ThreadTransport:
    """Two holders of blocks in one process, one per host thread, sharing one
    GPU: faces and sums meet in a host-side mailbox.  Every transfer is
    host-synchronised (the sender's stream is synchronised before its face is
    posted, the receiver copies and synchronises before acknowledging), so no
    kernel ever waits on another holder's work."""

    def __init__(self, holders: int):
        import threading
        self.cv = threading.Condition()
        self.box = {}
        self.acks = {}
        self.sums = {}
        self.round = 0
        self.holders = holders

    def for_holder(self, rank, rank_of):
        from paper_1811_00893_gb300 import dd_transport
        outer = self

        class Holder(dd_transport.TorchTransport):
            def exchange(self, msgs):
                self.calls["exchange"] += 1
                torch.cuda.current_stream().synchronize()
                with outer.cv:
                    for m in msgs:
                        if m["send"]:
                            outer.box[m["tag"]] = m["buf"]
                    outer.cv.notify_all()
                for m in msgs:
                    if not m["send"]:
                        with outer.cv:
                            outer.cv.wait_for(lambda: m["tag"] in outer.box, timeout=60)
                            src = outer.box.pop(m["tag"])
                        m["buf"].copy_(src)
                torch.cuda.current_stream().synchronize()
                with outer.cv:
                    for m in msgs:
                        if not m["send"]:
                            outer.acks[m["tag"]] = True
                    outer.cv.notify_all()
                    for m in msgs:  # our faces have been read: the buffer may be reused
                        if m["send"]:
                            outer.cv.wait_for(lambda: m["tag"] in outer.acks, timeout=60)
                            outer.acks.pop(m["tag"])

            def allreduce(self, t):
                self.calls["allreduce"] += 1
                val = t.cpu()
                with outer.cv:
                    r = outer.round
                    outer.sums.setdefault(r, []).append(val)
                    if len(outer.sums[r]) == outer.holders:
                        outer.round += 1
                        outer.cv.notify_all()
                    else:
                        outer.cv.wait_for(lambda: outer.round > r, timeout=60)
                    vals = outer.sums[r]
                total = vals[0].clone()
                for v in vals[1:]:
                    total += v
                t.copy_(total.to(t.device))
                torch.cuda.current_stream().synchronize()

        return Holder(rank_of=rank_of, rank=rank)


def test_two_holders_reach_the_undivided_results():
    """A t-cut lattice whose two blocks are held by two holders (threads), as
    two processes would hold them: the decomposed M_ee and an FP32
    defect-correction solve through the transport callbacks."""
    import threading
    dims, grid, bc, kappa = (4, 4, 4, 8), (1, 1, 1, 2), (1, 1, 1, -1), 0.124
    U = fields.gauge_field(dims, "haar", 3)
    Un, Ud = U.numpy(), U.cuda()
    psi = fields.gaussian_fermion(dims, 1, 93).cuda()
    ref = DDCase(dims, grid, bc)
    want = _mee_blocks(ref, psi)
    ref.close()
    tt = ThreadTransport(2)
    results, errors = {}, []

    def holder(rank):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                tr = tt.for_holder(rank, rank_of=lambda b: b)
                dd = wilson.Decomposition(dims, kappa, Ud, grid, bc=bc, held=(rank, 1), transport=tr)
                loc = dd.canonical(1)
                wilson.wl_dd_scatter(dd.handle, loc, psi, 1)
                g = dd.blocks[0][0]
                inp = dd.field("f32", 1)
                wilson.wl_field_to_internal(g, inp[0], loc[0], 0, wilson.WL_F32, 1)
                out = dd.field("f32", 1)
                wilson.wilson_mult_dd(dd.handle, out, inp, 1, 0, wilson.WL_F32, 1)
                back = dd.canonical(1)
                wilson.wl_field_to_canonical(g, back[0], out[0], 0, wilson.WL_F32, 1)
                mee = torch.zeros_like(psi)
                wilson.wl_dd_gather(dd.handle, mee, back, 1)
                xl = dd.canonical(1)
                rc, info = wilson.wilson_solve_dd(dd.handle, xl, loc, 1,
                                                  wilson.solve_params(tol=1e-10, inner=wilson.WL_F32))
                x = torch.zeros_like(psi)
                wilson.wl_dd_gather(dd.handle, x, xl, 1)
                stream.synchronize()
                results[rank] = (mee, x, info[0], tr.calls)
                dd.close()
        except Exception as e:  # reported by the main thread
            errors.append(repr(e))

    ths = [threading.Thread(target=holder, args=(r,)) for r in range(2)]
    for t in ths:
        t.start()
    for t in ths:
        t.join(timeout=600)
    assert not errors, errors
    mee = results[0][0] + results[1][0]  # each holder gathered its own block's sites
    assert torch.equal(mee, want)
    x = results[0][1] + results[1][1]
    assert oracle.true_residual(Un, psi[0].cpu().numpy(), x[0].cpu().numpy(), dims, bc, kappa) <= 1e-10
    assert results[0][2]["iters"] == results[1][2]["iters"]
    assert results[0][3]["allreduce"] > 0 and results[0][3]["exchange"] > 0
