"""GPU parity of the eight-real link format (WL_LINKS_R8).

With the flag, single-RHS FP32 Wilson hopping launches read eight reals per
hop matrix and rebuild the rest from unitarity and det 1 (hop.cuh
load_link_r8), with the boundary phases on the fly.  Results must match the
FP64 oracle to the FP32 tolerance: the rebuilt entries carry FP32 rounding,
and entries near zero an absolute error of about its square root, which
enters the relative L2 error only at the few sites where such an entry sits.
Haar, smooth and unit links (where U_00 = 1 forces the shifted row order),
twisted complex phases and L = 2 extents are covered.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import TOL, Case, rel
from paper_1811_00893_gb300 import fields, wilson

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 4), (1, 1, 1, -1), "haar"),
         ((6, 4, 2, 8), (np.exp(0.4j), np.exp(0.3j), 1, -1), "haar"),  # complex phases, L = 2, ragged
         ((2, 2, 2, 2), (1, np.exp(-0.7j), 1, -1), "haar"),            # L = 2 everywhere
         ((8, 6, 4, 10), (1, 1, 1, -1), "smooth"),
         ((4, 4, 4, 8), (1, 1, 1, -1), "unit")]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])) + "-" + c[2])
def case(request):
    dims, bc, kind = request.param
    c = Case(dims, kappa=0.124, kind=kind, seed=23, bc=bc, precs=("f64", "f32"), r8=True)
    yield c
    c.close()


@pytest.mark.parametrize("dagger", [0, 1])
def test_r8_dslash_matches_oracle(case, dagger):
    psi = case.source(nrhs=1, seed=21)
    for out_parity in (0, 1):
        inp = case.to_internal(psi, 1 - out_parity, "f32")
        out = case.g.field("f32", 1)
        wilson.wilson_dslash(case.g.handle, out, inp, out_parity, dagger, wilson.WL_F32, 1)
        got = case.to_canonical(out, out_parity, "f32")
        want = oracle.hop_eo(case.U, case.half(psi, 1 - out_parity), case.dims, case.bc, out_parity,
                             dagger=bool(dagger))
        assert rel(case.half(got, out_parity), want) < TOL["f32"], (out_parity, dagger)


def test_r8_D_and_Mee_match_oracle(case):
    psi = case.source(nrhs=1, seed=41)
    inp = case.to_internal(psi, 0, "f32")
    out = case.g.field("f32", 1)
    wilson.wilson_mult(case.g.handle, out, inp, 1, 0, wilson.WL_F32, 1)
    got = case.to_canonical(out, 0, "f32")
    want = oracle.Mee(case.U, case.half(psi, 0), case.dims, case.bc, case.kappa)
    assert rel(case.half(got, 0), want) < TOL["f32"]
    fb = wilson.wl_field_bytes(case.g.handle, wilson.WL_F32, 1)
    full = torch.empty(2 * fb, dtype=torch.uint8, device="cuda")
    for p in (0, 1):
        wilson.wl_field_to_internal(case.g.handle, full[p * fb:(p + 1) * fb], psi, p, wilson.WL_F32, 1)
    outf = torch.empty_like(full)
    wilson.wilson_mult(case.g.handle, outf, full, 0, 1, wilson.WL_F32, 1)
    gotf = torch.zeros_like(psi)
    for p in (0, 1):
        wilson.wl_field_to_canonical(case.g.handle, gotf, outf[p * fb:(p + 1) * fb], p, wilson.WL_F32, 1)
    wantf = oracle.D_full(case.U, psi[0].cpu().numpy(), case.dims, case.bc, case.kappa, dagger=True)
    assert rel(gotf[0].cpu().numpy(), wantf) < TOL["f32"]


def test_r8_multi_rhs_launches_use_full_links(case):
    """Multi-RHS launches on a gauge object with eight-real links take the
    full links (the eight-real form is for single-RHS Wilson launches only)
    and match the oracle."""
    nrhs = 3
    psi = case.source(nrhs=nrhs, seed=27)
    inp = case.to_internal(psi, 1, "f32")
    out = case.g.field("f32", nrhs)
    wilson.wilson_dslash(case.g.handle, out, inp, 0, 0, wilson.WL_F32, nrhs)
    got = case.to_canonical(out, 0, "f32", nrhs=nrhs)
    for r in range(nrhs):
        want = oracle.hop_eo(case.U, case.half(psi, 1, r), case.dims, case.bc, 0)
        assert rel(case.half(got, 0, r), want) < TOL["f32"], r


def test_r8_solve_reaches_true_residual(case):
    b = case.source(nrhs=1, seed=61)
    x = torch.zeros_like(b)
    rc, info = wilson.wilson_solve(case.g.handle, x, b, 1, wilson.solve_params(tol=1e-10, eo=True, inner=wilson.WL_F32))
    tr = oracle.true_residual(case.U, b[0].cpu().numpy(), x[0].cpu().numpy(), case.dims, case.bc, case.kappa)
    assert tr <= 1e-10 and info[0]["status"] == 0, (tr, info[0])


def test_r8_equals_full_links_within_rounding():
    """At 16^4 with Haar links the eight-real hop stays within FP32 rounding of
    the full-link hop in relative L2 (the sqrt-of-rounding error of entries
    near zero is confined to a few sites)."""
    dims = (16, 16, 16, 16)
    U = fields.gauge_field(dims, "haar", 29).cuda()
    psi = fields.gaussian_fermion(dims, 1, 31).cuda()
    outs = []
    for r8 in (False, True):
        g = wilson.Gauge(dims, 0.12, U, precs=("f64", "f32"), r8=r8)
        try:
            fb = wilson.wl_field_bytes(g.handle, wilson.WL_F32, 1)
            inp = torch.empty(fb, dtype=torch.uint8, device="cuda")
            wilson.wl_field_to_internal(g.handle, inp, psi, 1, wilson.WL_F32, 1)
            out = torch.empty_like(inp)
            wilson.wilson_dslash(g.handle, out, inp, 0, 0, wilson.WL_F32, 1)
            c = torch.zeros_like(psi)
            wilson.wl_field_to_canonical(g.handle, c, out, 0, wilson.WL_F32, 1)
            outs.append(c)
        finally:
            g.close()
    d = (outs[1] - outs[0]).abs().pow(2).sum().sqrt() / outs[0].abs().pow(2).sum().sqrt()
    assert float(d) < 2e-6, float(d)


def test_r8_rejects_non_su3_links():
    dims = (4, 4, 4, 4)
    U = fields.gauge_field(dims, "haar", 3) * np.exp(0.1j)  # U(3), det != 1
    with pytest.raises(wilson.WilsonError) as e:
        wilson.Gauge(dims, 0.12, U.to("cuda").contiguous(), precs=("f64", "f32"), r8=True)
    assert e.value.code == wilson.WL_ERR_ARG
