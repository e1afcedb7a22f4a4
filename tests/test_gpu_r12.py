"""GPU parity of the compressed-link hopping kernels (WL_LINKS_R12).

With the flag the FP32 / FP16 hopping kernels read two rows of each SU(3)
link and rebuild the third from unitarity, and apply the boundary phases on
the fly; results must match the FP64 oracle to the same tolerances as the full
links (FP32 1e-5: the rebuilt row carries FP32 rounding, ~1e-7; FP16 7e-4).
Twisted complex phases and L = 2 extents exercise the on-the-fly phases.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import PRECS, TOL, Case, rel
from paper_1811_00893_gb300 import fields, wilson

pytestmark = pytest.mark.gpu

SMALL = [((4, 4, 4, 4), (1, 1, 1, -1)),
         ((6, 4, 2, 8), (np.exp(0.4j), np.exp(0.3j), 1, -1)),  # complex phases, L = 2, ragged
         ((2, 2, 2, 2), (1, np.exp(-0.7j), 1, -1)),            # L = 2 everywhere
         ((8, 6, 4, 10), (1, 1, 1, -1))]


@pytest.fixture(scope="module", params=SMALL, ids=lambda c: "x".join(map(str, c[0])))
def case(request):
    dims, bc = request.param
    c = Case(dims, kappa=0.124, kind="haar", seed=17, bc=bc, precs=("f64", "f32", "f16"), r12=True)
    yield c
    c.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_r12_dslash_matches_oracle(case, prec, dagger, nrhs):
    psi = case.source(nrhs=nrhs, seed=21)
    for out_parity in (0, 1):
        inp = case.to_internal(psi, 1 - out_parity, prec)
        out = case.g.field(prec, nrhs)
        wilson.wilson_dslash(case.g.handle, out, inp, out_parity, dagger, PRECS[prec], nrhs)
        got = case.to_canonical(out, out_parity, prec, nrhs=nrhs)
        for r in range(nrhs):
            want = oracle.hop_eo(case.U, case.half(psi, 1 - out_parity, r), case.dims, case.bc,
                                 out_parity, dagger=bool(dagger))
            assert rel(case.half(got, out_parity, r), want) < TOL[prec], (prec, out_parity, r)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_r12_Mee_matches_oracle(case, prec):
    nrhs = 2
    psi = case.source(nrhs=nrhs, seed=41)
    inp = case.to_internal(psi, 0, prec)
    out = case.g.field(prec, nrhs)
    wilson.wilson_mult(case.g.handle, out, inp, 1, 0, PRECS[prec], nrhs)
    got = case.to_canonical(out, 0, prec, nrhs=nrhs)
    for r in range(nrhs):
        want = oracle.Mee(case.U, case.half(psi, 0, r), case.dims, case.bc, case.kappa)
        assert rel(case.half(got, 0, r), want) < TOL[prec], (prec, r)


@pytest.mark.parametrize("inner,delta", [(wilson.WL_F32, 0.0), (wilson.WL_F16, 0.003)],
                         ids=["f32", "f16-reliable"])
def test_r12_solve_reaches_true_residual(case, inner, delta):
    nrhs = 2
    b = case.source(nrhs=nrhs, seed=61)
    x = torch.zeros_like(b)
    p = wilson.solve_params(tol=1e-10, eo=True, inner=inner, delta=delta)
    rc, info = wilson.wilson_solve(case.g.handle, x, b, nrhs, p)
    bn, xn = b.cpu().numpy(), x.cpu().numpy()
    for r in range(nrhs):
        tr = oracle.true_residual(case.U, bn[r], xn[r], case.dims, case.bc, case.kappa)
        assert tr <= 1e-10 and info[r]["status"] == 0, (r, tr, info[r])


@pytest.mark.parametrize("shape", [2, 18])
def test_r12_multi_rhs_shapes(monkeypatch, shape):
    monkeypatch.setenv("WL_MRHS_SHAPE", str(shape))
    c = Case((6, 4, 2, 8), kappa=0.124, kind="haar", seed=9, bc=(1, np.exp(0.3j), 1, -1), r12=True)
    try:
        nrhs = 4
        psi = c.source(nrhs=nrhs, seed=71)
        inp = c.to_internal(psi, 0, "f32")
        out = c.g.field("f32", nrhs)
        wilson.wilson_dslash(c.g.handle, out, inp, 1, 1, wilson.WL_F32, nrhs)
        got = c.to_canonical(out, 1, "f32", nrhs=nrhs)
        for r in range(nrhs):
            want = oracle.hop_eo(c.U, c.half(psi, 0, r), c.dims, c.bc, 1, dagger=True)
            assert rel(c.half(got, 1, r), want) < TOL["f32"], (shape, r)
    finally:
        c.close()


def test_r12_clover_solve():
    c = Case((4, 4, 2, 8), kappa=0.124, kind="haar", seed=19, bc=(1, 1, np.exp(0.2j), -1), r12=True)
    try:
        F = fields.clover_field(c.dims, 77)
        Fn = F.numpy()
        wilson.wl_clover_set(c.g.handle, F.to("cuda"))
        b = c.source(nrhs=1, seed=5)
        x = torch.zeros_like(b)
        wilson.wilson_solve(c.g.handle, x, b, 1, wilson.solve_params(tol=1e-10, eo=True, inner=wilson.WL_F32))
        bn, xn = b.cpu().numpy()[0], x.cpu().numpy()[0]
        r = bn - oracle.clover_D_full(c.U, Fn, xn, c.dims, c.bc, c.kappa)
        assert np.linalg.norm(r) / np.linalg.norm(bn) <= 1e-10
    finally:
        c.close()


def test_r12_rejects_non_su3_links():
    dims = (4, 4, 4, 4)
    U = fields.gauge_field(dims, "haar", 3)
    U = U * np.exp(0.1j)  # U(3), det != 1: the third row cannot be rebuilt
    with pytest.raises(wilson.WilsonError) as e:
        wilson.Gauge(dims, 0.12, U.to("cuda").contiguous(), precs=("f64", "f32"), r12=True)
    assert e.value.code == wilson.WL_ERR_ARG
