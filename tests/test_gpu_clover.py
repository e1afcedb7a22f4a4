"""GPU parity of the clover term (Eq. 2) through the C ABI against the FP64 oracle.

The clover field is the synthetic F(x) of fields.clover_field: two random
Hermitian 6x6 blocks per site (scale 0.1, so 1 + F is well conditioned).
Tolerances follow gpu_helpers.TOL; FP16 additionally stores A and A^-1 in
half precision (relative rounding 2^-11 per entry; the clover FP16 tests
pass within the same 7e-4 FP16 bound).  Solves must reach a true residual
||b - D_clov x|| / ||b|| <= 1e-10 under the oracle's D_clov.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import PRECS, TOL, Case, rel
from paper_1811_00893_gb300 import fields, wilson

pytestmark = pytest.mark.gpu

SMALL = [((4, 4, 4, 4), (1, 1, 1, -1)),
         ((6, 4, 2, 8), (1, np.exp(0.3j), 1, -1)),   # ragged tail, L = 2, twisted phase
         ((8, 6, 4, 10), (1, 1, 1, -1))]


class CloverCase(Case):
    def __init__(self, dims, bc, seed=7, kappa=0.124):
        super().__init__(dims, kappa=kappa, kind="haar", seed=seed, bc=bc)
        self.F = fields.clover_field(dims, seed + 50).numpy()
        self.F_dev = torch.from_numpy(self.F).to("cuda").contiguous()
        wilson.wl_clover_set(self.g.handle, self.F_dev)


@pytest.fixture(scope="module", params=SMALL, ids=lambda c: "x".join(map(str, c[0])))
def case(request):
    dims, bc = request.param
    c = CloverCase(dims, bc)
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


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("inverse", [0, 1])
def test_clover_apply_matches_oracle(case, prec, inverse):
    psi = case.source(nrhs=2, seed=13)
    for parity in (0, 1):
        inp = case.to_internal(psi, parity, prec)
        out = case.g.field(prec, 2)
        wilson.wl_clover_apply(case.g.handle, out, inp, parity, inverse, PRECS[prec], 2)
        got = case.to_canonical(out, parity, prec, nrhs=2)
        for r in range(2):
            want = oracle.clover_diag(case.F, case.half(psi, parity, r), case.dims, parity,
                                      inverse=bool(inverse))
            assert rel(case.half(got, parity, r), want) < TOL[prec], (prec, parity, r)


def test_clover_apply_in_place_and_inverse_round_trip(case):
    psi = case.source(nrhs=1, seed=17)
    x = case.to_internal(psi, 1, "f64")
    wilson.wl_clover_apply(case.g.handle, x, x, 1, 0, wilson.WL_F64, 1)
    wilson.wl_clover_apply(case.g.handle, x, x, 1, 1, wilson.WL_F64, 1)
    back = case.to_canonical(x, 1, "f64")
    assert rel(case.half(back, 1), case.half(psi, 1)) < 1e-13


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_clover_D_matches_oracle(case, prec, dagger):
    nrhs = 2
    psi = case.source(nrhs=nrhs, seed=31)
    inp = full_internal(case, psi, prec)
    out = torch.empty_like(inp)
    wilson.wilson_mult(case.g.handle, out, inp, 0, dagger, PRECS[prec], nrhs)
    got = full_canonical(case, out, prec, nrhs).cpu().numpy()
    for r in range(nrhs):
        want = oracle.clover_D_full(case.U, case.F, psi[r].cpu().numpy(), case.dims, case.bc,
                                    case.kappa, dagger=bool(dagger))
        assert rel(got[r], want) < TOL[prec], (prec, r)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_clover_Mee_matches_oracle(case, prec, dagger):
    nrhs = 3
    psi = case.source(nrhs=nrhs, seed=41)
    inp = case.to_internal(psi, 0, prec)
    out = case.g.field(prec, nrhs)
    wilson.wilson_mult(case.g.handle, out, inp, 1, dagger, PRECS[prec], nrhs)
    got = case.to_canonical(out, 0, prec, nrhs=nrhs)
    for r in range(nrhs):
        pe = case.half(psi, 0, r)
        if not dagger:
            want = oracle.clover_Mee(case.U, case.F, pe, case.dims, case.bc, case.kappa)
        else:  # M_ee^dag = A_ee - kappa^2 (H^dag)_eo A_oo^-1 (H^dag)_oe  (A Hermitian)
            t = oracle.hop_eo(case.U, pe, case.dims, case.bc, 1, dagger=True)
            t = oracle.clover_diag(case.F, t, case.dims, 1, inverse=True)
            t = oracle.hop_eo(case.U, t, case.dims, case.bc, 0, dagger=True)
            want = oracle.clover_diag(case.F, pe, case.dims, 0) - case.kappa ** 2 * t
        assert rel(case.half(got, 0, r), want) < TOL[prec], (prec, r)


def clover_true_residual(c, b, x):
    r = b - oracle.clover_D_full(c.U, c.F, x, c.dims, c.bc, c.kappa)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.mark.parametrize("eo,inner,delta", [(False, wilson.WL_F64, 0.0), (True, wilson.WL_F64, 0.0),
                                            (True, wilson.WL_F32, 0.0), (True, wilson.WL_F16, 0.1)],
                         ids=["full-f64", "eo-f64", "eo-f32", "eo-f16-reliable"])
def test_clover_solve_reaches_true_residual(case, eo, inner, delta):
    nrhs = 2
    b = case.source(nrhs=nrhs, seed=61)
    x = torch.zeros_like(b)
    p = wilson.solve_params(tol=1e-10, eo=eo, inner=inner, delta=delta)
    rc, info = wilson.wilson_solve(case.g.handle, x, b, nrhs, p)
    bn, xn = b.cpu().numpy(), x.cpu().numpy()
    for r in range(nrhs):
        tr = clover_true_residual(case, bn[r], xn[r])
        assert tr <= 1e-10 and info[r]["status"] == 0, (r, tr, info[r])
        assert abs(info[r]["true_resid"] - tr) <= 0.05 * tr + 1e-15


def test_clover_batch_mixed_with_wilson():
    """A batch holding clover and plain Wilson lattices solves each to 1e-10."""
    specs = [((4, 4, 4, 4), 2, True), ((6, 4, 4, 8), 1, False), ((8, 4, 4, 4), 3, True)]
    cases, bs = [], []
    try:
        for n, (dims, nrhs, clov) in enumerate(specs):
            c = CloverCase(dims, (1, 1, 1, -1), seed=500 + n) if clov else \
                Case(dims, kappa=0.12, kind="haar", seed=500 + n)
            cases.append(c)
            bs.append(c.source(nrhs=nrhs, seed=600 + n))
        xs = [torch.zeros_like(b) for b in bs]
        p = wilson.solve_params(tol=1e-10, eo=True, inner=wilson.WL_F32)
        rc, infos = wilson.wilson_solve_batch([c.g.handle for c in cases], xs, bs,
                                              [b.shape[0] for b in bs], p)
        k = 0
        for c, b, x, (_, nrhs, clov) in zip(cases, bs, xs, specs):
            bn, xn = b.cpu().numpy(), x.cpu().numpy()
            for r in range(nrhs):
                tr = clover_true_residual(c, bn[r], xn[r]) if clov else \
                    oracle.true_residual(c.U, bn[r], xn[r], c.dims, c.bc, c.kappa)
                assert tr <= 1e-10 and infos[k]["status"] == 0, (c.dims, r, tr, infos[k])
                k += 1
    finally:
        for c in cases:
            c.close()


def test_clover_rejects_bad_input():
    c = Case((4, 4, 4, 4), kappa=0.12, kind="haar", seed=3)
    try:
        psi = c.source(nrhs=1, seed=1)
        x = c.to_internal(psi, 0, "f32")
        with pytest.raises(wilson.WilsonError) as e:  # no clover term yet
            wilson.wl_clover_apply(c.g.handle, x, x, 0, 0, wilson.WL_F32, 1)
        assert e.value.code == wilson.WL_ERR_STATE
        F = fields.clover_field(c.dims, 9)
        with pytest.raises(wilson.WilsonError) as e:  # host memory
            wilson.wl_clover_set(c.g.handle, F.numpy())
        assert e.value.code == wilson.WL_ERR_ARG
        bad = F.clone()
        bad[0, 0, 1, 0] += 0.05  # breaks Hermiticity at one site
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wl_clover_set(c.g.handle, bad.to("cuda"))
        assert e.value.code == wilson.WL_ERR_ARG
        sing = torch.zeros_like(F)
        sing[5, 1] = -torch.eye(6, dtype=F.dtype)  # 1 + F = 0 on one block
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wl_clover_set(c.g.handle, sing.to("cuda"))
        assert e.value.code == wilson.WL_ERR_ARG
        # a failed set leaves the plain Wilson operator; attach then detach
        wilson.wl_clover_set(c.g.handle, F.to("cuda"))
        wilson.wl_clover_set(c.g.handle, None)
        full = torch.empty(2 * wilson.wl_field_bytes(c.g.handle, wilson.WL_F64, 1),
                           dtype=torch.uint8, device="cuda")
        fb = full.numel() // 2
        wilson.wl_field_to_internal(c.g.handle, full[:fb], psi, 0, wilson.WL_F64, 1)
        wilson.wl_field_to_internal(c.g.handle, full[fb:], psi, 1, wilson.WL_F64, 1)
        out = torch.empty_like(full)
        wilson.wilson_mult(c.g.handle, out, full, 0, 0, wilson.WL_F64, 1)
        got = torch.zeros_like(psi)
        wilson.wl_field_to_canonical(c.g.handle, got, out[:fb], 0, wilson.WL_F64, 1)
        wilson.wl_field_to_canonical(c.g.handle, got, out[fb:], 1, wilson.WL_F64, 1)
        want = oracle.D_full(c.U, psi[0].cpu().numpy(), c.dims, c.bc, c.kappa)
        assert rel(got[0].cpu().numpy(), want) < 1e-12
    finally:
        c.close()
