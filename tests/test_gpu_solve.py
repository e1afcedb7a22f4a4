"""GPU solves against the oracle: every solution must have a true residual
||b - D x|| / ||b|| <= 1e-10 when evaluated with the oracle's FP64 D, the
library's own FP64 residual report must agree with the oracle's, and the
solution must match the oracle's solve within the forward-error bound
cond(D) * 1e-10 with cond(D) <= (1 + 8 kappa)/(1 - 8 kappa)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import Case, rel
from paper_1811_00893_gb300 import wilson

pytestmark = pytest.mark.gpu

TOL = 1e-10


def check_solution(c, b, x, infos, tol=TOL):
    bn, xn = b.cpu().numpy(), x.cpu().numpy()
    for r in range(b.shape[0]):
        tr = oracle.true_residual(c.U, bn[r], xn[r], c.dims, c.bc, c.kappa)
        assert tr <= tol, (r, tr, infos[r])
        assert infos[r]["status"] == 0
        assert abs(infos[r]["true_resid"] - tr) <= 0.05 * tr + 1e-15, (infos[r], tr)


SCHEMES = {
    "fp64-full": dict(eo=False, inner=wilson.WL_F64),
    "fp64-eo": dict(eo=True, inner=wilson.WL_F64),
    "fp32-dc-eo": dict(eo=True, inner=wilson.WL_F32),
    "fp32-dc-full": dict(eo=False, inner=wilson.WL_F32),
    "fp16-reliable-eo": dict(eo=True, inner=wilson.WL_F16, delta=0.1),
    "fp32-reliable-eo": dict(eo=True, inner=wilson.WL_F32, delta=0.1),
    "fp16-dc-eo": dict(eo=True, inner=wilson.WL_F16),
}


@pytest.fixture(scope="module")
def c8():
    c = Case((8, 8, 8, 8), kappa=0.12, kind="haar", seed=1000)
    yield c
    c.close()


@pytest.mark.parametrize("scheme", sorted(SCHEMES))
def test_solve_schemes(c8, scheme):
    b = c8.source(nrhs=1, seed=2000)
    x = torch.zeros_like(b)
    p = wilson.solve_params(tol=TOL, **SCHEMES[scheme])
    rc, infos = wilson.wilson_solve(c8.g.handle, x, b, 1, p)
    check_solution(c8, b, x, infos)


def test_solve_agrees_with_oracle_solution(c8):
    b = c8.source(nrhs=1, seed=2001)
    x = torch.zeros_like(b)
    wilson.wilson_solve(c8.g.handle, x, b, 1, wilson.solve_params(tol=1e-12, eo=True,
                                                                  inner=wilson.WL_F32))
    xo, info = oracle.solve(c8.U, b[0].cpu().numpy(), c8.dims, c8.bc, c8.kappa, eo=True, tol=1e-12)
    cond = (1 + 8 * c8.kappa) / (1 - 8 * c8.kappa)
    assert rel(x[0].cpu().numpy(), xo) < 2 * cond * 1e-12


@pytest.mark.parametrize("graph_iters", [0, -1, 8])
def test_multi_rhs_and_graphs(graph_iters):
    c = Case((6, 4, 4, 8), kappa=0.124, kind="haar", seed=3)
    try:
        b = c.source(nrhs=5, seed=30)
        x = torch.zeros_like(b)
        p = wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32, graph_iters=graph_iters)
        before = wilson.wl_launch_count()
        rc, infos = wilson.wilson_solve(c.g.handle, x, b, 5, p)
        assert wilson.wl_launch_count() > before
        check_solution(c, b, x, infos)
        # a second solve reuses the workspace (and the captured graph)
        x2 = torch.zeros_like(b)
        rc, infos2 = wilson.wilson_solve(c.g.handle, x2, b, 5, p)
        check_solution(c, b, x2, infos2)
    finally:
        c.close()


def test_timing_sees_graph_replays():
    """The per-launch timing records the hopping launches of the solver's graph
    replays like eager ones, and replaying the iterations changes no bit."""
    c = Case((8, 8, 8, 16), kappa=0.124, kind="haar", seed=5)
    try:
        b = c.source(nrhs=1, seed=50)
        got = {}
        for gi in (-4, 4):
            x = torch.zeros_like(b)
            p = wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32, graph_iters=gi)
            wilson.wilson_solve(c.g.handle, x, b, 1, p)  # capture outside the timed solve
            x = torch.zeros_like(b)
            wilson.wl_timing(c.g.handle, True)
            rc, infos = wilson.wilson_solve(c.g.handle, x, b, 1, p)
            wilson.wl_timing(c.g.handle, False)
            check_solution(c, b, x, infos)
            got[gi] = (x, infos[0]["iters"], wilson.wl_timing_read(c.g.handle, wilson.WL_F32))
        (xe, ie, (mse, ne, be)), (xg, ig, (msg, ng, bg)) = got[-4], got[4]
        assert ig == ie and torch.equal(xg, xe)
        assert ne == ng and be == bg
        assert abs(ne - 4 * ie) <= 4  # two hops per M_ee, two M_ee per iteration
        assert mse > 0 and msg > 0 and 0.2 < msg / mse < 5
    finally:
        c.close()


def test_resume_from_initial_guess(c8):
    b = c8.source(nrhs=1, seed=2002)
    x = torch.zeros_like(b)
    p = wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F64, maxiter=3)
    rc, infos = wilson.wilson_solve(c8.g.handle, x, b, 1, p, check=False)
    assert rc == wilson.WL_ERR_NOT_CONVERGED and infos[0]["true_resid"] > TOL
    assert infos[0]["iters"] <= 3  # maxiter bounds the inner iterations exactly
    p2 = wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F64, use_x0=True)
    rc, infos2 = wilson.wilson_solve(c8.g.handle, x, b, 1, p2)
    check_solution(c8, b, x, infos2)


def test_host_buffers(c8):
    b = c8.source(nrhs=1, seed=2003)
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    rc, infos = wilson.wilson_solve(c8.g.handle, xh, bh, 1,
                                    wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32))
    check_solution(c8, b, xh, infos)
    xn = np.zeros(b[0].shape, np.complex128)[None]
    bn = b.cpu().numpy()
    rc, infos = wilson.wilson_solve(c8.g.handle, xn, bn, 1,
                                    wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32))
    check_solution(c8, b, torch.from_numpy(xn), infos)


def test_degenerate_cases():
    c = Case((4, 4, 4, 4), kappa=0.0, kind="haar", seed=5)
    try:
        b = c.source(nrhs=2, seed=50)
        b[1].zero_()
        x = torch.zeros_like(b)
        rc, infos = wilson.wilson_solve(c.g.handle, x, b, 2,
                                        wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32))
        assert torch.allclose(x[0], b[0], rtol=0, atol=1e-12 * b[0].abs().max().item())
        assert torch.count_nonzero(x[1]) == 0 and infos[1]["true_resid"] == 0.0
    finally:
        c.close()


def test_bad_params_rejected(c8):
    b = c8.source(nrhs=1, seed=1)
    x = torch.zeros_like(b)
    for kw in (dict(tol=0.0), dict(maxiter=0), dict(inner=7)):
        args = dict(tol=TOL, eo=True, inner=wilson.WL_F32)
        args.update(kw)
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wilson_solve(c8.g.handle, x, b, 1, wilson.solve_params(**args))
        assert e.value.code == wilson.WL_ERR_ARG
