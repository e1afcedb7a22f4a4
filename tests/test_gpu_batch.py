"""Uneven multi-lattice batches (wilson_solve_batch) against the oracle.

Every system (lattice, right-hand side) of a batch must reach a true residual
||b - D x|| / ||b|| <= 1e-10 under the oracle's FP64 D for its own lattice,
the library's residual report must agree, and a batch must give the same
iteration counts as solving its lattices one by one (the batched kernels run
the same arithmetic on every system)."""
import pytest
import torch

import oracle
from gpu_helpers import Case
from paper_1811_00893_gb300 import wilson, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


def make_batch(specs):
    cases, bs = [], []
    for n, (dims, nrhs, kappa) in enumerate(specs):
        c = Case(dims, kappa=kappa, kind="haar", seed=300 + n, precs=("f64", "f32", "f16"))
        cases.append(c)
        bs.append(c.source(nrhs=nrhs, seed=400 + 10 * n))
    return cases, bs


def check(cases, bs, xs, infos, tol=TOL):
    k = 0
    for c, b, x in zip(cases, bs, xs):
        bn, xn = b.cpu().numpy(), x.cpu().numpy()
        for r in range(b.shape[0]):
            tr = oracle.true_residual(c.U, bn[r], xn[r], c.dims, c.bc, c.kappa)
            assert tr <= tol and infos[k]["status"] == 0, (c.dims, r, tr, infos[k])
            assert abs(infos[k]["true_resid"] - tr) <= 0.05 * tr + 1e-15
            k += 1


SMALL = [((4, 4, 4, 4), 2, 0.115), ((6, 4, 4, 8), 1, 0.12), ((8, 8, 4, 4), 3, 0.124),
         ((2, 2, 2, 2), 1, 0.11)]


@pytest.mark.parametrize("inner,delta,graph", [(wilson.WL_F32, 0.0, 0), (wilson.WL_F32, 0.0, 4),
                                               (wilson.WL_F16, 0.1, 0), (wilson.WL_F64, 0.0, 2)],
                         ids=["f32", "f32-graph", "f16-reliable", "f64-graph"])
def test_small_uneven_batch(inner, delta, graph):
    cases, bs = make_batch(SMALL)
    try:
        xs = [torch.zeros_like(b) for b in bs]
        p = wilson.solve_params(tol=TOL, eo=True, inner=inner, delta=delta, graph_iters=graph)
        rc, infos = wilson.wilson_solve_batch([c.g.handle for c in cases], xs, bs,
                                              [b.shape[0] for b in bs], p)
        check(cases, bs, xs, infos)
        # the same systems solved one lattice at a time take the same iterations
        k = 0
        for c, b in zip(cases, bs):
            x1 = torch.zeros_like(b)
            rc, inf1 = wilson.wilson_solve(c.g.handle, x1, b, b.shape[0], p)
            for r in range(b.shape[0]):
                assert abs(inf1[r]["iters"] - infos[k]["iters"]) <= 2 * max(graph, 4)
                k += 1
    finally:
        for c in cases:
            c.close()


def test_batch_rejects_bad_arguments():
    cases, bs = make_batch(SMALL[:2])
    try:
        xs = [torch.zeros_like(b) for b in bs]
        hs = [c.g.handle for c in cases]
        nr = [b.shape[0] for b in bs]
        with pytest.raises(wilson.WilsonError):  # batches are even-odd
            wilson.wilson_solve_batch(hs, xs, bs, nr, wilson.solve_params(eo=False, inner=1))
        with pytest.raises(wilson.WilsonError):  # one gauge twice
            wilson.wilson_solve_batch([hs[0], hs[0]], [xs[0], xs[0]], [bs[0], bs[0]],
                                      [nr[0], nr[0]], wilson.solve_params(inner=1))
    finally:
        for c in cases:
            c.close()


def test_uneven_batch_workload():
    """The 16-lattice workload: extents from {8^4, 12^3x24, 16^3x32, 16^4},
    1-8 RHS each, kappa in [0.11, 0.124], Haar links, FP32 inner, graphs."""
    spec = workloads.uneven_batch()
    cases, bs = [], []
    for m in spec:
        c = Case(m.dims, kappa=m.kappa, kind="haar", seed=m.gauge_seed, precs=("f64", "f32"))
        cases.append(c)
        bs.append(c.source(nrhs=m.nrhs, seed=m.source_seed))
    try:
        xs = [torch.zeros_like(b) for b in bs]
        p = wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32, graph_iters=8)
        rc, infos = wilson.wilson_solve_batch([c.g.handle for c in cases], xs, bs,
                                              [m.nrhs for m in spec], p)
        check(cases, bs, xs, infos)
    finally:
        for c in cases:
            c.close()


def test_alternating_batches_keep_their_contexts():
    """Two callers alternating between two batches (and a batch sharing a
    lattice with another): each batch finds its cached device description
    again, and every solve reaches the oracle residual."""
    cases, bs = make_batch(SMALL)
    try:
        groups = [[0, 1], [2, 3], [1, 2]]
        p = wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32, graph_iters=4)
        for rep in range(3):
            for grp in groups:
                cs = [cases[i] for i in grp]
                bb = [bs[i] for i in grp]
                xs = [torch.zeros_like(b) for b in bb]
                rc, infos = wilson.wilson_solve_batch([c.g.handle for c in cs], xs, bb,
                                                      [b.shape[0] for b in bb], p)
                check(cs, bb, xs, infos)
    finally:
        for c in cases:
            c.close()


def test_batch_with_host_buffers_on_a_busy_stream():
    """Host and device buffers mixed in one batch (pinned host, pageable host,
    device), called on a side stream whose last work, the write of a device b,
    is still running when the call starts: every lattice's own stream waits for
    the caller's stream, and every solve reaches the oracle residual."""
    cases, bs = make_batch(SMALL)
    try:
        nr = [b.shape[0] for b in bs]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            b0 = torch.empty_like(bs[0])
            torch.cuda._sleep(50_000_000)  # about 25 ms of GPU time before b0 is written
            b0.copy_(bs[0])
        bb = [b0, bs[1].cpu().pin_memory(), bs[2].cpu(), bs[3]]
        xs = [torch.zeros_like(bs[0]), torch.zeros_like(bb[1]).pin_memory(), torch.zeros_like(bb[2]),
              torch.zeros_like(bs[3])]
        p = wilson.solve_params(tol=TOL, eo=True, inner=wilson.WL_F32, graph_iters=4)
        rc, infos = wilson.wilson_solve_batch([c.g.handle for c in cases], xs, bb, nr, p, stream=side)
        side.synchronize()
        check(cases, bs, xs, infos)
    finally:
        for c in cases:
            c.close()
