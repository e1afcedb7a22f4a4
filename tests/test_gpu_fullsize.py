"""Parity at the full workload sizes, in the launch configuration the bench
times (same gauge objects, autotuned launch shapes and solve parameters).

The oracle cannot apply D to a whole 48^3 x 96 lattice in test time, but it
evaluates the hopping term one site at a time (oracle.hop_eo_sites), so:

* the GPU hopping term is compared with the oracle at a few hundred sampled
  output sites (first and last sites of the half lattice, boundary sites in
  every direction, random sites);
* each full-size solve is checked through a property that holds at any size:
  the sampled residual components r_S = (b - D x)_S, recomputed by the oracle
  in FP64 at the sampled sites, obey ||r_S|| <= ||r|| <= tol ||b||, with the
  exact ||b|| of the full source.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import PRECS, TOL, rel
from paper_1811_00893_gb300 import fields, wilson, workloads

pytestmark = pytest.mark.gpu

# workload -> (storage precision of the hopping term, solve parameters), as in bench.SCHEMES
SCHEMES = {"fp32-defect-correction": ("f32", dict(eo=True, inner=wilson.WL_F32)),
           "fp16-reliable": ("f16", dict(eo=True, inner=wilson.WL_F16, delta=0.003)),
           "fp32-multirhs": ("f32", dict(eo=True, inner=wilson.WL_F32, graph_iters=4))}


def sample_sites(dims, parity, n_random=256, seed=0):
    """Half indices of parity `parity`: the first and last sites, sites on
    every face of the lattice, and random ones."""
    coords = fields.site_coords(dims)
    par = coords.sum(1) % 2 == parity
    idx = np.nonzero(par)[0]              # canonical sites of this parity, in half-index order
    picks = {0, len(idx) - 1}
    c = coords[idx]
    for mu in range(4):
        for edge in (0, dims[mu] - 1):
            on = np.nonzero(c[:, mu] == edge)[0]
            picks.update(on[:: max(1, len(on) // 16)][:16].tolist())
    rng = np.random.default_rng(seed)
    picks.update(rng.choice(len(idx), size=min(n_random, len(idx)), replace=False).tolist())
    return np.array(sorted(picks), dtype=np.int64)


@pytest.fixture(scope="module", params=[1, 2, 3, 5], ids=lambda i: workloads.by_index(i).name[:24])
def full(request):
    wl = workloads.by_index(request.param)
    prec, params = SCHEMES[wl.scheme]
    U = fields.gauge_field(wl.dims, wl.links, wl.gauge_seed, device="cuda")
    g = wilson.Gauge(wl.dims, wl.kappa, U, precs=("f64", prec), bc=wl.bc)
    F = None
    if wl.clover:
        F = fields.clover_field(wl.dims, wl.clover_seed, device="cuda")
        wilson.wl_clover_set(g.handle, F)
    Uh = U.cpu().numpy()
    del U
    b = fields.gaussian_fermion(wl.dims, wl.nrhs, wl.source_seed, device="cuda")
    yield wl, prec, params, g, Uh, b, (F.cpu().numpy() if F is not None else None)
    g.close()
    torch.cuda.empty_cache()


def test_fullsize_dslash_sampled(full):
    """The hopping term in the bench's configuration, at sampled sites."""
    wl, prec, params, g, Uh, b, F = full
    P = PRECS[prec]
    nr = wl.nrhs
    fin = g.field(prec, nr)
    fout = g.field(prec, nr)
    wilson.wl_field_to_internal(g.handle, fin, b, 1, P, nr)
    for _ in range(3):  # autotuned as in the bench's timed launches
        wilson.wilson_dslash(g.handle, fout, fin, 0, 0, P, nr)
    got = torch.zeros((nr, wl.volume, 4, 3), dtype=torch.complex128, device="cuda")
    wilson.wl_field_to_canonical(g.handle, got, fout, 0, P, nr)
    # the oracle hops the field as stored (rounded to the storage precision)
    inp = torch.zeros_like(got)
    wilson.wl_field_to_canonical(g.handle, inp, fin, 1, P, nr)
    sites = sample_sites(wl.dims, 0)
    coords = fields.site_coords(wl.dims)
    even = np.nonzero(coords.sum(1) % 2 == 0)[0]
    for r in range(min(nr, 3)):
        _, odd_half = oracle.split(inp[r].cpu().numpy(), wl.dims)
        want = oracle.hop_eo_sites(Uh, odd_half, wl.dims, wl.bc, 0, sites)
        mine = got[r].cpu().numpy()[even[sites]]
        assert rel(mine, want) < TOL[prec], (wl.name, r)


def test_fullsize_solve_residual_sampled(full):
    """The full-size solve: the library's true residual, and an independent
    check of it at sampled sites by the oracle in FP64."""
    wl, prec, params, g, Uh, b, F = full
    x = torch.zeros_like(b)
    p = wilson.solve_params(tol=1e-10, **params)
    rc, info = wilson.wilson_solve(g.handle, x, b, wl.nrhs, p)
    coords = fields.site_coords(wl.dims)
    for r in range(wl.nrhs if wl.nrhs <= 2 else 2):
        assert info[r]["status"] == 0 and info[r]["true_resid"] <= 1e-10, info[r]
        bn, xn = b[r].cpu().numpy(), x[r].cpu().numpy()
        bnorm = np.linalg.norm(bn)
        xe, xo = oracle.split(xn, wl.dims)
        rs2 = 0.0
        for parity in (0, 1):
            sites = sample_sites(wl.dims, parity, n_random=128, seed=parity + 1)
            canon = np.nonzero(coords.sum(1) % 2 == parity)[0][sites]
            hop = oracle.hop_eo_sites(Uh, xo if parity == 0 else xe, wl.dims, wl.bc, parity, sites)
            dx = xn[canon] - wl.kappa * hop.reshape(len(sites), 4, 3)
            if F is not None:  # + F(x) x(x) (Eq. 2), one site at a time
                for k, s in enumerate(canon):
                    Fs = np.zeros((12, 12), np.complex128)
                    Fs[:6, :6], Fs[6:, 6:] = F[s, 0], F[s, 1]
                    dx[k] += (Fs @ xn[s].reshape(12)).reshape(4, 3)
            rs2 += float(np.sum(np.abs(bn[canon] - dx) ** 2))
        assert np.sqrt(rs2) <= 1e-10 * bnorm * (1 + 1e-6), (wl.name, r, np.sqrt(rs2) / bnorm)
