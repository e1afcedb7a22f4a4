"""Pins of oracle.blocks (Eq. 1 on one block of a decomposed lattice, with the
hops that leave the block fed by the neighbours' projected faces) against the
undivided oracle: the blocks tile the lattice, the face reconstruction gives
back (1 -+ gamma_mu) psi, and every block's hopping term equals the
undivided hopping term at the block's sites, for cuts along t, z x t and
y x z x t, block extent 2 on a cut, twisted phases and the adjoint."""
import numpy as np
import pytest

import oracle
from oracle import blocks
from paper_1811_00893_gb300 import fields

CASES = [((4, 4, 4, 8), (1, 1, 1, 2), (1, 1, 1, -1)),
         ((6, 4, 4, 4), (1, 1, 1, 2), (1, 1, 1, np.exp(0.7j))),
         ((4, 4, 8, 8), (1, 1, 2, 2), (1, np.exp(0.2j), 1, -1)),
         ((4, 4, 4, 8), (1, 2, 2, 2), (1, 1, np.exp(0.7j), -1)),
         ((4, 2, 2, 12), (1, 1, 1, 3), (1, 1, 1, -1))]


def _faces_for(U, psi_in_half, dims, grid, block, parity, dagger):
    """The halos block `block` receives: its neighbours' faces."""
    L, _, c = blocks.layout(dims, grid, block)
    halos = {}
    for mu in (1, 2, 3):
        if grid[mu] == 1:
            continue
        for side in (0, 1):
            # side 0 arrives from the forward neighbour (its x_mu = 0 face),
            # side 1 from the backward one (its x_mu = L - 1 face)
            cc = list(c)
            cc[mu] = (c[mu] + (1 if side == 0 else -1)) % grid[mu]
            nb = cc[1] + grid[1] * (cc[2] + grid[2] * cc[3])
            nb_half = blocks.block_half(psi_in_half, dims, grid, nb, parity)
            halos[(mu, side)] = blocks.face_halves(nb_half, L, parity, mu, side, dagger)
    return halos


@pytest.mark.parametrize("dims,grid,bc", CASES, ids=lambda v: str(v))
def test_blocks_tile_the_lattice(dims, grid, bc):
    V = int(np.prod(dims))
    seen = np.zeros(V // 2, int)
    idx = np.arange(V // 2, dtype=np.float64).reshape(-1, 1, 1) * np.ones((1, 4, 3))
    nblk = grid[1] * grid[2] * grid[3]
    for b in range(nblk):
        h = blocks.block_half(idx, dims, grid, b, 0)
        seen[h[:, 0, 0].astype(int)] += 1
    assert np.all(seen == 1)


@pytest.mark.parametrize("mu", [0, 1, 2, 3])
@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_reconstruct_gives_the_projected_spinor(mu, sign, dagger):
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((7, 4, 3)) + 1j * rng.standard_normal((7, 4, 3))
    P = blocks.projector(mu, sign, dagger)
    full = np.einsum("ab,nbc->nac", P, psi)
    assert np.allclose(blocks.reconstruct(full[:, :2], mu, sign, dagger), full, atol=1e-14, rtol=0)


@pytest.mark.parametrize("dims,grid,bc", CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("dagger", [False, True])
def test_block_hop_equals_undivided(dims, grid, bc, dagger):
    U = fields.gauge_field(dims, "haar", 11).numpy()
    psi = fields.gaussian_fermion(dims, 1, 12)[0].numpy()
    nblk = grid[1] * grid[2] * grid[3]
    for out_parity in (0, 1):
        e, o = oracle.split(psi, dims)
        inp = o if out_parity == 0 else e
        want = oracle.hop_eo(U, inp, dims, bc, out_parity, dagger=dagger)
        for b in range(nblk):
            halos = _faces_for(U, inp, dims, grid, b, 1 - out_parity, dagger)
            got = blocks.hop_block(U, dims, bc, grid, b, blocks.block_half(inp, dims, grid, b, 1 - out_parity),
                                   out_parity, halos, dagger)
            ref = blocks.block_half(want, dims, grid, b, out_parity)
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (b, out_parity)
