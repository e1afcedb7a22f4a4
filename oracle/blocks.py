"""Eq. 1 on one block of a decomposed lattice, for checking the face exchange.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the test suite
may import it.  It restates the hopping sum of Eq. 1 (Sec. 2) on one block of
a lattice cut into blocks along y, z and t, where the spinors of hops that
leave the block arrive as faces of the neighbouring blocks (the pack /
communicate / boundary steps of Sec. 4.4).  It shares no code with the GPU
library.  All arithmetic is numpy FP64 with the oracle's own gamma matrices
(``oracle.gamma``), one direction at a time.

A face holds, per face site, spin rows 0 and 1 of P psi with P = 1 - gamma_mu
(faces sent backward: the receiver's forward hop) or 1 + gamma_mu (sent
forward: the receiver's backward hop); the adjoint operator flips the signs.
The other two rows follow from these: in the chiral basis the diagonal 2x2
spin blocks of gamma_mu vanish, so P = [[1, B], [C, 1]], and P P = 2 P gives
C B = 1, hence rows 2, 3 of P psi = C (rows 0, 1).  ``reconstruct`` uses this
identity; ``tests/test_oracle_blocks.py`` pins every function here against
the undivided oracle.

Face site order: the site's half index with the mu coordinate dropped,
x / 2 fastest, then the remaining directions in the order y, z, t.
"""
from __future__ import annotations

import numpy as np

from . import gamma as _gamma


def layout(dims, grid, block: int):
    """(local extents, origin, coordinates of the block in the grid)."""
    L = [dims[m] // grid[m] for m in range(4)]
    c = [0, block % grid[1], (block // grid[1]) % grid[2], block // (grid[1] * grid[2])]
    return L, [c[m] * L[m] for m in range(4)], c


def _coords(L, n):
    s = np.arange(n)
    x = s % L[0]
    y = (s // L[0]) % L[1]
    z = (s // (L[0] * L[1])) % L[2]
    t = s // (L[0] * L[1] * L[2])
    return np.stack([x, y, z, t], axis=1)


def half_sites(L, parity: int):
    """Coordinates (x, y, z, t) of the parity sites of a lattice L, by half index."""
    V = int(np.prod(L))
    c = _coords(L, V)
    keep = (c.sum(axis=1) % 2) == parity
    s = np.nonzero(keep)[0]
    order = np.argsort(s // 2, kind="stable")
    return c[s[order]]


def block_half(psi_half_global, dims, grid, block: int, parity: int):
    """The parity half field of one block, from the whole lattice's half field."""
    L, o, _ = layout(dims, grid, block)
    cl = half_sites(L, parity)
    cg = cl + np.asarray(o)
    sg = cg[:, 0] + dims[0] * (cg[:, 1] + dims[1] * (cg[:, 2] + dims[2] * cg[:, 3]))
    return psi_half_global[sg // 2]


def face_index(L, mu: int, c):
    """Index of sites with coordinates c in the face of direction mu."""
    xh = c[:, 0] // 2
    if mu == 1:
        return xh + (L[0] // 2) * (c[:, 2] + L[2] * c[:, 3])
    if mu == 2:
        return xh + (L[0] // 2) * (c[:, 1] + L[1] * c[:, 3])
    return xh + (L[0] // 2) * (c[:, 1] + L[1] * c[:, 2])


def projector(mu: int, sign: int, dagger: bool = False):
    """1 + sign gamma_mu (sign flipped for the adjoint operator)."""
    s = -sign if dagger else sign
    return np.eye(4) + s * _gamma(mu)


def face_halves(psi_block_half, L, parity: int, mu: int, side: int, dagger: bool = False):
    """The face a block sends: side 0 is its x_mu = 0 face under 1 - gamma_mu,
    side 1 its x_mu = L_mu - 1 face under 1 + gamma_mu; rows 0, 1 of P psi at
    each face site, in face order.  Shape (face sites, 2, 3)."""
    c = half_sites(L, parity)
    at = c[:, mu] == (0 if side == 0 else L[mu] - 1)
    f = face_index(L, mu, c[at])
    P = projector(mu, -1 if side == 0 else +1, dagger)
    full = np.einsum("ab,nbc->nac", P, psi_block_half[at])
    out = np.zeros((int(np.prod(L)) // 2 // L[mu], 2, 3), np.complex128)
    out[f] = full[:, :2, :]
    return out


def reconstruct(h, mu: int, sign: int, dagger: bool = False):
    """P psi from its rows 0, 1 (P = 1 + sign gamma_mu): rows 2, 3 = C h."""
    P = projector(mu, sign, dagger)
    C = P[2:, :2]
    return np.concatenate([h, np.einsum("ab,nbc->nac", C, h)], axis=1)


def hop_block(U, dims, bc, grid, block: int, psi_block_half, out_parity: int, halos, dagger: bool = False):
    """H_{p,1-p} of Eq. 1 on one block: out_parity sites from the block's
    (1 - out_parity) half field and the received faces halos[(mu, side)]
    (side 0: for the forward hops of x_mu = L_mu - 1 sites, side 1: for the
    backward hops of x_mu = 0 sites).  U is the whole lattice's canonical
    gauge field (V, 4, 3, 3)."""
    L, o, _ = layout(dims, grid, block)
    U = np.asarray(U).reshape(-1, 4, 3, 3)
    co = half_sites(L, out_parity)
    n = co.shape[0]
    # half index of any local site of the input parity
    Lxh = L[0] // 2

    def local_half(c):
        return c[:, 0] // 2 + Lxh * (c[:, 1] + L[1] * (c[:, 2] + L[2] * c[:, 3]))

    def gsite(c):
        g = (c + np.asarray(o)) % np.asarray(dims)
        return g[:, 0] + dims[0] * (g[:, 1] + dims[1] * (g[:, 2] + dims[2] * g[:, 3]))

    out = np.zeros((n, 4, 3), np.complex128)
    gco = co + np.asarray(o)
    for mu in range(4):
        cut = grid[mu] > 1
        for fwd in (True, False):
            step = np.zeros(4, int)
            step[mu] = 1 if fwd else -1
            nb = co + step
            leaves = (nb[:, mu] < 0) | (nb[:, mu] >= L[mu])
            nb[:, mu] %= L[mu]  # inside an uncut direction the block is the whole extent
            sign = -1 if fwd else +1  # Eq. 1: (1 - gamma) forward, (1 + gamma) backward
            P = projector(mu, sign, dagger)
            # link of the hop: U_mu(x) forward, U_mu(x - mu)^dag backward, with
            # the boundary phase when the hop crosses the lattice's edge
            if fwd:
                W = U[gsite(co), mu]
                edge = gco[:, mu] == dims[mu] - 1
                ph = np.where(edge, bc[mu], 1.0)
            else:
                W = np.conj(np.transpose(U[gsite(co + step), mu], (0, 2, 1)))
                edge = gco[:, mu] == 0
                ph = np.where(edge, np.conj(bc[mu]), 1.0)
            W = W * ph[:, None, None]
            psi_nb = psi_block_half[local_half(nb)]
            Ppsi = np.einsum("ab,nbc->nac", P, psi_nb)
            if cut and np.any(leaves):
                h = halos[(mu, 0 if fwd else 1)]
                f = face_index(L, mu, co[leaves])
                Ppsi[leaves] = reconstruct(h[f], mu, sign, dagger)
            out += np.einsum("nij,naj->nai", W, Ppsi)
    return out
