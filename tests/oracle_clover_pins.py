"""Pins of the oracle's clover operator (Eq. 2: D_clov = D_W + F(x) delta_xy).

* dense brute force: D_W assembled from Eq. 1 (oracle_pins.dense_D) plus the
  block-diagonal 12x12 F(x) per site, on 2^4 and 4x2x2x4 lattices;
* free field with a constant F: D e^{ipx} chi = e^{ipx} (M(p) + F0) chi;
* gamma5-hermiticity: F is Hermitian and block diagonal in the chiral basis,
  so it commutes with gamma5 and D_clov^dag = g5 D_clov g5 still holds;
* gauge covariance with F'(x) = (1 x g(x)) F(x) (1 x g(x))^dag;
* the per-site inverse (1 + F)^{-1} against numpy's inverse;
* M_ee = A_ee - D_eo A_oo^{-1} D_oe composed from the full operator, with the
  per-site inverse taken from numpy;
* solve: the oracle's clover BiCGStab (full and even-odd) against dense LU of
  D_clov, and its true residual against the dense matrix.
"""
import numpy as np

import oracle
import oracle_pins as P
from paper_1811_00893_gb300 import fields

I4 = np.eye(4)


def _F(dims, seed, scale=0.1):
    return fields.clover_field(dims, seed, scale=scale).numpy()


def block12(Fs):
    M = np.zeros((12, 12), np.complex128)
    M[:6, :6] = Fs[0]
    M[6:, 6:] = Fs[1]
    return M


def dense_clover(U, F, dims, bc, kappa):
    Dm = P.dense_D(U, dims, bc, kappa)
    for s in range(F.shape[0]):
        Dm[12 * s:12 * s + 12, 12 * s:12 * s + 12] += block12(F[s])
    return Dm


def check_clover_hermitian_blocks():
    F = _F((4, 2, 2, 2), 1)
    assert np.allclose(F, F.conj().transpose(0, 1, 3, 2), atol=0)
    g5 = np.kron(np.diag([1, 1, -1, -1]), np.eye(3))
    for s in range(F.shape[0]):
        assert np.allclose(g5 @ block12(F[s]), block12(F[s]) @ g5), "F must commute with gamma5"


def check_clover_dense():
    for n, (dims, bc) in enumerate([((2, 2, 2, 2), (1, 1, 1, -1)),
                                     ((4, 2, 2, 4), (1, np.exp(0.4j), 1, -1))]):
        U = P._haar_links(dims, 500 + n)
        F = _F(dims, 510 + n, scale=0.3)
        psi = P._source(dims, 520 + n)
        Dm = dense_clover(U, F, dims, bc, 0.12)
        got = oracle.clover_D_full(U, F, psi, dims, bc, 0.12).reshape(-1)
        assert P._rel(got, Dm @ psi.reshape(-1)) < 1e-14
        gotd = oracle.clover_D_full(U, F, psi, dims, bc, 0.12, dagger=True).reshape(-1)
        assert P._rel(gotd, Dm.conj().T @ psi.reshape(-1)) < 1e-14


def check_clover_plane_wave():
    g = P.gammas()
    dims, theta = (4, 4, 2, 6), (0, 0, 0, np.pi)
    bc = tuple(np.exp(1j * t) for t in theta)
    F0 = _F((2, 1, 1, 1), 530)[0]
    F = np.broadcast_to(F0, (int(np.prod(dims)), 2, 6, 6)).copy()
    rng = np.random.default_rng(3)
    U = P._unit_links(dims)
    for _ in range(3):
        n = [rng.integers(0, L) for L in dims]
        p = [(2 * np.pi * n[m] + theta[m]) / dims[m] for m in range(4)]
        chi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        kappa = 0.13
        Mp = (1 - 2 * kappa * sum(np.cos(p))) * I4 + 2j * kappa * sum(np.sin(p[m]) * g[m] for m in range(4))
        want_chi = (np.kron(Mp, np.eye(3)) + block12(F0)) @ chi.reshape(-1)
        want = P._plane_wave(dims, p, want_chi.reshape(4, 3))
        got = oracle.clover_D_full(U, F, P._plane_wave(dims, p, chi), dims, bc, kappa)
        assert P._rel(got, want) < 1e-13


def check_clover_gamma5():
    dims, bc = (4, 2, 4, 4), (1, 1, 1, -1)
    U, F = P._haar_links(dims, 540), _F(dims, 541, scale=0.3)
    phi, psi = P._source(dims, 542), P._source(dims, 543)
    g5 = lambda f: np.einsum("st,vtc->vsc", P.G5, f)
    lhs = np.vdot(phi, oracle.clover_D_full(U, F, psi, dims, bc, 0.12))
    rhs = np.vdot(g5(oracle.clover_D_full(U, F, g5(phi), dims, bc, 0.12)), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def check_clover_gauge_covariance():
    dims, bc = (4, 2, 2, 4), (1, 1, np.exp(0.3j), -1)
    U, F = P._haar_links(dims, 550), _F(dims, 551, scale=0.3)
    psi = P._source(dims, 552)
    g = fields.gauge_transform(dims, 553).numpy()
    c = fields.site_coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        f = c.copy()
        f[:, mu] = (f[:, mu] + 1) % dims[mu]
        fi = f[:, 0] + dims[0] * (f[:, 1] + dims[1] * (f[:, 2] + dims[2] * f[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ g[fi].conj().transpose(0, 2, 1)
    G = np.einsum("ab,vcd->vacbd", np.eye(2), g).reshape(-1, 6, 6)  # 1_2 (x) g
    Fg = np.einsum("vij,vbjk,vlk->vbil", G, F, G.conj())
    gpsi = np.einsum("vab,vsb->vsa", g, psi)
    lhs = oracle.clover_D_full(Ug, Fg, gpsi, dims, bc, 0.12)
    rhs = np.einsum("vab,vsb->vsa", g, oracle.clover_D_full(U, F, psi, dims, bc, 0.12))
    assert P._rel(lhs, rhs) < 1e-13


def check_clover_inverse():
    dims = (4, 2, 2, 2)
    F = _F(dims, 560, scale=0.4)
    e, o = oracle.split(P._source(dims, 561), dims)
    for par, half in ((0, e), (1, o)):
        got = oracle.clover_diag(F, half, dims, par, inverse=True)
        back = oracle.clover_diag(F, got, dims, par, inverse=False)
        assert P._rel(back, half) < 1e-14
        sites = np.nonzero(fields.site_coords(dims).sum(1) % 2 == par)[0]
        for i, s in enumerate(sites):
            A = np.eye(12) + block12(F[s])
            assert P._rel(got[i].reshape(-1), np.linalg.solve(A, half[i].reshape(-1))) < 1e-14


def check_clover_schur():
    dims, bc = (4, 4, 2, 4), (1, 1, 1, -1)
    U, F = P._haar_links(dims, 570), _F(dims, 571, scale=0.3)
    kappa = 0.12
    e, _ = oracle.split(P._source(dims, 572), dims)
    zero = np.zeros_like(e)
    Ae, y = oracle.split(oracle.clover_D_full(U, F, oracle.join(e, zero, dims), dims, bc, kappa), dims)
    odd_sites = np.nonzero(fields.site_coords(dims).sum(1) % 2 == 1)[0]
    z = np.stack([np.linalg.solve(np.eye(12) + block12(F[s]), y[i].reshape(-1)).reshape(4, 3)
                  for i, s in enumerate(odd_sites)])
    w, _ = oracle.split(oracle.clover_D_full(U, F, oracle.join(zero, z, dims), dims, bc, kappa), dims)
    got = oracle.clover_Mee(U, F, e, dims, bc, kappa)
    assert P._rel(got, Ae - w) < 1e-14


def check_clover_solve():
    for n, (dims, bc) in enumerate([((2, 2, 2, 2), (1, 1, 1, -1)),
                                     ((4, 2, 2, 4), (1, np.exp(0.2j), 1, -1))]):
        U, F = P._haar_links(dims, 580 + n), _F(dims, 585 + n, scale=0.3)
        b = P._source(dims, 590 + n)
        kappa = 0.12
        Dm = dense_clover(U, F, dims, bc, kappa)
        want = np.linalg.solve(Dm, b.reshape(-1))
        for eo in (False, True):
            x, info = oracle.clover_solve(U, F, b, dims, bc, kappa, eo=eo, tol=1e-12)
            assert info["status"] == 0, info
            assert P._rel(x.reshape(-1), want) < 1e-9, (dims, eo)
            r = b.reshape(-1) - Dm @ x.reshape(-1)
            dense_res = np.linalg.norm(r) / np.linalg.norm(b)
            got = oracle.clover_true_residual(U, F, b, x, dims, bc, kappa)
            assert abs(got - dense_res) <= 1e-3 * dense_res + 1e-16, (got, dense_res)


CLOVER_CHECKS = [check_clover_hermitian_blocks, check_clover_dense, check_clover_plane_wave,
                 check_clover_gamma5, check_clover_gauge_covariance, check_clover_inverse,
                 check_clover_schur, check_clover_solve]
