"""Checks that pin the FP64 oracle to facts other than itself.

Each ``check_*`` function raises ``AssertionError`` when the oracle disagrees
with what Eq. 1 and linear algebra fix.  They are run directly by
``test_oracle_pins.py`` and, against deliberately mutated builds of the
oracle source, by ``test_oracle_mutants.py`` (every planted mistake must make
at least one check fail).

What pins what:

* gamma table: Clifford algebra {g_mu, g_nu} = 2 delta, Hermiticity,
  g5 = g1 g2 g3 g4 = diag(1, 1, -1, -1) (the chiral basis the oracle states).
* H, D (Eq. 1): a dense 12V x 12V matrix assembled block by block from
  Eq. 1 with numpy kron on 2^4 and 4x2x2x4 lattices (L = 2 makes the +mu and
  -mu neighbours coincide, so the blocks must add); the free-field plane-wave
  closed form D e^{ipx} chi = e^{ipx} [1 - 2k sum cos p + 2ik sum g sin p] chi
  with periodic, antiperiodic and complex twisted phases; the free spectrum
  1 - 2k sum cos p +- 2ik |sin p|, each six-fold; gamma_5-hermiticity
  D^dag = g5 D g5; gauge covariance D[U^g] g psi = g D[U] psi; the norm bound
  ||H psi|| <= 8 ||psi|| with equality for the constant free field.
* D^dag: <phi, D psi> = <D^dag phi, psi>.
* even-odd: H_{p,1-p} is the parity block of the full-lattice H; M_ee equals
  the Schur complement D_ee - D_eo D_oo^{-1} D_oe composed from the full D.
* solves: true residual <= 1e-10; agreement with dense LU on 2^4; agreement
  with the closed-form free-field solution by 4D FFT with an antiperiodic
  twist; full and even-odd solves agree.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle
from paper_1811_00893_gb300 import fields

I4 = np.eye(4)
G5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)


def _haar_links(dims, seed):
    return fields.gauge_field(dims, "haar", seed).numpy()


def _unit_links(dims):
    return fields.gauge_field(dims, "unit", 0).numpy()


def _source(dims, seed, nrhs=1):
    s = fields.gaussian_fermion(dims, nrhs, seed).numpy()
    return s[0] if nrhs == 1 else s


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gammas():
    return [oracle.gamma(m) for m in range(4)]


# ----------------------------------------------------------------------------
# dense brute force
# ----------------------------------------------------------------------------

def dense_D(U, dims, bc, kappa, gam=None):
    """Dense D of Eq. 1 assembled block by block (contributions added)."""
    gam = gammas() if gam is None else gam
    V = int(np.prod(dims))
    c = fields.site_coords(dims)
    Dm = np.eye(12 * V, dtype=np.complex128)

    def idx(v):
        return int(v[0] + dims[0] * (v[1] + dims[1] * (v[2] + dims[2] * v[3])))

    for s in range(V):
        for mu in range(4):
            f = c[s].copy()
            f[mu] += 1
            crossed = f[mu] == dims[mu]
            f[mu] %= dims[mu]
            ph = bc[mu] if crossed else 1.0
            fi = idx(f)
            Dm[12 * s:12 * s + 12, 12 * fi:12 * fi + 12] += -kappa * ph * np.kron(I4 - gam[mu], U[s, mu])
            b = c[s].copy()
            b[mu] -= 1
            crossed = b[mu] < 0
            b[mu] %= dims[mu]
            ph = np.conj(bc[mu]) if crossed else 1.0
            bi = idx(b)
            Dm[12 * s:12 * s + 12, 12 * bi:12 * bi + 12] += (
                -kappa * ph * np.kron(I4 + gam[mu], U[bi, mu].conj().T))
    return Dm


def oracle_matrix(U, dims, bc, kappa):
    """The oracle's D as a dense matrix (applied to every unit vector)."""
    V = int(np.prod(dims))
    N = 12 * V
    M = np.empty((N, N), np.complex128)
    e = np.zeros((V, 4, 3), np.complex128)
    for j in range(N):
        e.reshape(-1)[:] = 0
        e.reshape(-1)[j] = 1
        M[:, j] = oracle.D_full(U, e, dims, bc, kappa).reshape(-1)
    return M


# ----------------------------------------------------------------------------
# checks
# ----------------------------------------------------------------------------

def check_gamma_algebra():
    g = gammas()
    for a, b in itertools.product(range(4), range(4)):
        ac = g[a] @ g[b] + g[b] @ g[a]
        assert np.allclose(ac, 2 * I4 * (a == b), atol=1e-15), f"Clifford fails for {a},{b}"
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=1e-15), f"gamma_{a} not Hermitian"
    assert np.allclose(g[0] @ g[1] @ g[2] @ g[3], G5, atol=1e-15), "gamma_5 != diag(1,1,-1,-1)"


def check_dense_bruteforce():
    cases = [((2, 2, 2, 2), (1, 1, 1, -1)),
             ((4, 2, 2, 4), (1, np.exp(0.7j), 1, -1)),
             ((2, 2, 2, 4), (1, 1, np.exp(-1.1j), 1))]
    for n, (dims, bc) in enumerate(cases):
        U = _haar_links(dims, 11 + n)
        psi = _source(dims, 21 + n)
        for kappa in (0.12, 0.31):
            Dm = dense_D(U, dims, bc, kappa)
            got = oracle.D_full(U, psi, dims, bc, kappa).reshape(-1)
            assert _rel(got, Dm @ psi.reshape(-1)) < 1e-14, f"dense mismatch {dims} k={kappa}"
            gotd = oracle.D_full(U, psi, dims, bc, kappa, dagger=True).reshape(-1)
            assert _rel(gotd, Dm.conj().T @ psi.reshape(-1)) < 1e-14, f"dense D^dag mismatch {dims}"


def _plane_wave(dims, p, chi):
    c = fields.site_coords(dims)
    ph = np.exp(1j * (c @ np.asarray(p)))
    return ph[:, None, None] * chi[None, :, :]


def check_free_field_plane_wave():
    g = gammas()
    rng = np.random.default_rng(7)
    dims = (4, 6, 4, 8)
    U = _unit_links(dims)
    for bc_theta in [(0, 0, 0, np.pi), (0.3, 0, -1.2, np.pi), (0, 0, 0, 0)]:
        bc = tuple(np.exp(1j * t) for t in bc_theta)
        for _ in range(4):
            n = [rng.integers(0, L) for L in dims]
            p = [(2 * np.pi * n[m] + bc_theta[m]) / dims[m] for m in range(4)]
            chi = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
            psi = _plane_wave(dims, p, chi)
            kappa = 0.13
            Mp = (1 - 2 * kappa * sum(np.cos(p))) * I4 + 2j * kappa * sum(
                np.sin(p[m]) * g[m] for m in range(4))
            want = _plane_wave(dims, p, Mp @ chi)
            got = oracle.D_full(U, psi, dims, bc, kappa)
            assert _rel(got, want) < 1e-13, f"plane wave mismatch p={p} bc={bc_theta}"


def check_free_spectrum():
    for dims, theta in [((2, 2, 2, 2), (0, 0, 0, np.pi)), ((4, 2, 2, 4), (0, 0, 0, np.pi)),
                        ((2, 2, 2, 4), (0, 0, 0, 0))]:
        kappa = 0.11
        bc = tuple(np.exp(1j * t) for t in theta)
        M = oracle_matrix(_unit_links(dims), dims, bc, kappa)
        ev = np.linalg.eigvals(M)
        pred = []
        for n in itertools.product(*[range(L) for L in dims]):
            p = [(2 * np.pi * n[m] + theta[m]) / dims[m] for m in range(4)]
            a = 1 - 2 * kappa * sum(np.cos(p))
            b = 2 * kappa * np.sqrt(sum(np.sin(q) ** 2 for q in p))
            pred += [a + 1j * b] * 6 + [a - 1j * b] * 6
        key = lambda z: (round(z.real, 9), round(z.imag, 9))
        got = sorted(ev, key=key)
        want = sorted(pred, key=key)
        assert np.max(np.abs(np.array(got) - np.array(want))) < 1e-12, f"spectrum {dims}"


def check_gamma5_hermiticity():
    dims, bc = (4, 4, 2, 4), (1, 1, 1, -1)
    U = _haar_links(dims, 31)
    phi, psi = _source(dims, 41), _source(dims, 42)
    kappa = 0.124

    def g5(f):
        return np.einsum("st,vtc->vsc", G5, f)

    lhs = np.vdot(phi, oracle.D_full(U, psi, dims, bc, kappa))
    rhs = np.vdot(g5(oracle.D_full(U, g5(phi), dims, bc, kappa)), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs), "gamma5-hermiticity fails"
    rhs_dag = np.vdot(oracle.D_full(U, phi, dims, bc, kappa, dagger=True), psi)
    assert abs(lhs - rhs_dag) < 1e-12 * abs(lhs), "<phi, D psi> != <D^dag phi, psi>"


def check_gauge_covariance():
    dims, bc = (4, 2, 4, 6), (1, np.exp(0.4j), 1, -1)
    U = _haar_links(dims, 51)
    psi = _source(dims, 52)
    g = fields.gauge_transform(dims, 53).numpy()
    c = fields.site_coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        f = c.copy()
        f[:, mu] = (f[:, mu] + 1) % dims[mu]
        fi = f[:, 0] + dims[0] * (f[:, 1] + dims[1] * (f[:, 2] + dims[2] * f[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ g[fi].conj().transpose(0, 2, 1)
    gpsi = np.einsum("vab,vsb->vsa", g, psi)
    for kappa in (0.12, 0.5):
        lhs = oracle.D_full(Ug, gpsi, dims, bc, kappa)
        rhs = np.einsum("vab,vsb->vsa", g, oracle.D_full(U, psi, dims, bc, kappa))
        assert _rel(lhs, rhs) < 1e-13, "gauge covariance fails"


def check_norm_bound():
    dims, bc = (4, 4, 4, 4), (1, 1, 1, -1)
    U = _haar_links(dims, 61)
    for seed in (62, 63):
        psi = _source(dims, seed)
        r = np.linalg.norm(oracle.hop_full(U, psi, dims, bc)) / np.linalg.norm(psi)
        assert r <= 8.0 + 1e-12 and r > 1.0, f"||H psi||/||psi|| = {r}"
    const = np.ones((int(np.prod(dims)), 4, 3), np.complex128)
    r = np.linalg.norm(oracle.hop_full(_unit_links(dims), const, dims, (1, 1, 1, 1)))
    assert abs(r / np.linalg.norm(const) - 8.0) < 1e-13, "free constant field must saturate ||H|| = 8"


def check_even_odd_blocks():
    dims, bc = (4, 2, 6, 4), (1, 1, np.exp(0.2j), -1)
    U = _haar_links(dims, 71)
    psi = _source(dims, 72)
    e, o = oracle.split(psi, dims)
    assert np.array_equal(oracle.join(e, o, dims), psi), "split/join round trip"
    # row i of the parity-p half is the site s of parity p with s // 2 == i
    c = fields.site_coords(dims)
    par = c.sum(1) % 2
    for p, half in ((0, e), (1, o)):
        sites = np.nonzero(par == p)[0]
        assert np.array_equal(sites // 2, np.arange(sites.size)), "half index must be s//2"
        assert np.array_equal(half, psi[sites]), "split picks the wrong sites"
    zero = np.zeros_like(e)
    for p in (0, 1):
        src_half = o if p == 0 else e
        full_in = oracle.join(zero, o, dims) if p == 0 else oracle.join(e, zero, dims)
        h = oracle.hop_full(U, full_in, dims, bc)
        he, ho = oracle.split(h, dims)
        got = oracle.hop_eo(U, src_half, dims, bc, p)
        assert _rel(got, he if p == 0 else ho) < 1e-15, f"H_(p,1-p) block p={p}"
        assert np.max(np.abs(ho if p == 0 else he)) == 0.0, "H must not connect equal parities"
        sites = np.array([0, 3, got.shape[0] - 1, 5])
        rows = oracle.hop_eo_sites(U, src_half, dims, bc, p, sites)
        assert _rel(rows, got[sites]) < 1e-15, "hop_eo_sites rows"


def check_schur_complement():
    dims, bc = (4, 4, 2, 4), (1, 1, 1, -1)
    U = _haar_links(dims, 81)
    psi = _source(dims, 82)
    kappa = 0.124
    e, _ = oracle.split(psi, dims)
    zero = np.zeros_like(e)
    # D_oe e = odd part of D (e, 0); D_eo y = even part of D (0, y); D_oo = 1
    _, y = oracle.split(oracle.D_full(U, oracle.join(e, zero, dims), dims, bc, kappa), dims)
    z, _ = oracle.split(oracle.D_full(U, oracle.join(zero, y, dims), dims, bc, kappa), dims)
    want = e - z  # D_ee e - D_eo D_oo^-1 D_oe e with D_ee = D_oo = 1
    got = oracle.Mee(U, e, dims, bc, kappa)
    assert _rel(got, want) < 1e-14, "M_ee is not the Schur complement of D"


def check_solve_dense_lu():
    dims, bc = (2, 2, 2, 2), (1, 1, 1, -1)
    U = _haar_links(dims, 91)
    b = _source(dims, 92)
    kappa = 0.12
    xd = np.linalg.solve(dense_D(U, dims, bc, kappa), b.reshape(-1)).reshape(b.shape)
    for eo in (False, True):
        x, info = oracle.solve(U, b, dims, bc, kappa, eo=eo, tol=1e-12)
        assert info["status"] == 0 and info["true_resid"] <= 1e-12, info
        assert _rel(x, xd) < 1e-10, f"solve (eo={eo}) != dense LU"


def check_solve_free_field_fft():
    dims, theta = (4, 4, 4, 8), np.array([0, 0, 0, np.pi])
    bc = tuple(np.exp(1j * t) for t in theta)
    kappa = 0.124
    b = _source(dims, 101)
    g = gammas()
    # x = sum_p e^{ipx} M(p)^{-1} beta(p) / V, p_mu = (2 pi n + theta)/L
    c = fields.site_coords(dims)
    twist = np.exp(-1j * (c @ (theta / np.array(dims))))
    bt = (b * twist[:, None, None]).reshape(dims[3], dims[2], dims[1], dims[0], 4, 3)
    beta = np.fft.fftn(bt, axes=(0, 1, 2, 3))
    n = np.stack(np.meshgrid(*[np.arange(L) for L in dims[::-1]], indexing="ij"), -1)[..., ::-1]
    p = (2 * np.pi * n + theta) / np.array(dims)
    a = 1 - 2 * kappa * np.cos(p).sum(-1)
    bm = 2 * kappa * np.sin(p)
    Minv = (a[..., None, None] * I4 - 1j * np.einsum("...m,mst->...st", bm, np.array(g)))
    Minv /= (a ** 2 + (bm ** 2).sum(-1))[..., None, None]
    xk = np.einsum("...st,...tc->...sc", Minv, beta)
    x_exact = (np.fft.ifftn(xk, axes=(0, 1, 2, 3)).reshape(-1, 4, 3)) / twist[:, None, None]
    U = _unit_links(dims)
    assert oracle.true_residual(U, b, x_exact, dims, bc, kappa) < 1e-12, "FFT solution wrong"
    for eo in (True, False):
        x, info = oracle.solve(U, b, dims, bc, kappa, eo=eo, tol=1e-11)
        assert info["true_resid"] <= 1e-11, info
        assert _rel(x, x_exact) < 1e-8, f"free-field solve (eo={eo}) != closed form"


def check_solve_eo_vs_full():
    dims, bc = (4, 4, 4, 4), (1, 1, 1, -1)
    U = fields.gauge_field(dims, "smooth", 111).numpy()
    b = _source(dims, 112)
    kappa = 0.124
    x1, i1 = oracle.solve(U, b, dims, bc, kappa, eo=False, tol=1e-10)
    x2, i2 = oracle.solve(U, b, dims, bc, kappa, eo=True, tol=1e-10)
    assert i1["true_resid"] <= 1e-10 and i2["true_resid"] <= 1e-10, (i1, i2)
    # cond(D) <= (1 + 8k)/(1 - 8k) bounds the forward error by cond * residual
    cond = (1 + 8 * kappa) / (1 - 8 * kappa)
    assert _rel(x1, x2) < 2 * cond * 1e-10, "eo and full solves disagree"
    r = oracle.true_residual(U, b, x2, dims, bc, kappa)
    assert abs(r - i2["true_resid"]) <= 1e-6 * r, "reported residual is not ||b - Dx||/||b||"


def check_reductions():
    """(a, b) = sum conj(a) b: closed forms (a, i a) = i ||a||^2 and
    (a, b) = conj((b, a)), and agreement with numpy's vdot."""
    a, b = _source((4, 2, 2, 2), 121), _source((4, 2, 2, 2), 122)
    n2 = float(np.sum(np.abs(a) ** 2))
    assert abs(oracle.cdot(a, 1j * a) - 1j * n2) < 1e-13 * n2, "(a, i a) != i ||a||^2"
    assert abs(oracle.cdot(a, b) - np.conj(oracle.cdot(b, a))) < 1e-13 * n2
    assert abs(oracle.cdot(a, b) - np.vdot(a, b)) < 1e-13 * n2


ALL_CHECKS = [
    check_gamma_algebra,
    check_reductions,
    check_dense_bruteforce,
    check_free_field_plane_wave,
    check_free_spectrum,
    check_gamma5_hermiticity,
    check_gauge_covariance,
    check_norm_bound,
    check_even_odd_blocks,
    check_schur_complement,
    check_solve_dense_lu,
    check_solve_free_field_fft,
    check_solve_eo_vs_full,
]


def failing_checks(checks=None):
    """Names of the checks that fail (used against mutated oracle builds)."""
    out = []
    for chk in (ALL_CHECKS if checks is None else checks):
        try:
            chk()
        except Exception:  # a mutant may also crash or raise
            out.append(chk.__name__)
    return out
