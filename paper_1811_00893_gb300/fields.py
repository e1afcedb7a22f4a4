"""Seeded synthetic inputs: SU(3) gauge links, Gaussian fermion sources,
random gauge transformations.

This module holds none of the Wilson-matrix arithmetic.  It only draws the
inputs that the GPU library and the CPU oracle are both handed, so the two
sides compare results on identical arrays.  Every generator takes an explicit
seed and a torch device; the same seed gives the same field on the same kind
of device (CPU and CUDA random streams differ, so a field drawn on the GPU is
copied to the host when the oracle needs it).

Layouts are the canonical ones (site index ``s = x + Lx*(y + Ly*(z + Lz*t))``):

* gauge field ``(V, 4, 3, 3)`` complex128, direction mu = 0..3 for x, y, z, t;
* fermion field ``(nrhs, V, 4, 3)`` complex128 (spin, colour).

Distributions (Sec. 2 names SU(3) links and 4x3 complex spinors; the paper
generates ensembles by Monte Carlo, which synthetic draws stand in for):

* ``haar``: Z = (N(0,1) + i N(0,1))/sqrt(2) per entry; the QR factor of Z with
  the diagonal of R made real positive (Gram-Schmidt) is Haar on U(3)
  (Mezzadri 2007); dividing by the principal cube root of its determinant
  gives det = 1;
* ``smooth``: U = exp(i eps A), A = sum_a omega_a lambda_a / 2 with
  omega_a ~ N(0,1) iid and lambda_a the Gell-Mann matrices, eps = 0.3;
* sources: every real and imaginary part N(0,1) iid.
"""
from __future__ import annotations

import math

import numpy as np
import torch

CHUNK = 1 << 22  # matrices per generation chunk (bounds device memory)


def generator(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def _cgauss(shape, gen, device) -> torch.Tensor:
    re = torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
    im = torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
    return torch.complex(re, im)


def _gram_schmidt(Z: torch.Tensor) -> torch.Tensor:
    c0, c1, c2 = Z[..., :, 0], Z[..., :, 1], Z[..., :, 2]

    def proj(q, v):
        return (q.conj() * v).sum(-1, keepdim=True) * q

    q0 = c0 / torch.linalg.vector_norm(c0, dim=-1, keepdim=True)
    v1 = c1 - proj(q0, c1)
    q1 = v1 / torch.linalg.vector_norm(v1, dim=-1, keepdim=True)
    v2 = c2 - proj(q0, c2)
    v2 = v2 - proj(q1, v2)
    q2 = v2 / torch.linalg.vector_norm(v2, dim=-1, keepdim=True)
    return torch.stack([q0, q1, q2], dim=-1)


def det3(M: torch.Tensor) -> torch.Tensor:
    """Determinant of each 3x3 matrix by cofactor expansion along the first row."""
    return (M[..., 0, 0] * (M[..., 1, 1] * M[..., 2, 2] - M[..., 1, 2] * M[..., 2, 1])
            - M[..., 0, 1] * (M[..., 1, 0] * M[..., 2, 2] - M[..., 1, 2] * M[..., 2, 0])
            + M[..., 0, 2] * (M[..., 1, 0] * M[..., 2, 1] - M[..., 1, 1] * M[..., 2, 0]))


def unitarise(Z: torch.Tensor) -> torch.Tensor:
    """Q factor of Z = QR with R's diagonal real positive (Gram-Schmidt on the
    columns, repeated once to restore orthogonality lost to rounding), then
    divided by the principal cube root of its determinant."""
    Q = _gram_schmidt(_gram_schmidt(Z))
    theta = torch.angle(det3(Q))
    return Q * torch.polar(torch.ones_like(theta), -theta / 3.0)[..., None, None]


def haar_su3(n: int, gen: torch.Generator, device="cpu") -> torch.Tensor:
    """n Haar-random SU(3) matrices, shape (n, 3, 3)."""
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    for a in range(0, n, CHUNK):
        b = min(n, a + CHUNK)
        Z = _cgauss((b - a, 3, 3), gen, device) / math.sqrt(2.0)
        out[a:b] = unitarise(Z)
    return out


def gell_mann(device="cpu") -> torch.Tensor:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / math.sqrt(3)
    l[7][2, 2] = -2 / math.sqrt(3)
    return torch.from_numpy(l).to(device)


def expm(X: torch.Tensor, order: int = 16) -> torch.Tensor:
    """exp of each 3x3 matrix: scale by 2^-k so that ||X||_F <= 1/2, Taylor
    series to `order` (truncation < 0.5^17/17! ~ 2e-20), square k times."""
    nrm = torch.linalg.vector_norm(X.reshape(X.shape[0], -1), dim=-1).max().item()
    k = max(0, int(math.ceil(math.log2(nrm / 0.5)))) if nrm > 0.5 else 0
    Y = X / (2.0 ** k)
    I = torch.eye(3, dtype=X.dtype, device=X.device).expand_as(X)
    term = I.clone()
    E = I.clone()
    for n in range(1, order + 1):
        term = torch.bmm(term, Y) / n
        E = E + term
    for _ in range(k):
        E = torch.bmm(E, E)
    return E


def smooth_su3(n: int, gen: torch.Generator, device="cpu", eps: float = 0.3) -> torch.Tensor:
    """n matrices exp(i eps A), A = sum_a omega_a lambda_a/2, shape (n, 3, 3)."""
    lam = gell_mann(device) / 2.0
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    for a in range(0, n, CHUNK):
        b = min(n, a + CHUNK)
        w = torch.randn((b - a, 8), generator=gen, dtype=torch.float64, device=device)
        A = torch.einsum("na,aij->nij", w.to(torch.complex128), lam)
        out[a:b] = unitarise(expm(1j * eps * A))
    return out


def volume(dims) -> int:
    return int(np.prod(dims))


def gauge_field(dims, kind: str, seed: int, device="cpu", eps: float = 0.3) -> torch.Tensor:
    """Canonical gauge field (V, 4, 3, 3): 'haar', 'smooth' or 'unit'."""
    V = volume(dims)
    if kind == "unit":
        return torch.eye(3, dtype=torch.complex128, device=device).expand(V, 4, 3, 3).clone()
    gen = generator(seed, device)
    if kind == "haar":
        U = haar_su3(4 * V, gen, device)
    elif kind == "smooth":
        U = smooth_su3(4 * V, gen, device, eps)
    else:
        raise ValueError(f"unknown link distribution {kind!r}")
    return U.reshape(V, 4, 3, 3)


def gaussian_fermion(dims, nrhs: int, seed: int, device="cpu") -> torch.Tensor:
    """nrhs Gaussian sources (nrhs, V, 4, 3); source j uses seed + j."""
    V = volume(dims)
    out = torch.empty((nrhs, V, 4, 3), dtype=torch.complex128, device=device)
    for j in range(nrhs):
        out[j] = _cgauss((V, 4, 3), generator(seed + j, device), device)
    return out


def clover_field(dims, seed: int, device="cpu", scale: float = 0.1) -> torch.Tensor:
    """Synthetic clover term F(x) of Eq. 2: two Hermitian 6x6 blocks per site,
    shape (V, 2, 6, 6), each scale * (Z + Z^dag)/2 with Z complex Gaussian of
    unit-variance entries / sqrt(6).  (The paper takes F as a precomputed
    input and ignores how it is built.)"""
    V = volume(dims)
    Z = _cgauss((V, 2, 6, 6), generator(seed, device), device) / math.sqrt(12.0)
    return scale * 0.5 * (Z + Z.conj().transpose(-1, -2))


def gauge_transform(dims, seed: int, device="cpu") -> torch.Tensor:
    """Haar-random g(x) in SU(3) per site, shape (V, 3, 3)."""
    return haar_su3(volume(dims), generator(seed, device), device)


def site_coords(dims) -> np.ndarray:
    """(V, 4) integer coordinates (x, y, z, t) of every canonical site index."""
    V = volume(dims)
    s = np.arange(V, dtype=np.int64)
    c = np.empty((V, 4), np.int64)
    for mu in range(4):
        c[:, mu] = s % dims[mu]
        s //= dims[mu]
    return c
