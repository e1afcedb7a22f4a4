"""Input generators: unitarity, det = 1, Haar moments, smooth-link statistics.

Haar on SU(3) has E[Tr U] = 0, E[|Tr U|^2] = 1 and E[(Tr U)^3] = 1 (one
singlet in 3 x 3 x 3); a U(3)-Haar draw without the determinant fix would
give E[(Tr U)^3] = 0, so the last moment pins the det = 1 step.  The smooth
links exp(i eps A) with A = sum omega_a lambda_a / 2 have
E[Re Tr U]/3 = 1 - eps^2 E[Tr A^2]/6 + O(eps^4) with E[Tr A^2] = 4.
"""
import numpy as np
import torch

from paper_1811_00893_gb300 import fields, workloads


def _unitarity(U):
    I = torch.eye(3, dtype=U.dtype)
    err_u = (U.conj().transpose(-1, -2) @ U - I).abs().amax().item()
    err_d = (torch.linalg.det(U) - 1).abs().amax().item()
    return err_u, err_d


def test_haar_su3_unitary_det1():
    U = fields.haar_su3(20000, fields.generator(3))
    eu, ed = _unitarity(U)
    assert eu < 1e-14 and ed < 1e-14


def test_haar_moments():
    U = fields.haar_su3(200000, fields.generator(4))
    tr = torch.diagonal(U, dim1=-2, dim2=-1).sum(-1).numpy()
    assert abs(tr.mean()) < 0.01
    assert abs(np.mean(np.abs(tr) ** 2) - 1.0) < 0.02
    assert abs(np.mean(tr ** 3) - 1.0) < 0.05


def test_smooth_links():
    U = fields.smooth_su3(100000, fields.generator(5), eps=0.3)
    eu, ed = _unitarity(U)
    assert eu < 1e-14 and ed < 1e-14
    m = torch.diagonal(U, dim1=-2, dim2=-1).sum(-1).real.mean().item() / 3
    assert abs(m - (1 - 0.09 * 4 / 6)) < 0.003
    gm = fields.gell_mann()
    tr = torch.einsum("aij,bji->ab", gm, gm)
    assert torch.allclose(tr, 2 * torch.eye(8, dtype=tr.dtype), atol=1e-14)


def test_expm_matches_library_exponential():
    w = torch.randn((2000, 8), generator=fields.generator(7), dtype=torch.float64)
    A = torch.einsum("na,aij->nij", w.to(torch.complex128), fields.gell_mann() / 2)
    for eps in (0.3, 3.0):
        X = 1j * eps * A
        assert torch.allclose(fields.expm(X), torch.linalg.matrix_exp(X), rtol=0, atol=1e-13)


def test_det3_matches_library_determinant():
    Z = fields._cgauss((1000, 3, 3), fields.generator(6), "cpu")
    assert torch.allclose(fields.det3(Z), torch.linalg.det(Z), rtol=1e-12, atol=1e-12)


def test_seeded_reproducible():
    a = fields.gauge_field((4, 2, 2, 2), "haar", 9)
    b = fields.gauge_field((4, 2, 2, 2), "haar", 9)
    assert torch.equal(a, b)
    s = fields.gaussian_fermion((4, 2, 2, 2), 3, 17)
    assert torch.equal(s[1], fields.gaussian_fermion((4, 2, 2, 2), 1, 18)[0])
    assert abs(s.real.std().item() - 1) < 0.15 and abs(s.imag.std().item() - 1) < 0.15


def test_uneven_batch_spec():
    b = workloads.uneven_batch()
    assert len(b) == 16
    assert all(m.dims in workloads.BATCH_SHAPES and 1 <= m.nrhs <= 8 for m in b)
    assert all(0.11 <= m.kappa <= 0.124 for m in b)
    assert workloads.uneven_batch() == b
