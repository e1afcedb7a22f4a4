"""Helpers shared by the GPU parity tests: build a gauge object from seeded
fields, move fermion fields between the canonical layout and the library's
internal layout through the C ABI, and relative-error measures."""
from __future__ import annotations

import numpy as np
import torch

from paper_1811_00893_gb300 import fields, wilson

PRECS = {"f64": wilson.WL_F64, "f32": wilson.WL_F32, "f16": wilson.WL_F16,
         "df64": wilson.WL_DF64}

# Relative L2 tolerances against the FP64 oracle.  FP64 and FP32 are the
# stated targets.  FP16 storage: test_gpu_parity.test_fp16_error_margins
# measures the hopping term, D and M_ee in FP16 on every parity lattice
# (Haar and smooth links, both parities and signs): the worst relative error
# is 3.5e-4 (the per-component binary16 rounding, 2^-12 of the site scale,
# over 24 components and eight hops adds incoherently to ~3e-4); the bound is
# twice that.  df64 (hi + lo FP32 pairs): inputs carry <= 2^-48 relative
# rounding, each df64 add or multiply <= 2^-44 (5.7e-14), and an output
# component takes ~100 dependent operations, so <= 5.7e-12; 1e-11.
TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 7e-4, "df64": 1e-11}


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Case:
    """A seeded lattice: canonical links on host and device, a gauge object."""

    def __init__(self, dims, kappa=0.12, kind="haar", seed=1, bc=(1, 1, 1, -1),
                 precs=("f64", "f32", "f16"), device_gen=False, r12=False, r8=False):
        self.dims = tuple(dims)
        self.kappa = kappa
        self.bc = bc
        dev = "cuda" if device_gen else "cpu"
        U = fields.gauge_field(dims, kind, seed, device=dev)
        self.U_dev = U.to("cuda").contiguous()
        self.U = U.cpu().numpy()
        self.g = wilson.Gauge(dims, kappa, self.U_dev, precs=precs, bc=bc, r12=r12, r8=r8)
        self.V = int(np.prod(dims))
        self.Vh = self.V // 2

    def source(self, nrhs=1, seed=100, device_gen=False):
        dev = "cuda" if device_gen else "cpu"
        return fields.gaussian_fermion(self.dims, nrhs, seed, device=dev).to("cuda").contiguous()

    def to_internal(self, psi_dev, parity, prec, nrhs=None):
        nrhs = psi_dev.shape[0] if nrhs is None else nrhs
        out = self.g.field(prec, nrhs)
        wilson.wl_field_to_internal(self.g.handle, out, psi_dev, parity, PRECS[prec], nrhs)
        return out

    def to_canonical(self, internal, parity, prec, nrhs=1, fill=None):
        out = torch.zeros((nrhs, self.V, 4, 3), dtype=torch.complex128, device="cuda") \
            if fill is None else fill
        wilson.wl_field_to_canonical(self.g.handle, out, internal, parity, PRECS[prec], nrhs)
        return out

    def half(self, canon_dev, parity, r=0):
        """Canonical half field (numpy) of one right-hand side."""
        import oracle
        e, o = oracle.split(canon_dev[r].cpu().numpy(), self.dims)
        return e if parity == 0 else o

    def close(self):
        self.g.close()
