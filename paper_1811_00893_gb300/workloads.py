"""The synthetic workloads the library is measured and parity-tested on.

Each workload is a lattice size, a hopping parameter, a link distribution,
a number of right-hand sides and the precision scheme of the solve (and, for
the clover workload, the synthetic clover field of fields.clover_field).
Seeds: gauge field 1000 + workload index, sources 2000 + workload index + RHS
index, clover field 3000 + workload index, uneven batch 5005.  Boundary phases are periodic in space and antiperiodic in
time (Sec. 2 allows either condition per direction).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BC_PPPA = (1.0, 1.0, 1.0, -1.0)


@dataclass(frozen=True)
class Workload:
    index: int
    name: str
    dims: tuple
    kappa: float
    links: str          # 'haar' or 'smooth'
    nrhs: int
    eo: bool
    scheme: str         # 'fp64', 'fp32-defect-correction', 'fp16-reliable', 'fp32-multirhs'
    bc: tuple = BC_PPPA
    clover: bool = False  # D_clov of Eq. 2 with the synthetic clover field

    @property
    def volume(self) -> int:
        return int(np.prod(self.dims))

    @property
    def gauge_seed(self) -> int:
        return 1000 + self.index

    @property
    def source_seed(self) -> int:
        return 2000 + self.index

    @property
    def clover_seed(self) -> int:
        return 3000 + self.index


WORKLOADS = [
    Workload(0, "8^4 FP64 full D, Haar links", (8, 8, 8, 8), 0.12, "haar", 1, False, "fp64"),
    Workload(1, "32^3x64 even-odd, FP32 inner BiCGStab, FP64 defect correction",
             (32, 32, 32, 64), 0.124, "smooth", 1, True, "fp32-defect-correction"),
    Workload(2, "48^3x96 even-odd, FP16 storage + per-site norm, FP64 reliable updates",
             (48, 48, 48, 96), 0.124, "smooth", 1, True, "fp16-reliable"),
    Workload(3, "24^3x48 even-odd, 12 RHS multi-RHS FP32, FP64 refinement",
             (24, 24, 24, 48), 0.12, "haar", 12, True, "fp32-multirhs"),
    # index 4 is the uneven multi-lattice batch (uneven_batch below)
    Workload(5, "32^3x64 even-odd clover (Eq. 2), FP32 inner BiCGStab, FP64 defect correction",
             (32, 32, 32, 64), 0.124, "smooth", 1, True, "fp32-defect-correction", clover=True),
]


def by_index(index: int) -> Workload:
    """The single-lattice workload with this index."""
    for w in WORKLOADS:
        if w.index == index:
            return w
    raise KeyError(f"no single-lattice workload {index}")

BATCH_SHAPES = [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), (16, 16, 16, 16)]


@dataclass(frozen=True)
class BatchMember:
    dims: tuple
    nrhs: int
    kappa: float
    gauge_seed: int
    source_seed: int


def uneven_batch(seed: int = 5005, n: int = 16):
    """16 independent lattices: extents uniform over BATCH_SHAPES, 1-8 RHS
    each, kappa uniform in [0.11, 0.124], Haar links."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        dims = BATCH_SHAPES[int(rng.integers(0, len(BATCH_SHAPES)))]
        nrhs = int(rng.integers(1, 9))
        kappa = float(rng.uniform(0.11, 0.124))
        out.append(BatchMember(dims, nrhs, kappa, seed * 10 + i, seed * 100 + 16 * i))
    return out
