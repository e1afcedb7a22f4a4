"""FP64 CPU oracle for the Wilson matrix (Eq. 1) and its BiCGStab solve.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The GPU
library never imports it, and the two share no code: the oracle is the plain
C file ``wilson_oracle.c`` (one site at a time, literal 4x4 gamma and 3x3
colour products), loaded here through ctypes.

Every function takes and returns numpy ``complex128`` arrays in the
canonical layout:

* gauge field ``U``: shape ``(V, 4, 3, 3)``, site index
  ``s = x + Lx*(y + Ly*(z + Lz*t))``, direction ``mu = 0..3`` for x, y, z, t;
* fermion field: shape ``(V, 4, 3)`` (spin, colour);
* half field of parity ``p``: shape ``(V/2, 4, 3)``, row ``i`` holds the
  site ``s`` of parity ``p`` with ``s // 2 == i``.

``dims`` is ``(Lx, Ly, Lz, Lt)``; ``bc`` is four complex boundary phases.

Parity status of each function (what pins it) is listed in the module
docstrings of ``tests/test_oracle_*.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "wilson_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_SIG = {
    "orc_set_threads": (None, ["I"]),
    "orc_get_threads": ("I", []),
    "orc_gamma": (None, ["I", "P"]),
    "orc_hop_full": (None, ["P", "P", "P", "P", "P", "I"]),
    "orc_D_full": (None, ["P", "P", "P", "P", "P", "D", "I"]),
    "orc_hop_eo": (None, ["P", "P", "P", "P", "P", "I", "I"]),
    "orc_hop_eo_sites": (None, ["P", "P", "P", "P", "I", "I", "P", "L", "P"]),
    "orc_Mee": (None, ["P", "P", "P", "P", "P", "D", "I"]),
    "orc_split": (None, ["P", "P", "P", "P"]),
    "orc_join": (None, ["P", "P", "P", "P"]),
    "orc_norm2": ("D", ["L", "P"]),
    "orc_cdot": (None, ["L", "P", "P", "P"]),
    "orc_true_residual": ("D", ["P", "P", "P", "P", "P", "D"]),
    "orc_solve": ("I", ["P", "P", "P", "P", "P", "D", "I", "D", "I", "P", "P"]),
    "orc_bicgstab_fixed": ("I", ["P", "P", "P", "P", "P", "D", "I", "I"]),
    "orc_clover_true_residual": ("D", ["P", "P", "P", "P", "P", "P", "D"]),
    "orc_clover_solve": ("I", ["P", "P", "P", "P", "P", "P", "D", "I", "D", "I", "P", "P"]),
    "orc_clover_bicgstab_fixed": ("I", ["P", "P", "P", "P", "P", "P", "D", "I", "I"]),
    "orc_clover_D_full": (None, ["P", "P", "P", "P", "P", "P", "D", "I"]),
    "orc_clover_diag": (None, ["P", "P", "P", "P", "I", "I"]),
    "orc_clover_Mee": (None, ["P", "P", "P", "P", "P", "P", "D"]),
}
_CT = {"P": ctypes.c_void_p, "I": ctypes.c_int, "D": ctypes.c_double, "L": ctypes.c_long}


def compile_source(src_path: str, out_path: str) -> str:
    """Compile an oracle C source into a shared library with gcc (+OpenMP)."""
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", out_path, src_path, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    return out_path


def build(force: bool = False) -> str:
    """Compile ``wilson_oracle.c`` into ``liboracle.so``."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(SOURCE)):
        return _LIB
    return compile_source(SOURCE, _LIB)


def open_library(path: str):
    """Load an oracle shared library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIG.items():
        f = getattr(lib, name)
        f.restype = _CT[res] if res else None
        f.argtypes = [_CT[a] for a in args]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = open_library(build())
        return _lib


class use_library:
    """Context manager: route this module's functions through another build
    of the oracle source (the planted-mistake tests use it)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved, _lib = _lib, open_library(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dims(dims) -> np.ndarray:
    d = np.asarray(dims, dtype=np.int32)
    if d.shape != (4,) or np.any(d < 2) or d[0] % 2:
        raise ValueError(f"bad lattice extents {dims}: need 4 extents >= 2 with Lx even")
    return d


def _bc(bc) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(bc, dtype=np.complex128).reshape(4))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(dims) -> int:
    return int(np.prod(dims))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def gamma(mu: int) -> np.ndarray:
    """The oracle's gamma_mu (mu = 0..3 for x, y, z, t) as a 4x4 complex matrix."""
    out = np.zeros((4, 4), np.complex128)
    _load().orc_gamma(int(mu), _p(out))
    return out


def hop_full(U, psi, dims, bc, dagger: bool = False) -> np.ndarray:
    """H psi on the whole lattice (the hopping sum of Eq. 1); D^dag's if dagger."""
    d, b, U, psi = _dims(dims), _bc(bc), _c(U), _c(psi)
    out = np.empty_like(psi)
    _load().orc_hop_full(_p(U), _p(psi), _p(out), _p(d), _p(b), -1 if dagger else 1)
    return out


def D_full(U, psi, dims, bc, kappa: float, dagger: bool = False) -> np.ndarray:
    """D psi = psi - kappa H psi (Eq. 1); D^dag psi if dagger."""
    d, b, U, psi = _dims(dims), _bc(bc), _c(U), _c(psi)
    out = np.empty_like(psi)
    _load().orc_D_full(_p(U), _p(psi), _p(out), _p(d), _p(b), float(kappa),
                       -1 if dagger else 1)
    return out


def hop_eo(U, psi_half, dims, bc, out_parity: int, dagger: bool = False) -> np.ndarray:
    """H_{p,1-p} psi_{1-p}: parity-p half field from a parity-(1-p) half field."""
    d, b, U, psi = _dims(dims), _bc(bc), _c(U), _c(psi_half)
    out = np.empty_like(psi)
    _load().orc_hop_eo(_p(U), _p(psi), _p(out), _p(d), _p(b), int(out_parity),
                       -1 if dagger else 1)
    return out


def hop_eo_sites(U, psi_half, dims, bc, out_parity: int, sites, dagger: bool = False):
    """hop_eo evaluated only at the given half indices (rows in list order)."""
    d, b, U, psi = _dims(dims), _bc(bc), _c(U), _c(psi_half)
    idx = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.empty((idx.size, 4, 3), np.complex128)
    _load().orc_hop_eo_sites(_p(U), _p(psi), _p(d), _p(b), int(out_parity),
                             -1 if dagger else 1, _p(idx), idx.size, _p(out))
    return out


def Mee(U, psi_e, dims, bc, kappa: float, dagger: bool = False) -> np.ndarray:
    """Schur complement M_ee psi_e = psi_e - kappa^2 H_eo H_oe psi_e."""
    d, b, U, psi = _dims(dims), _bc(bc), _c(U), _c(psi_e)
    out = np.empty_like(psi)
    _load().orc_Mee(_p(U), _p(psi), _p(out), _p(d), _p(b), float(kappa),
                    -1 if dagger else 1)
    return out


def split(psi, dims):
    """Full field -> (even half, odd half)."""
    d, psi = _dims(dims), _c(psi)
    Vh = psi.shape[0] // 2
    e = np.empty((Vh, 4, 3), np.complex128)
    o = np.empty((Vh, 4, 3), np.complex128)
    _load().orc_split(_p(d), _p(psi), _p(e), _p(o))
    return e, o


def join(even, odd, dims):
    """(even half, odd half) -> full field."""
    d, e, o = _dims(dims), _c(even), _c(odd)
    out = np.empty((2 * e.shape[0], 4, 3), np.complex128)
    _load().orc_join(_p(d), _p(e), _p(o), _p(out))
    return out


def cdot(a, b) -> complex:
    """(a, b) = sum conj(a) b."""
    a, b = _c(a), _c(b)
    out = np.zeros(2, np.float64)
    _load().orc_cdot(a.size, _p(a), _p(b), _p(out))
    return complex(out[0], out[1])


def true_residual(U, b, x, dims, bc, kappa: float) -> float:
    """||b - D x||_2 / ||b||_2 on the full lattice."""
    d, bb, U, b, x = _dims(dims), _bc(bc), _c(U), _c(b), _c(x)
    return float(_load().orc_true_residual(_p(U), _p(b), _p(x), _p(d), _p(bb), float(kappa)))


def solve(U, b, dims, bc, kappa: float, eo: bool = True, tol: float = 1e-10,
          maxiter: int = 10000, x0=None):
    """Solve D x = b by BiCGStab (full or even-odd); returns (x, info dict)."""
    d, bb, U, b = _dims(dims), _bc(bc), _c(U), _c(b)
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    info = np.zeros(4, np.int32)
    res = np.zeros(1, np.float64)
    rc = _load().orc_solve(_p(U), _p(b), _p(x), _p(d), _p(bb), float(kappa), int(bool(eo)),
                           float(tol), int(maxiter), _p(info), _p(res))
    return x, {"status": int(rc), "iters": int(info[0]), "restarts": int(info[1]),
               "bicgstab_status": int(info[2]), "passes": int(info[3]),
               "true_resid": float(res[0])}


def bicgstab_fixed(U, b_sys, dims, bc, kappa: float, eo: bool, niter: int):
    """Exactly ``niter`` BiCGStab iterations on D (eo=False) or M_ee (eo=True)
    from x = 0; returns x.  For timing a bounded sample of a long solve."""
    d, bb, U, b = _dims(dims), _bc(bc), _c(U), _c(b_sys)
    x = np.zeros_like(b)
    _load().orc_bicgstab_fixed(_p(U), _p(b), _p(x), _p(d), _p(bb), float(kappa),
                               int(bool(eo)), int(niter))
    return x


# ---------------------------------------------------------------------------
# clover term (Eq. 2): F has shape (V, 2, 6, 6), block b acting on spins
# {2b, 2b+1} x colour, row index local_spin*3 + colour
# ---------------------------------------------------------------------------

def clover_D_full(U, F, psi, dims, bc, kappa: float, dagger: bool = False) -> np.ndarray:
    """D_clov psi = D_W psi + F psi (Eq. 2)."""
    d, b, U, F, psi = _dims(dims), _bc(bc), _c(U), _c(F), _c(psi)
    out = np.empty_like(psi)
    _load().orc_clover_D_full(_p(U), _p(F), _p(psi), _p(out), _p(d), _p(b), float(kappa),
                              -1 if dagger else 1)
    return out


def clover_diag(F, psi_half, dims, parity: int, inverse: bool = False) -> np.ndarray:
    """(1 + F) psi or (1 + F)^{-1} psi on the sites of one parity."""
    d, F, psi = _dims(dims), _c(F), _c(psi_half)
    out = np.empty_like(psi)
    _load().orc_clover_diag(_p(F), _p(psi), _p(out), _p(d), int(parity), int(bool(inverse)))
    return out


def clover_Mee(U, F, psi_e, dims, bc, kappa: float) -> np.ndarray:
    """Schur complement A_ee - kappa^2 H_eo A_oo^{-1} H_oe with A = 1 + F."""
    d, b, U, F, psi = _dims(dims), _bc(bc), _c(U), _c(F), _c(psi_e)
    out = np.empty_like(psi)
    _load().orc_clover_Mee(_p(U), _p(F), _p(psi), _p(out), _p(d), _p(b), float(kappa))
    return out


def clover_true_residual(U, F, b, x, dims, bc, kappa: float) -> float:
    """||b - D_clov x||_2 / ||b||_2 on the full lattice."""
    d, bb, U, F, b, x = _dims(dims), _bc(bc), _c(U), _c(F), _c(b), _c(x)
    return float(_load().orc_clover_true_residual(_p(U), _p(F), _p(b), _p(x), _p(d), _p(bb),
                                                  float(kappa)))


def clover_solve(U, F, b, dims, bc, kappa: float, eo: bool = True, tol: float = 1e-10,
                 maxiter: int = 10000, x0=None):
    """Solve D_clov x = b by BiCGStab (full or even-odd Schur system)."""
    d, bb, U, F, b = _dims(dims), _bc(bc), _c(U), _c(F), _c(b)
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    info = np.zeros(4, np.int32)
    res = np.zeros(1, np.float64)
    rc = _load().orc_clover_solve(_p(U), _p(F), _p(b), _p(x), _p(d), _p(bb), float(kappa),
                                  int(bool(eo)), float(tol), int(maxiter), _p(info), _p(res))
    return x, {"status": int(rc), "iters": int(info[0]), "restarts": int(info[1]),
               "bicgstab_status": int(info[2]), "passes": int(info[3]),
               "true_resid": float(res[0])}


def clover_bicgstab_fixed(U, F, b_sys, dims, bc, kappa: float, eo: bool, niter: int):
    """Exactly ``niter`` BiCGStab iterations on D_clov or its Schur complement."""
    d, bb, U, F, b = _dims(dims), _bc(bc), _c(U), _c(F), _c(b_sys)
    x = np.zeros_like(b)
    _load().orc_clover_bicgstab_fixed(_p(U), _p(F), _p(b), _p(x), _p(d), _p(bb), float(kappa),
                                      int(bool(eo)), int(niter))
    return x
