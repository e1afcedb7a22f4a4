"""Python binding of the C ABI in ``include/wilson.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: tensors are passed as raw device (or host) pointers,
the CUDA stream defaults to torch's current stream, and a negative status
raises ``WilsonError`` with the library's message.  PyTorch supplies device
memory and streams; all computation runs in ``libwilson.so``.  There is no
CPU fallback: if the CUDA library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

WL_F64, WL_F32, WL_F16, WL_DF64 = 0, 1, 2, 3
PREC = {"f64": WL_F64, "f32": WL_F32, "f16": WL_F16, "df64": WL_DF64}
WL_OK, WL_ERR_ARG, WL_ERR_CUDA, WL_ERR_NOT_CONVERGED = 0, -1, -2, -3
WL_ERR_BREAKDOWN, WL_ERR_NAN, WL_ERR_STATE = -4, -5, -7
ERR_NAMES = {0: "WL_OK", -1: "WL_ERR_ARG", -2: "WL_ERR_CUDA", -3: "WL_ERR_NOT_CONVERGED",
             -4: "WL_ERR_BREAKDOWN", -5: "WL_ERR_NAN", -7: "WL_ERR_STATE"}


#: wl_gauge_create flag: also keep two-row (reconstruct-12) FP32/FP16 links
WL_LINKS_R12 = 1 << 8
WL_LINKS_R8 = 1 << 9


def prec_mask(*precs) -> int:
    m = 0
    for p in precs:
        m |= 1 << (PREC[p] if isinstance(p, str) else int(p))
    return m


class WilsonError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class wl_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("kappa", ctypes.c_double),
                ("bc_re", ctypes.c_double * 4), ("bc_im", ctypes.c_double * 4)]


class wl_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("eo", ctypes.c_int),
                ("inner", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("delta", ctypes.c_double), ("use_x0", ctypes.c_int),
                ("graph_iters", ctypes.c_int)]


class wl_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("restarts", ctypes.c_int),
                ("status", ctypes.c_int), ("true_resid", ctypes.c_double),
                ("secs", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
LIB_PATH = _build.LIB


def load() -> ctypes.CDLL:
    """Load libwilson.so (building it first if its sources are newer).  The
    environment variable WL_LIBRARY names another build of it to load instead
    (a build variant; it is not rebuilt)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("WL_LIBRARY") or LIB_PATH
        if path == LIB_PATH and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, I, D, LL, SZ = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                           ctypes.c_size_t)
        sig = {
            "wl_gauge_create": (I, [ctypes.POINTER(P), ctypes.POINTER(wl_lattice), P, I, P]),
            "wl_gauge_destroy": (I, [P]),
            "wl_half_volume": (LL, [P]),
            "wl_field_bytes": (SZ, [P, I, I]),
            "wl_field_to_internal": (I, [P, P, P, I, I, I, P]),
            "wl_field_to_canonical": (I, [P, P, P, I, I, I, P]),
            "wilson_dslash": (I, [P, P, P, I, I, I, I, P]),
            "wilson_mult": (I, [P, P, P, I, I, I, I, P]),
            "wl_clover_set": (I, [P, P, P]),
            "wl_clover_apply": (I, [P, P, P, I, I, I, I, P]),
            "wl_cdot": (I, [P, P, P, P, I, I, P]),
            "wl_cdot_noalloc": (I, [P, P, P, LL, I, I, P]),
            "wilson_solve": (I, [P, P, P, I, ctypes.POINTER(wl_solve_params),
                                 ctypes.POINTER(wl_solve_info), P]),
            "wilson_solve_batch": (I, [I, P, P, P, P, ctypes.POINTER(wl_solve_params),
                                       ctypes.POINTER(wl_solve_info), P]),
            "wl_dd_create": (I, [ctypes.POINTER(P), ctypes.POINTER(wl_lattice), ctypes.POINTER(I), P, I, P]),
            "wl_dd_create_part": (I, [ctypes.POINTER(P), ctypes.POINTER(wl_lattice), ctypes.POINTER(I),
                                      I, I, P, I, P, P]),
            "wl_dd_plan": (I, [ctypes.POINTER(I), ctypes.POINTER(I), I, I, I, I, P, I]),
            "wl_dd_destroy": (I, [P]),
            "wl_dd_blocks": (I, [P]),
            "wl_dd_block": (I, [P, I, ctypes.POINTER(P), ctypes.POINTER(I)]),
            "wl_dd_set_exchange": (I, [P, I]),
            "wl_dd_scatter": (I, [P, P, P, I, P]),
            "wl_dd_gather": (I, [P, P, P, I, P]),
            "wl_dd_clover_set": (I, [P, P, P]),
            "wilson_dslash_dd": (I, [P, P, P, I, I, I, I, P]),
            "wilson_mult_dd": (I, [P, P, P, I, I, I, I, P]),
            "wl_cdot_dd": (I, [P, P, P, P, I, I, P]),
            "wilson_solve_dd": (I, [P, P, P, I, ctypes.POINTER(wl_solve_params),
                                    ctypes.POINTER(wl_solve_info), P]),
            "wl_last_error": (ctypes.c_char_p, []),
            "wl_spinor16_format": (I, []),
            "wl_launch_count": (LL, []),
            "wl_algorithmic_bytes": (D, []),
            "wl_timing": (I, [P, I]),
            "wl_timing_read": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(LL), ctypes.POINTER(D)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return ["wl_gauge_create", "wl_gauge_destroy", "wl_half_volume", "wl_field_bytes",
            "wl_field_to_internal", "wl_field_to_canonical", "wilson_dslash", "wilson_mult",
            "wl_clover_set", "wl_clover_apply", "wl_cdot", "wl_cdot_noalloc", "wilson_solve",
            "wilson_solve_batch", "wl_dd_create", "wl_dd_create_part", "wl_dd_plan", "wl_dd_destroy", "wl_dd_blocks", "wl_dd_block",
            "wl_dd_set_exchange", "wl_dd_scatter", "wl_dd_gather", "wl_dd_clover_set", "wilson_dslash_dd",
            "wilson_mult_dd", "wl_cdot_dd", "wilson_solve_dd", "wl_last_error",
            "wl_spinor16_format",
            "wl_launch_count", "wl_algorithmic_bytes", "wl_timing", "wl_timing_read"]


def _check(rc: int) -> int:
    if rc < 0:
        raise WilsonError(rc, load().wl_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):  # numpy array
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def lattice(dims, kappa, bc=(1, 1, 1, -1)) -> wl_lattice:
    lat = wl_lattice()
    for k in range(4):
        lat.dims[k] = int(dims[k])
        z = complex(bc[k])
        lat.bc_re[k] = z.real
        lat.bc_im[k] = z.imag
    lat.kappa = float(kappa)
    return lat


def wl_gauge_create(lat: wl_lattice, U: torch.Tensor, mask: int, stream=None) -> ctypes.c_void_p:
    g = ctypes.c_void_p()
    _check(load().wl_gauge_create(ctypes.byref(g), ctypes.byref(lat), _ptr(U), int(mask),
                                  _stream(stream)))
    return g


def wl_gauge_destroy(g) -> None:
    _check(load().wl_gauge_destroy(g))


def wl_half_volume(g) -> int:
    return int(load().wl_half_volume(g))


def wl_field_bytes(g, prec: int, nrhs: int) -> int:
    return int(load().wl_field_bytes(g, int(prec), int(nrhs)))


def wl_field_to_internal(g, out, inp, parity: int, prec: int, nrhs: int, stream=None) -> None:
    _check(load().wl_field_to_internal(g, _ptr(out), _ptr(inp), int(parity), int(prec),
                                       int(nrhs), _stream(stream)))


def wl_field_to_canonical(g, out, inp, parity: int, prec: int, nrhs: int, stream=None) -> None:
    _check(load().wl_field_to_canonical(g, _ptr(out), _ptr(inp), int(parity), int(prec),
                                        int(nrhs), _stream(stream)))


def wilson_dslash(g, out, inp, out_parity: int, dagger: int, prec: int, nrhs: int,
                  stream=None) -> None:
    _check(load().wilson_dslash(g, _ptr(out), _ptr(inp), int(out_parity), int(dagger),
                                int(prec), int(nrhs), _stream(stream)))


def wilson_mult(g, out, inp, eo: int, dagger: int, prec: int, nrhs: int, stream=None) -> None:
    _check(load().wilson_mult(g, _ptr(out), _ptr(inp), int(eo), int(dagger), int(prec),
                              int(nrhs), _stream(stream)))


def wl_clover_set(g, F, stream=None) -> None:
    """Attach the clover term F (device FP64 [V][2][6][6] complex; None detaches)."""
    _check(load().wl_clover_set(g, _ptr(F), _stream(stream)))


def wl_clover_apply(g, out, inp, parity: int, inverse: int, prec: int, nrhs: int,
                    stream=None) -> None:
    _check(load().wl_clover_apply(g, _ptr(out), _ptr(inp), int(parity), int(inverse), int(prec),
                                  int(nrhs), _stream(stream)))


def wl_cdot(g, out, a, b, prec: int, nrhs: int, stream=None) -> None:
    _check(load().wl_cdot(g, _ptr(out), _ptr(a), _ptr(b), int(prec), int(nrhs), _stream(stream)))


def wl_cdot_noalloc(out, a, b, Vh: int, prec: int, nrhs: int, stream=None) -> None:
    """wl_cdot for callers that cannot allocate device memory (fixed built-in
    scratch, at most 64 right-hand sides, concurrent calls race)."""
    _check(load().wl_cdot_noalloc(_ptr(out), _ptr(a), _ptr(b), int(Vh), int(prec), int(nrhs),
                                  _stream(stream)))


def solve_params(tol=1e-10, maxiter=20000, eo=True, inner=WL_F64, inner_tol=0.0, delta=0.0,
                 use_x0=False, graph_iters=0) -> wl_solve_params:
    p = wl_solve_params()
    p.tol, p.maxiter, p.eo, p.inner = float(tol), int(maxiter), int(bool(eo)), int(inner)
    p.inner_tol, p.delta, p.use_x0 = float(inner_tol), float(delta), int(bool(use_x0))
    p.graph_iters = int(graph_iters)
    return p


def _infos(arr, n):
    return [{"iters": arr[k].iters, "outer": arr[k].outer, "restarts": arr[k].restarts,
             "status": arr[k].status, "true_resid": arr[k].true_resid, "secs": arr[k].secs}
            for k in range(n)]


def wilson_solve(g, x, b, nrhs: int, params: wl_solve_params, stream=None, check=True):
    """Returns (status, [info per rhs]); raises on failure when check is set."""
    info = (wl_solve_info * nrhs)()
    rc = load().wilson_solve(g, _ptr(x), _ptr(b), int(nrhs), ctypes.byref(params), info,
                             _stream(stream))
    if check:
        _check(rc)
    return rc, _infos(info, nrhs)


def wilson_solve_batch(gs, xs, bs, nrhs, params: wl_solve_params, stream=None, check=True):
    n = len(gs)
    G = (ctypes.c_void_p * n)(*[g.value for g in gs])
    X = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs])
    B = (ctypes.c_void_p * n)(*[t.data_ptr() for t in bs])
    R = (ctypes.c_int * n)(*[int(k) for k in nrhs])
    total = sum(int(k) for k in nrhs)
    info = (wl_solve_info * total)()
    rc = load().wilson_solve_batch(n, G, X, B, R, ctypes.byref(params), info, _stream(stream))
    if check:
        _check(rc)
    return rc, _infos(info, total)


# ---------------------------------------------------------------------------
# domain decomposition (block fields are passed as lists, one per block)
# ---------------------------------------------------------------------------

def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[_ptr(t).value for t in ts])


def wl_dd_create(lat: wl_lattice, grid, U: torch.Tensor, mask: int, stream=None) -> ctypes.c_void_p:
    dd = ctypes.c_void_p()
    G = (ctypes.c_int * 4)(*[int(k) for k in grid])
    _check(load().wl_dd_create(ctypes.byref(dd), ctypes.byref(lat), G, _ptr(U), int(mask),
                               _stream(stream)))
    return dd


def wl_dd_create_part(lat: wl_lattice, grid, first: int, count: int, U: torch.Tensor, mask: int,
                      transport=None, stream=None) -> ctypes.c_void_p:
    """transport: a dd_transport.wl_dd_transport (or None when every block is held)."""
    dd = ctypes.c_void_p()
    G = (ctypes.c_int * 4)(*[int(k) for k in grid])
    tp = ctypes.cast(ctypes.byref(transport), ctypes.c_void_p) if transport is not None else None
    _check(load().wl_dd_create_part(ctypes.byref(dd), ctypes.byref(lat), G, int(first), int(count),
                                    _ptr(U), int(mask), tp, _stream(stream)))
    return dd


def wl_dd_destroy(dd) -> None:
    _check(load().wl_dd_destroy(dd))


def wl_dd_blocks(dd) -> int:
    return int(load().wl_dd_blocks(dd))


def wl_dd_block(dd, k: int):
    """(gauge handle, grid coordinates) of block k."""
    g = ctypes.c_void_p()
    c = (ctypes.c_int * 4)()
    _check(load().wl_dd_block(dd, int(k), ctypes.byref(g), c))
    return g, tuple(c)


def wl_dd_set_exchange(dd, mode: int) -> None:
    _check(load().wl_dd_set_exchange(dd, int(mode)))


def wl_dd_scatter(dd, local, glob, nrhs: int, stream=None) -> None:
    _check(load().wl_dd_scatter(dd, _ptrs(local), _ptr(glob), int(nrhs), _stream(stream)))


def wl_dd_gather(dd, glob, local, nrhs: int, stream=None) -> None:
    _check(load().wl_dd_gather(dd, _ptr(glob), _ptrs(local), int(nrhs), _stream(stream)))


def wl_dd_clover_set(dd, F, stream=None) -> None:
    """Attach the clover term F of the whole lattice to every held block (None detaches)."""
    _check(load().wl_dd_clover_set(dd, _ptr(F), _stream(stream)))


def wilson_dslash_dd(dd, out, inp, out_parity: int, dagger: int, prec: int, nrhs: int,
                     stream=None) -> None:
    _check(load().wilson_dslash_dd(dd, _ptrs(out), _ptrs(inp), int(out_parity), int(dagger),
                                   int(prec), int(nrhs), _stream(stream)))


def wilson_mult_dd(dd, out, inp, eo: int, dagger: int, prec: int, nrhs: int, stream=None) -> None:
    _check(load().wilson_mult_dd(dd, _ptrs(out), _ptrs(inp), int(eo), int(dagger), int(prec),
                                 int(nrhs), _stream(stream)))


def wl_cdot_dd(dd, out, a, b, prec: int, nrhs: int, stream=None) -> None:
    _check(load().wl_cdot_dd(dd, _ptr(out), _ptrs(a), _ptrs(b), int(prec), int(nrhs),
                             _stream(stream)))


def wilson_solve_dd(dd, xs, bs, nrhs: int, params: wl_solve_params, stream=None, check=True):
    """Returns (status, [info per rhs]); xs, bs: block-local canonical fields."""
    info = (wl_solve_info * nrhs)()
    rc = load().wilson_solve_dd(dd, _ptrs(xs), _ptrs(bs), int(nrhs), ctypes.byref(params), info,
                                _stream(stream))
    if check:
        _check(rc)
    return rc, _infos(info, nrhs)


def wl_last_error() -> str:
    return load().wl_last_error().decode()


def wl_spinor16_format() -> int:
    """0: binary16 spinor words (default build); 1: int16 fixed point."""
    return int(load().wl_spinor16_format())


def wl_launch_count() -> int:
    return int(load().wl_launch_count())


def wl_algorithmic_bytes() -> float:
    return float(load().wl_algorithmic_bytes())


def wl_timing(g, enable: bool) -> None:
    _check(load().wl_timing(g, int(bool(enable))))


def wl_timing_read(g, prec: int = -1):
    ms, n, by = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
    _check(load().wl_timing_read(g, int(prec), ctypes.byref(ms), ctypes.byref(n),
                                 ctypes.byref(by)))
    return ms.value, n.value, by.value


# ---------------------------------------------------------------------------
# small conveniences over the raw calls (allocation of internal fields)
# ---------------------------------------------------------------------------

class Gauge:
    """Owns a wl_gauge handle; `fields(prec, nrhs)` allocates internal fields."""

    def __init__(self, dims, kappa, U: torch.Tensor, precs=("f64", "f32", "f16"),
                 bc=(1, 1, 1, -1), stream=None, r12: bool = False, r8: bool = False):
        self.dims = tuple(int(d) for d in dims)
        self.kappa = float(kappa)
        self.bc = tuple(bc)
        self.lat = lattice(dims, kappa, bc)
        mask = prec_mask(*precs) | (WL_LINKS_R12 if r12 else 0) | (WL_LINKS_R8 if r8 else 0)
        self.handle = wl_gauge_create(self.lat, U, mask, stream)
        self.Vh = wl_half_volume(self.handle)

    def field(self, prec, nrhs: int = 1, nhalf: int = 1) -> torch.Tensor:
        p = PREC[prec] if isinstance(prec, str) else prec
        n = wl_field_bytes(self.handle, p, nrhs) * nhalf
        return torch.empty(n, dtype=torch.uint8, device="cuda")

    def close(self):
        if self.handle is not None:
            wl_gauge_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Decomposition:
    """Owns a wl_dd handle: the lattice `dims` cut into `grid` blocks."""

    def __init__(self, dims, kappa, U: torch.Tensor, grid, precs=("f64", "f32", "f16"),
                 bc=(1, 1, 1, -1), stream=None, r12: bool = False, held=None, transport=None):
        """held = (first, count): the blocks this process holds (default: all),
        with `transport` (dd_transport.TorchTransport) for the others."""
        self.dims = tuple(int(d) for d in dims)
        self.grid = tuple(int(k) for k in grid)
        self.kappa = float(kappa)
        self.lat = lattice(dims, kappa, bc)
        mask = prec_mask(*precs) | (WL_LINKS_R12 if r12 else 0)
        self.transport = transport
        if held is None and transport is None:
            self.handle = wl_dd_create(self.lat, self.grid, U, mask, stream)
        else:
            nblk = self.grid[1] * self.grid[2] * self.grid[3]
            first, count = held if held is not None else (0, nblk)
            self.handle = wl_dd_create_part(self.lat, self.grid, first, count, U, mask,
                                            transport.as_c() if transport is not None else None, stream)
        self.n = wl_dd_blocks(self.handle)
        self.blocks = [wl_dd_block(self.handle, k) for k in range(self.n)]
        self.local_dims = tuple(self.dims[m] // self.grid[m] for m in range(4))
        self.Vh = wl_half_volume(self.blocks[0][0])

    def field(self, prec, nrhs: int = 1, nhalf: int = 1):
        """One internal field per block."""
        p = PREC[prec] if isinstance(prec, str) else prec
        n = wl_field_bytes(self.blocks[0][0], p, nrhs) * nhalf
        return [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(self.n)]

    def canonical(self, nrhs: int = 1):
        """One block-local canonical FP64 field per block."""
        V = 2 * self.Vh
        return [torch.zeros((nrhs, V, 4, 3), dtype=torch.complex128, device="cuda")
                for _ in range(self.n)]

    def close(self):
        if self.handle is not None:
            wl_dd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
