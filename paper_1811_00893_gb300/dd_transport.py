"""Transport of the domain-decomposed operator between processes.

A decomposition (``wl_dd_create_part``) whose blocks are spread over several
processes moves its packed faces and its global sums through a
``wl_dd_transport``: two callbacks the library calls at the exchange step of
every hopping application (Sec. 4.4, "communication") and at every global sum
of the solver.  ``TorchTransport`` implements them with ``torch.distributed``:
point-to-point sends and receives between ranks (NCCL on GPUs; gloo for host
buffers), plain copies between blocks of the same rank, and an all-reduce of
the sums.  It moves bytes only; all arithmetic stays in the library.

Matching of messages: every face message has a tag, equal at both ends
(12 * receiving block + segment).  Operations with one peer are posted in tag
order on both sides, which is the order NCCL matches them in (it ignores
tags); gloo matches by tag.
"""
from __future__ import annotations

import ctypes
import traceback

import torch

from . import wilson


class wl_dd_msg(ctypes.Structure):
    _fields_ = [("send", ctypes.c_int), ("block", ctypes.c_int), ("peer", ctypes.c_int),
                ("tag", ctypes.c_int), ("offset", ctypes.c_size_t), ("bytes", ctypes.c_size_t),
                ("buf", ctypes.c_void_p)]


EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(wl_dd_msg),
                               ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                ctypes.c_int, ctypes.c_void_p)


class wl_dd_transport(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("exchange", EXCHANGE_FN), ("allreduce", ALLREDUCE_FN),
                ("all", ctypes.c_int)]


def plan(dims, grid, block: int, prec: int, nrhs: int = 1, nparity: int = 1):
    """The face messages of one block (``wl_dd_plan``; host code, no GPU)."""
    lib = wilson.load()
    D = (ctypes.c_int * 4)(*[int(v) for v in dims])
    G = (ctypes.c_int * 4)(*[int(v) for v in grid])
    arr = (wl_dd_msg * 32)()
    n = lib.wl_dd_plan(D, G, int(block), int(prec), int(nrhs), int(nparity), arr, 32)
    if n < 0:
        raise wilson.WilsonError(n, lib.wl_last_error().decode())
    return [{"send": m.send, "block": m.block, "peer": m.peer, "tag": m.tag, "offset": m.offset,
             "bytes": m.bytes} for m in arr[:n]]


class _DeviceBytes:
    """A raw device range as an object torch can view (CUDA array interface)."""

    def __init__(self, ptr: int, n: int, typestr: str = "|u1", itemsize: int = 1):
        self.__cuda_array_interface__ = {"shape": (n // itemsize,), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr: int, nbytes: int, dtype=torch.uint8) -> torch.Tensor:
    """A tensor over nbytes of device memory at ptr (no copy)."""
    if dtype == torch.float64:
        return torch.as_tensor(_DeviceBytes(ptr, nbytes, "<f8", 8), device="cuda")
    return torch.as_tensor(_DeviceBytes(ptr, nbytes), device="cuda")


class TorchTransport:
    """Faces and sums through torch.distributed.

    rank_of(block) gives the rank holding a block; blocks of this rank are
    copied locally.  With route_all the library also hands the faces between
    blocks of this process to the transport (instead of its own device
    copies).  `group` is the torch.distributed group (None: the default one,
    or no process group at all when every block is held by this process).
    """

    def __init__(self, rank_of, rank: int = 0, group=None, route_all: bool = False):
        self.rank_of = rank_of
        self.rank = int(rank)
        self.group = group
        self.route_all = bool(route_all)
        self._c = None
        self.calls = {"exchange": 0, "allreduce": 0}

    # ---- the two operations, on tensors ------------------------------------
    def exchange(self, msgs) -> None:
        """msgs: dicts with send, peer, tag and buf (a uint8 tensor)."""
        import torch.distributed as dist
        self.calls["exchange"] += 1
        local = {}
        ops = []
        for m in sorted(msgs, key=lambda q: (q["tag"], q["send"])):
            r = self.rank_of(m["peer"])
            if r == self.rank:
                if m["send"]:
                    local[m["tag"]] = m["buf"]
                continue
            op = dist.isend if m["send"] else dist.irecv
            ops.append(dist.P2POp(op, m["buf"], r, group=self.group, tag=int(m["tag"])))
        for m in msgs:
            if not m["send"] and self.rank_of(m["peer"]) == self.rank:
                m["buf"].copy_(local[m["tag"]])
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def allreduce(self, t: torch.Tensor) -> None:
        import torch.distributed as dist
        self.calls["allreduce"] += 1
        if dist.is_available() and dist.is_initialized() and dist.get_world_size(self.group) > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)

    # ---- the C callbacks ----------------------------------------------------
    def as_c(self) -> wl_dd_transport:
        """The wl_dd_transport handed to wl_dd_create_part (kept alive here)."""
        if self._c is not None:
            return self._c

        def _exchange(ctx, n, msgs, stream):
            try:
                ms = [{"send": m.send, "block": m.block, "peer": m.peer, "tag": m.tag,
                       "buf": device_view(m.buf, m.bytes)} for m in msgs[:n]]
                with torch.cuda.stream(torch.cuda.ExternalStream(int(stream or 0))):
                    self.exchange(ms)
                return 0
            except Exception:  # the library reports the failure as WL_ERR_CUDA
                traceback.print_exc()
                return -1

        def _allreduce(ctx, buf, n, stream):
            try:
                t = device_view(ctypes.cast(buf, ctypes.c_void_p).value, 8 * n, torch.float64)
                with torch.cuda.stream(torch.cuda.ExternalStream(int(stream or 0))):
                    self.allreduce(t)
                return 0
            except Exception:
                traceback.print_exc()
                return -1

        self._fns = (EXCHANGE_FN(_exchange), ALLREDUCE_FN(_allreduce))
        self._c = wl_dd_transport(None, self._fns[0], self._fns[1], 1 if self.route_all else 0)
        return self._c
