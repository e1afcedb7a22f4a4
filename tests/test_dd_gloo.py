"""The multi-process path of the domain decomposition on CPU: two gloo ranks,
each holding one block of a 4x4x4x8 lattice cut along t.

Each rank takes its face messages from the library's planner (wl_dd_plan,
host code), packs its faces in the documented FP64 face layout (the oracle's
projection of its block field), and moves them with the product's
TorchTransport (point-to-point over gloo).  Checked against the undivided
lattice:
  * every received face equals the neighbour's face of the undivided field;
  * Eq. 1 on each block with those faces equals the undivided hopping term;
  * the transport's allreduce of the per-block dot products equals the
    undivided dot product;
  * a BiCGStab on M_ee run by the two ranks (two exchanges per M_ee, one
    allreduce per global sum) reaches the undivided oracle solution.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

DIMS, GRID, BC, KAPPA = (4, 4, 4, 8), (1, 1, 1, 2), (1, 1, 1, -1), 0.124


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _seg(tag):
    seg = tag % 12
    return seg // 6, (seg % 6) // 2 + 1, seg % 2  # launch parity, mu, side


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from oracle import blocks
    from paper_1811_00893_gb300 import dd_transport, fields, wilson
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        U = fields.gauge_field(DIMS, "haar", 3).numpy()
        psi = fields.gaussian_fermion(DIMS, 1, 7)[0].numpy()
        L, _, _ = blocks.layout(DIMS, GRID, rank)
        tr = dd_transport.TorchTransport(rank_of=lambda b: b, rank=rank)
        res = {}

        def exchange(field_half, in_parity):
            """Pack this block's faces, exchange them, return the halos."""
            msgs = dd_transport.plan(DIMS, GRID, rank, wilson.WL_F64, 1, 1)
            size = max(m["offset"] + m["bytes"] for m in msgs)
            send = torch.zeros(size, dtype=torch.uint8)
            recv = torch.zeros(size, dtype=torch.uint8)
            for m in msgs:
                _, mu, side = _seg(m["tag"])
                buf = (send if m["send"] else recv)[m["offset"]:m["offset"] + m["bytes"]]
                if m["send"]:
                    h = blocks.face_halves(field_half, L, in_parity, mu, side)
                    planes = np.ascontiguousarray(h.transpose(1, 2, 0).reshape(6, -1))  # plane 3 s + c
                    assert planes.nbytes == m["bytes"]
                    buf.copy_(torch.from_numpy(planes.view(np.uint8).reshape(-1)))
                m["buf"] = buf
            tr.exchange(msgs)
            halos = {}
            for m in msgs:
                if not m["send"]:
                    _, mu, side = _seg(m["tag"])
                    planes = m["buf"].numpy().view(np.complex128).reshape(6, -1)
                    halos[(mu, side)] = planes.reshape(2, 3, -1).transpose(2, 0, 1).copy()
            return halos

        def hop(field_half, out_parity):
            halos = exchange(field_half, 1 - out_parity)
            return blocks.hop_block(U, DIMS, BC, GRID, rank, field_half, out_parity, halos), halos

        # faces and the hopping term against the undivided lattice
        e, o = oracle.split(psi, DIMS)
        mine_o = blocks.block_half(o, DIMS, GRID, rank, 1)
        out, halos = hop(mine_o, 0)
        other = blocks.block_half(o, DIMS, GRID, 1 - rank, 1)
        res["face_err"] = max(float(np.abs(halos[(3, s)] - blocks.face_halves(other, L, 1, 3, s)).max())
                              for s in (0, 1))
        want = blocks.block_half(oracle.hop_eo(U, o, DIMS, BC, 0), DIMS, GRID, rank, 0)
        res["hop_err"] = float(np.abs(out - want).max() / np.abs(want).max())

        # global sums through the transport's allreduce
        def gdot(a, b):
            t = torch.tensor([np.vdot(a, b).real, np.vdot(a, b).imag], dtype=torch.float64)
            tr.allreduce(t)
            return complex(t[0].item(), t[1].item())

        mine_e = blocks.block_half(e, DIMS, GRID, rank, 0)
        res["dot_err"] = abs(gdot(mine_e, mine_o) - oracle.cdot(e, o)) / abs(oracle.cdot(e, o))

        # BiCGStab on M_ee = 1 - kappa^2 H_eo H_oe, blocks on two ranks
        def Mee(x):
            t, _ = hop(x, 1)
            y, _ = hop(t, 0)
            return x - KAPPA ** 2 * y

        bsys_full = e + KAPPA * oracle.hop_eo(U, o, DIMS, BC, 0)
        b = blocks.block_half(bsys_full, DIMS, GRID, rank, 0)
        x = np.zeros_like(b)
        r = b.copy()
        rh = r.copy()
        p = np.zeros_like(b)
        v = np.zeros_like(b)
        rho_old = alpha = omega = 1.0
        bnorm = np.sqrt(gdot(b, b).real)
        it = 0
        while it < 200:
            rho = gdot(rh, r)
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = Mee(p)
            alpha = rho / gdot(rh, v)
            s = r - alpha * v
            t = Mee(s)
            omega = gdot(t, s) / gdot(t, t).real
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho_old = rho
            it += 1
            if np.sqrt(gdot(r, r).real) <= 1e-11 * bnorm:
                break
        xo_ref, info = oracle.solve(U, psi, DIMS, BC, KAPPA, eo=True, tol=1e-11)
        xe_ref = blocks.block_half(oracle.split(xo_ref, DIMS)[0], DIMS, GRID, rank, 0)
        res["solve_err"] = float(np.linalg.norm(x - xe_ref) / np.linalg.norm(xe_ref))
        res["iters"] = it
        res["oracle_iters"] = info["iters"]
        res["exchanges"] = tr.calls["exchange"]
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_ranks_exchange_faces_and_sums():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, res in out.items():
        assert res["face_err"] == 0.0, res            # the neighbour's face, bit for bit
        assert res["hop_err"] <= 1e-14, res
        assert res["dot_err"] <= 1e-14, res
        assert res["solve_err"] <= 1e-8, res          # cond(M_ee) * 1e-11, with margin
        assert abs(res["iters"] - res["oracle_iters"]) <= 2, res
        assert res["exchanges"] >= 4 * res["iters"]
    assert out[0]["iters"] == out[1]["iters"]          # both ranks take the same decisions
