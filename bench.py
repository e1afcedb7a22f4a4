#!/usr/bin/env python
"""Benchmark of the Wilson-matrix solve on one GB300 (or N independent replicas).

Default workload: a 32^3x64 lattice, even-odd preconditioned Wilson matrix,
kappa = 0.124, smooth SU(3) links exp(i 0.3 A), one Gaussian source, solved to
a true FP64 residual ||b - D x||/||b|| <= 1e-10 by FP32 BiCGStab with FP64
defect correction.  One step = one complete solve through the C ABI
(conversion of b, even-odd source, inner FP32 iterations with fused
reductions, FP64 residual recomputations, reconstruction, final true
residual, conversion of x).

Reported:
  value      whole-solve algorithmic HBM traffic / step time (GB/s), inputs
             resident in device memory before the timed region;
  e2e        the same with host (pinned) b and x: H2D and D2H inside each step;
  roofline   the FP32 hopping kernel: its algorithmic bytes over its CUDA-event
             time in the solve (a second pass of the same K solves with an
             event pair around every hopping launch; the timed region runs
             without them), against the measured HBM copy peak;
  dslash     the paper's protocol (Sec. 5.4): 1000 back-to-back FP32 hopping
             applications timed with CUDA events (GB/s, GFlop/s at 1320/site);
  solve      mixed-precision vs plain FP64 BiCGStab time to 1e-10;
  cpu_baseline  the FP64 CPU oracle on a bounded sample (BiCGStab iterations).

`--impl reference` times the oracle itself on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dslash GB/s & GFlop/s (% HBM peak); mixed vs FP64 solve time to 1e-10 residual"
UNIT = "GB/s"
FALLBACK_HBM_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25  # GB300 non-tensor FP64, nominal
WORKLOAD_INDEX = 1  # 32^3x64 even-odd, FP32 inner, FP64 defect correction
PROFILE = os.path.join(ROOT, "profiles", "hop_f32_32x32x32x64.md")
KERNEL_SOURCES = ["paper_1811_00893_gb300/csrc/dslash.cu", "paper_1811_00893_gb300/csrc/hop_kernels.cuh",
                  "paper_1811_00893_gb300/csrc/hop.cuh", "paper_1811_00893_gb300/csrc/clover.cuh",
                  "paper_1811_00893_gb300/csrc/common.cuh", "paper_1811_00893_gb300/csrc/df64.cuh"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle sample (for quick runs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target duration of the oracle sample")
    ap.add_argument("--workload", type=int, default=WORKLOAD_INDEX,
                    help="workload index (workloads.WORKLOADS); the default is the headline one")
    ap.add_argument("--no-r12", action="store_true",
                    help="skip the compressed-link measurement")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads' sub-records (default: measured after the headline)")
    ap.add_argument("--dims", type=str, default=None,
                    help="override the lattice extents, e.g. 24,24,24,48 (smaller profiling runs)")
    ap.add_argument("--dd", action="store_true",
                    help="measure only the decomposed operator and solve (2 and 4 blocks) on the "
                         "workload's lattice, --steps launches per timing (profiling runs)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# process group
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def aggregate(local_bytes: float, local_ms: float, world: int, device="cpu"):
    """Whole-job totals: bytes summed over ranks, time = max over ranks."""
    if world <= 1:
        return local_bytes, local_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_bytes], dtype=torch.float64, device=device)
    m = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(t.item()), float(m.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_index],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to start: wait (bounded) for its first
            # sample, so that the timed region that follows is sampled from its
            # start; samples up to here are not the timed region's
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.first = len(self.lines)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        # the timed region's samples; a region shorter than the sampling period
        # keeps the sample taken just before it
        lines = self.lines[self.first:] or self.lines[-1:]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ---------------------------------------------------------------------------
# peaks and the committed ncu summary
# ---------------------------------------------------------------------------

def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the FP32 hopping kernel from the committed ncu
    summary, or None when the kernel sources changed since it was taken."""
    try:
        with open(PROFILE) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln and ln.lstrip().startswith("- "):
            k, v = ln.lstrip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def make_inputs(wl, rank: int, device: str):
    from paper_1811_00893_gb300 import fields
    U = fields.gauge_field(wl.dims, wl.links, wl.gauge_seed, device=device)
    b = fields.gaussian_fermion(wl.dims, wl.nrhs, wl.source_seed + 100 * rank, device=device)
    return U, b


SCHEMES = {  # workload scheme -> (inner precision name, solve parameters)
    "fp64": ("f64", dict(eo=False, inner=0)),
    "fp32-defect-correction": ("f32", dict(eo=True, inner=1)),
    "fp16-reliable": ("f16", dict(eo=True, inner=2, delta=0.003)),
    "fp32-multirhs": ("f32", dict(eo=True, inner=1, graph_iters=4)),
}


def config_of(wl):
    from paper_1811_00893_gb300 import costs
    prec, kw = SCHEMES[wl.scheme]
    links = costs.link_bytes(prec) * 8 * wl.volume  # both parities
    extra = {}
    if wl.clover:
        extra["clover"] = ("synthetic F(x): two random Hermitian 6x6 blocks per site, scale 0.1, "
                           f"seed {wl.clover_seed}")
    return {**{"workload": wl.name + f", kappa={wl.kappa}, {wl.links} links, {wl.nrhs} Gaussian "
                                     f"RHS, to 1e-10 true residual"}, **extra,
            "dims": list(wl.dims), "kappa": wl.kappa, "bc": "periodic xyz, antiperiodic t",
            "nrhs": wl.nrhs, "tol": 1e-10, "inner": prec, "outer": "f64", "scheme": wl.scheme,
            "seeds": {"gauge": wl.gauge_seed, "source": wl.source_seed},
            "l2": (f"inputs larger than L2 ({prec.upper()} links {links / 1e6:.0f} MB)"
                   if links > 129e6 else
                   f"inputs smaller than L2 ({links / 1e6:.1f} MB of links): cache-resident")}


def _bsys(wl, U_host, b_host, F_host=None):
    """The oracle's system right-hand side: b'_e (even-odd) or b (full D)."""
    import oracle
    if not wl.eo:
        return b_host
    be, bo = oracle.split(b_host, wl.dims)
    if F_host is not None:  # b' = b_e + kappa H_eo A_oo^-1 b_o
        bo = oracle.clover_diag(F_host, bo, wl.dims, 1, inverse=True)
    return be + wl.kappa * oracle.hop_eo(U_host, bo, wl.dims, wl.bc, 0)


def oracle_iterations(wl, U_host, bsys, F_host=None):
    """A callable running n oracle BiCGStab iterations from x = 0 (one
    start-up: the initial residual, then n iterations), and the start-up's
    own time (n = 0, median of two)."""
    import oracle

    def run(n):
        t0 = time.perf_counter()
        if F_host is not None:
            oracle.clover_bicgstab_fixed(U_host, F_host, bsys, wl.dims, wl.bc, wl.kappa, wl.eo, n)
        else:
            oracle.bicgstab_fixed(U_host, bsys, wl.dims, wl.bc, wl.kappa, wl.eo, n)
        return time.perf_counter() - t0

    start = statistics.median([run(0), run(0)])
    return run, start


def oracle_sample(wl, U_host, b_host, seconds: float, F_host=None, iters_to_tol=None):
    """Time the FP64 oracle's BiCGStab (even-odd or full, Wilson or clover) on
    this lattice for about `seconds`: n iterations after one start-up, the
    start-up's time taken out.  Returns a dict (GB/s on the oracle's own
    FP64 byte model, ms per iteration, cores, description)."""
    import oracle
    from paper_1811_00893_gb300 import costs
    oracle.build()
    clover = F_host is not None
    run, start = oracle_iterations(wl, U_host, _bsys(wl, U_host, b_host, F_host), F_host)
    t1 = max(run(1) - start, 1e-4)
    n = int(max(2, min(60, seconds / t1)))
    dt = max(run(n) - start, 1e-9)
    sites = wl.volume // 2 if wl.eo else wl.volume
    per_iter = costs.bicgstab_iteration_bytes("f64", "f64", eo=wl.eo, clover=clover) * sites
    kind = ("even-odd" if wl.eo else "full-D") + (" clover" if clover else "")
    out = {"value": n * per_iter / dt / 1e9, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
           "sample": (f"{n} FP64 {kind} BiCGStab iterations of the oracle (one right-hand side) on the "
                      f"full {'x'.join(map(str, wl.dims))} lattice after one start-up ({dt:.1f} s, the "
                      f"start-up's {start:.2f} s taken out), bytes counted with the library's FP64 "
                      f"per-iteration model"),
           "ms_per_iteration": dt / n * 1e3, "startup_s": start}
    if iters_to_tol:
        out["seconds_to_1e-10_extrapolated"] = start + iters_to_tol * dt / n
        out["iterations_assumed"] = iters_to_tol
    return out


def oracle_d_gflops(wl, U_host, b_host):
    """The oracle's full D (Eq. 1, 1368 flop per site) on all host cores and
    on one core: one application each."""
    import oracle
    from paper_1811_00893_gb300 import costs
    cores = oracle.get_threads()
    res = {}
    for label, nt in (("all_cores", cores), ("one_core", 1)):
        oracle.set_threads(nt)
        t0 = time.perf_counter()
        oracle.D_full(U_host, b_host, wl.dims, wl.bc, wl.kappa)
        dt = time.perf_counter() - t0
        res[label] = {"gflops": costs.FLOPS_D_SITE * wl.volume / dt / 1e9, "seconds": dt, "cores": nt}
    oracle.set_threads(cores)
    res["flop_per_site"] = costs.FLOPS_D_SITE
    return res


def oracle_solve(wl, U_host, b_host, nrhs_total=1):
    """A full oracle solve to 1e-10 (one right-hand side); nrhs_total > 1
    extrapolates the time to that many right-hand sides."""
    import oracle
    t0 = time.perf_counter()
    x, info = oracle.solve(U_host, b_host, wl.dims, wl.bc, wl.kappa, eo=wl.eo, tol=1e-10)
    dt = time.perf_counter() - t0
    out = {"seconds": dt, "iters": info["iters"], "true_resid": info["true_resid"],
           "cores": oracle.get_threads(), "rhs_solved": 1}
    if nrhs_total > 1:
        out["seconds_all_rhs_extrapolated"] = dt * nrhs_total
        out["rhs_total"] = nrhs_total
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def time_dslash(fn, launches: int, repeats: int, stream):
    """The paper's mult protocol (Sec. 5.4): back-to-back applications timed
    with CUDA events; the median over repeats of the per-launch time (s)."""
    import torch
    for _ in range(10):
        fn()
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(repeats):
        d0.record(stream)
        for _ in range(launches):
            fn()
        d1.record(stream)
        torch.cuda.synchronize()
        ts.append(d0.elapsed_time(d1) / 1e3 / launches)
    return statistics.median(ts), ts


def measure_single(wl, rank, world, local, steps, warmup, *, e2e=True, r12=True, cpu=False,
                   cpu_seconds=15.0, dslash_launches=1000, dslash_repeats=5, oracle_items=False):
    """One single-lattice workload: K timed solves (inputs resident), the
    end-to-end solve with host buffers, the Dslash protocol, the compressed
    links, the plain FP64 GPU solve and (rank 0) the oracle baselines."""
    import torch
    from paper_1811_00893_gb300 import costs, fields, wilson

    dev = f"cuda:{local}"
    pname, pkw = SCHEMES[wl.scheme]
    P = wilson.PREC[pname]
    U, b = make_inputs(wl, rank, dev)
    want_cpu = cpu and rank == 0 and world == 1
    U_host = U.cpu().numpy() if (want_cpu or oracle_items) else None
    b_host = b[0].cpu().numpy() if (want_cpu or oracle_items) else None
    g = wilson.Gauge(wl.dims, wl.kappa, U, precs=("f64", pname), bc=wl.bc)
    # the same operator with compressed (two-row) links, measured beside it
    g12 = (wilson.Gauge(wl.dims, wl.kappa, U, precs=("f64", pname), bc=wl.bc, r12=True)
           if pname in ("f32", "f16") and r12 else None)
    # eight-real links: FP32 single-RHS Wilson launches
    g8 = (wilson.Gauge(wl.dims, wl.kappa, U, precs=("f64", pname), bc=wl.bc, r8=True)
          if pname == "f32" and r12 and wl.nrhs == 1 and not wl.clover else None)
    del U
    F_host = None
    if wl.clover:  # D_clov of Eq. 2: attach the seeded synthetic clover field
        F = fields.clover_field(wl.dims, wl.clover_seed, device=dev)
        wilson.wl_clover_set(g.handle, F)
        if g12 is not None:
            wilson.wl_clover_set(g12.handle, F)
        F_host = F.cpu().numpy() if (want_cpu or oracle_items) else None
        del F
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    x = torch.zeros_like(b)
    mixed = wilson.solve_params(tol=1e-10, **pkw)

    def solve(xx, bb, p=mixed):
        return wilson.wilson_solve(g.handle, xx, bb, wl.nrhs, p)

    for _ in range(max(3, warmup)):
        rc, info = solve(x, b)
    # ---------------- timed region: K solves, inputs resident in HBM
    clk = ClockSampler(gpu_index_for(local)).start()
    l0, b0 = wilson.wl_launch_count(), wilson.wl_algorithmic_bytes()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(steps):
        rc, info = solve(x, b)
        infos.extend(info)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    ms_local = e0.elapsed_time(e1)
    launches = wilson.wl_launch_count() - l0
    bytes_local = wilson.wl_algorithmic_bytes() - b0
    # ---------------- the same K solves again with a CUDA-event pair around
    # every hopping launch (the kernels' own durations; the records between
    # launches cost ~2 % of a step, so the timed region above runs without)
    wilson.wl_timing(g.handle, True)
    torch.cuda.synchronize()
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record(stream)
    for _ in range(steps):
        solve(x, b)
    i1.record(stream)
    torch.cuda.synchronize()
    ms_instr = i0.elapsed_time(i1)
    wilson.wl_timing(g.handle, False)
    hop_ms, hop_n, hop_bytes = wilson.wl_timing_read(g.handle, P)
    h64_ms, h64_n, h64_bytes = wilson.wl_timing_read(g.handle, wilson.WL_F64)
    if P == wilson.WL_F64:
        h64_ms = 0.0
    total_bytes, ms = aggregate(bytes_local, ms_local, world, device=dev)
    ms_per_step = ms / steps
    value = total_bytes / (ms / 1e3) / 1e9

    # ---------------- e2e: host buffers through the same C call
    nbytes_io = b.numel() * b.element_size()
    e2e_rec = None
    if e2e:
        b_h = b.cpu().pin_memory()
        x_h = torch.zeros_like(b_h).pin_memory()
        # warm-up calls like the device timing's: the first host transfer after
        # a long stretch of device work can run several times slower
        for _ in range(max(3, warmup)):
            solve(x_h, b_h)
        e2e_steps = max(5, steps // 2)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solve(x_h, b_h)
        e2e_s = time.perf_counter() - t0
        _, e2e_ms = aggregate(0.0, e2e_s * 1e3 / e2e_steps, world, device=dev)
        step_bytes = total_bytes / steps
        e2e_rec = {"value": step_bytes / (e2e_ms / 1e3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": nbytes_io,
                   "d2h_bytes_per_step": nbytes_io, "ms_per_step": e2e_ms,
                   "timer": "wall clock around wilson_solve with pinned host b and x"}

    # ---------------- the paper's mult protocol: 1000 back-to-back hops, 5 times
    nr = wl.nrhs
    fin = g.field(pname, nr)
    fout = g.field(pname, nr)
    wilson.wl_field_to_internal(g.handle, fin, b, 1, P, nr)
    dslash_s, reps = time_dslash(lambda: wilson.wilson_dslash(g.handle, fout, fin, 0, 0, P, nr),
                                 dslash_launches, dslash_repeats, stream)
    Vh = wl.volume // 2
    peak, peak_kind = hbm_peak()
    bps = costs.hop_bytes_per_site(pname, nrhs=nr)
    dslash_gbs = bps * Vh / dslash_s / 1e9
    dslash = {"precision": pname, "nrhs": nr, "gbs": dslash_gbs,
              "gflops": costs.FLOPS_HOP_SITE * Vh * nr / dslash_s / 1e9,
              "us_per_launch": dslash_s * 1e6, "frac_hbm": dslash_gbs / peak,
              "bytes_per_site": bps, "launches": dslash_launches, "repeats": dslash_repeats,
              "statistic": "median over repeats",
              "us_per_launch_repeats": [round(t * 1e6, 2) for t in reps]}
    if not wl.eo:  # the full D apply of this workload (1368 flop per site)
        fin2 = g.field(pname, nr, nhalf=2)
        fout2 = g.field(pname, nr, nhalf=2)
        fb = wilson.wl_field_bytes(g.handle, P, 1)
        wilson.wl_field_to_internal(g.handle, fin2[:fb], b, 0, P, nr)
        wilson.wl_field_to_internal(g.handle, fin2[fb:], b, 1, P, nr)
        d_s, _ = time_dslash(lambda: wilson.wilson_mult(g.handle, fout2, fin2, 0, 0, P, nr),
                             dslash_launches, dslash_repeats, stream)
        dslash["full_D"] = {"us_per_apply": d_s * 1e6,
                            "gflops": costs.FLOPS_D_SITE * wl.volume * nr / d_s / 1e9,
                            "flop_per_site": costs.FLOPS_D_SITE}
    if wl.clover:  # the fused clover Schur apply: A_oo^-1 H_oe, then A_ee in - k^2 H_eo tmp
        mult_s, _ = time_dslash(lambda: wilson.wilson_mult(g.handle, fout, fin, 1, 0, P, nr), 200, 3, stream)
        mbps = (costs.hop_bytes_per_site(pname, nrhs=nr, clover=True) +
                costs.hop_bytes_per_site(pname, nrhs=nr, extra_in=1, clover=True))
        dslash["clover_mee"] = {"gbs": mbps * Vh / mult_s / 1e9, "us_per_apply": mult_s * 1e6,
                                "bytes_per_site": mbps, "frac_hbm": mbps * Vh / mult_s / 1e9 / peak,
                                "launches_per_apply": 2}

    # ---------------- compressed links: the same Dslash protocol and solve
    def compressed(gc, cb):
        t_s, _ = time_dslash(lambda: wilson.wilson_dslash(gc.handle, fout, fin, 0, 0, P, nr),
                             dslash_launches, 1, stream)
        xc = torch.zeros_like(b)
        rcc, infc = wilson.wilson_solve(gc.handle, xc, b, wl.nrhs, mixed)  # warm
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(3):
            rcc, infc = wilson.wilson_solve(gc.handle, xc, b, wl.nrhs, mixed)
        f1.record(stream)
        torch.cuda.synchronize()
        return {"dslash_us_per_launch": t_s * 1e6,
                "dslash_gbs_compressed_bytes": cb * Vh / t_s / 1e9,
                "dslash_gbs_equivalent": bps * Vh / t_s / 1e9,
                "dslash_gflops": costs.FLOPS_HOP_SITE * Vh * nr / t_s / 1e9,
                "bytes_per_site_compressed": cb,
                "solve_ms": f0.elapsed_time(f1) / 3, "solve_iters": max(i["iters"] for i in infc),
                "solve_true_resid": max(i["true_resid"] for i in infc)}

    r12_rec = r8_rec = None
    if g12 is not None:
        r12_rec = compressed(g12, costs.hop_bytes_per_site(pname, nrhs=nr, r12=True))
        g12.close()
    if g8 is not None:
        r8_rec = compressed(g8, 8 * 32 + 2 * costs.spinor_bytes(pname))
        g8.close()

    # ---------------- plain FP64 GPU solve for the time-to-solution comparison
    p64 = wilson.solve_params(tol=1e-10, eo=wl.eo, inner=wilson.WL_F64, graph_iters=0)
    if P == wilson.WL_F64:
        fp64_ms, info64 = ms_per_step, infos[-nr:]
    else:
        x64 = torch.zeros_like(b)
        solve(x64, b, p64)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        rc64, info64 = solve(x64, b, p64)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = f0.elapsed_time(f1)

    achieved = hop_bytes / (hop_ms / 1e3) / 1e9 if hop_ms > 0 else None
    kname = f"hop_kernel<{pname}>" if nr == 1 else f"hop_mrhs_kernel<{pname}>"
    if P == wilson.WL_F64:
        # FP64 arithmetic bounds the FP64 stencil on GB300; no measured FP64
        # peak exists, so the nominal rate is the denominator
        tf = dslash["gflops"] / 1e3
        roofline = {"kernel": kname + " (1000-launch protocol)", "bound": "alu", "achieved": tf,
                    "peak": FP64_NOMINAL_TFLOPS, "peak_kind": "nominal FP64 rate of GB300",
                    "unit": "TFLOP/s", "frac": tf / FP64_NOMINAL_TFLOPS, "traffic": None,
                    "launches": dslash_launches, "avg_us": dslash["us_per_launch"]}
    elif hop_n == 0:
        # the solve's hopping launches run inside CUDA graphs, which the
        # per-launch timer does not see: report the kernel timed alone
        roofline = {"kernel": kname + " (1000-launch protocol; the solve replays it in CUDA graphs)",
                    "bound": "hbm", "achieved": dslash_gbs, "peak": peak, "peak_kind": peak_kind,
                    "unit": "GB/s", "frac": dslash_gbs / peak, "traffic": None, "launches": dslash_launches,
                    "algorithmic_bytes_per_launch": bps * Vh, "avg_us": dslash["us_per_launch"]}
    else:
        traffic = profiled_traffic()
        roofline = {"kernel": kname + " (all hopping launches of the inner solve; per-launch CUDA events "
                              "in a second pass of the same K solves)",
                    "bound": "hbm", "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": (achieved / peak) if achieved else None,
                    "traffic": traffic if (P == wilson.WL_F32 and nr == 1 and not wl.clover
                                           and wl.dims == (32, 32, 32, 64)) else None,
                    "launches": hop_n,
                    "algorithmic_bytes_per_launch": hop_bytes / max(hop_n, 1),
                    "avg_us": hop_ms * 1e3 / max(hop_n, 1),
                    "share_of_step": hop_ms / ms_instr if ms_instr else None,
                    "f64_hop_share_of_step": h64_ms / ms_instr if ms_instr else None,
                    "instrumented_ms_per_step": ms_instr / steps}
    mixed_iters = max(i["iters"] for i in infos[-nr:])
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": max(3, warmup), "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": pname, "dtype_outer": "f64", "data": "synthetic",
        "config": config_of(wl),
        "clocks": clocks,
        "e2e": e2e_rec,
        "gpu_launches": launches,
        # library launch-counter values around the timed region: launches
        # [l0, l1) of this process's library kernels are the timed ones
        "launch_index_range": [l0, l0 + launches],
        "roofline": roofline,
        "dslash": dslash,
        "r12": r12_rec,
        "r8": r8_rec,
        "solve": {"mixed_ms": ms_per_step, "fp64_ms": fp64_ms,
                  "speedup_vs_fp64": fp64_ms / ms_per_step,
                  "mixed_iters": mixed_iters,
                  "mixed_ms_per_iteration": ms_per_step / max(mixed_iters, 1),
                  "mixed_outer": max(i["outer"] for i in infos[-nr:]),
                  "mixed_true_resid": max(i["true_resid"] for i in infos),
                  "fp64_iters": max(i["iters"] for i in info64),
                  "fp64_ms_per_iteration": fp64_ms / max(max(i["iters"] for i in info64), 1),
                  "fp64_true_resid": max(i["true_resid"] for i in info64)},
    }
    if want_cpu:
        out["cpu_baseline"] = oracle_sample(wl, U_host, b_host, cpu_seconds, F_host,
                                            iters_to_tol=out["solve"]["fp64_iters"])
        out["cpu_baseline"]["oracle_D"] = oracle_d_gflops(wl, U_host, b_host)
    else:
        out["cpu_baseline"] = None
    if oracle_items and rank == 0 and F_host is None:
        out["oracle_solve"] = oracle_solve(wl, U_host, b_host, nrhs_total=wl.nrhs)
    g.close()
    torch.cuda.empty_cache()
    return out


def measure_dd(wl, local, grids=((1, 1, 1, 2), (1, 1, 2, 2)), launches=200, repeats=5):
    """The decomposed operator on one GPU (Sec. 4.4's pack / exchange ||
    interior / boundary): per block grid, the decomposed FP32 Dslash in both
    exchange modes and the decomposed mixed solve, beside the undivided ones."""
    import torch
    from paper_1811_00893_gb300 import costs, wilson
    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream()
    U, b = make_inputs(wl, 0, dev)
    Vh = wl.volume // 2
    peak, peak_kind = hbm_peak()
    bps = costs.hop_bytes_per_site("f32")
    mixed = wilson.solve_params(tol=1e-10, eo=True, inner=wilson.WL_F32)
    clk = ClockSampler(gpu_index_for(local)).start()
    out = {"workload": f"{'x'.join(map(str, wl.dims))} even-odd, FP32 Dslash and FP32 defect-correction "
                       f"solve, kappa={wl.kappa}, {wl.links} links",
           "bytes_per_site": bps, "peak": peak, "peak_kind": peak_kind, "grids": []}
    with wilson.Gauge(wl.dims, wl.kappa, U, precs=("f64", "f32"), bc=wl.bc) as g:
        fin, fout = g.field("f32"), g.field("f32")
        wilson.wl_field_to_internal(g.handle, fin, b, 1, wilson.WL_F32, 1)
        t, _ = time_dslash(lambda: wilson.wilson_dslash(g.handle, fout, fin, 0, 0, wilson.WL_F32, 1),
                           launches, repeats, stream)
        x = torch.zeros_like(b)
        wilson.wilson_solve(g.handle, x, b, 1, mixed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = wilson.wilson_solve(g.handle, x, b, 1, mixed)
        out["undivided"] = {"dslash_us": t * 1e6, "dslash_gbs": bps * Vh / t / 1e9,
                            "solve_ms": (time.perf_counter() - t0) * 1e3, "iters": info[0]["iters"]}
    for grid in grids:
        with wilson.Decomposition(wl.dims, wl.kappa, U, grid, precs=("f64", "f32"), bc=wl.bc) as dd:
            loc = dd.canonical(1)
            wilson.wl_dd_scatter(dd.handle, loc, b, 1)
            fin, fout = dd.field("f32"), dd.field("f32")
            for k, (gk, _) in enumerate(dd.blocks):
                wilson.wl_field_to_internal(gk, fin[k], loc[k], 1, wilson.WL_F32, 1)
            rec = {"grid": list(grid), "blocks": dd.n, "block_dims": list(dd.local_dims)}
            for mode, name in ((0, "copy"), (1, "direct")):
                wilson.wl_dd_set_exchange(dd.handle, mode)
                t, _ = time_dslash(lambda: wilson.wilson_dslash_dd(dd.handle, fout, fin, 0, 0, wilson.WL_F32, 1),
                                   launches, repeats, stream)
                rec[f"dslash_{name}"] = {"us": t * 1e6, "gbs": bps * Vh / t / 1e9, "frac_hbm": bps * Vh / t / 1e9 / peak,
                                         "vs_undivided": out["undivided"]["dslash_us"] / (t * 1e6)}
            wilson.wl_dd_set_exchange(dd.handle, 0)
            xl = dd.canonical(1)
            wilson.wilson_solve_dd(dd.handle, xl, loc, 1, mixed)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = wilson.wilson_solve_dd(dd.handle, xl, loc, 1, mixed)
            solve_ms = (time.perf_counter() - t0) * 1e3
            rec["solve"] = {"ms": solve_ms, "iters": info[0]["iters"], "true_resid": info[0]["true_resid"],
                            "vs_undivided": out["undivided"]["solve_ms"] / solve_ms}
            out["grids"].append(rec)
    out["clocks"] = clk.stop()
    del U, b
    torch.cuda.empty_cache()
    return out


SUB_KEYS = ("config", "value", "unit", "ms_per_step", "steps", "clocks", "roofline", "dslash", "r12", "solve",
            "gpu_launches", "oracle_solve")


def run_ours(args, rank, world, local):
    import dataclasses

    import torch
    from paper_1811_00893_gb300.workloads import by_index

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    wl = by_index(args.workload)
    if args.dims:
        wl = dataclasses.replace(wl, dims=tuple(int(v) for v in args.dims.split(",")))
    out = measure_single(wl, rank, world, local, args.steps, args.warmup, e2e=True, r12=not args.no_r12,
                         cpu=not args.no_cpu_baseline, cpu_seconds=args.cpu_seconds)
    if rank != 0:
        return None
    if world == 1 and not args.no_extra and args.workload == WORKLOAD_INDEX and not args.dims:
        # every other workload (and the decomposition), each with its own clocks
        for idx, key in ((0, "w0_8x8x8x8_fp64_full_D"), (2, "w2_48x48x48x96_fp16_reliable"),
                         (3, "w3_24x24x24x48_12rhs"), (5, "w5_32x32x32x64_clover")):
            sub = measure_single(by_index(idx), 0, 1, local, 5 if idx else 20, 3, e2e=False, r12=False,
                                 oracle_items=idx in (0, 3))
            out[key] = {k: sub[k] for k in SUB_KEYS if k in sub}
        out["w4_uneven_batch16"] = run_batch(args, rank, world, local, steps=5, sub=True)
        out["dd_32x32x32x64_f32"] = measure_dd(wl, local)
    return out


def run_dd(args, rank, world, local):
    """The decomposed operator alone (one process holds every block)."""
    import dataclasses

    import torch
    from paper_1811_00893_gb300.workloads import by_index

    if rank != 0:
        return None
    torch.cuda.set_device(local)
    wl = by_index(args.workload)
    if args.dims:
        wl = dataclasses.replace(wl, dims=tuple(int(v) for v in args.dims.split(",")))
    return {"impl": "ours", "decomposition": measure_dd(wl, local, launches=max(1, args.steps), repeats=1)}


# ---------------------------------------------------------------------------
# the uneven multi-lattice batch
# ---------------------------------------------------------------------------

BATCH_INDEX = 4


def run_batch(args, rank, world, local, steps=None, sub=False):
    import numpy as np
    import torch
    from paper_1811_00893_gb300 import fields, wilson, workloads

    steps = args.steps if steps is None else steps
    torch.cuda.set_device(local)
    if not sub:
        dist_init(world, "nccl")
    dev = f"cuda:{local}"
    spec = workloads.uneven_batch()
    gs, bs, xs = [], [], []
    for m in spec:
        U = fields.gauge_field(m.dims, "haar", m.gauge_seed, device=dev)
        gs.append(wilson.Gauge(m.dims, m.kappa, U, precs=("f64", "f32"), bc=workloads.BC_PPPA))
        bs.append(fields.gaussian_fermion(m.dims, m.nrhs, m.source_seed + 100 * rank, device=dev))
        xs.append(torch.zeros_like(bs[-1]))
    hs = [g.handle for g in gs]
    nr = [m.nrhs for m in spec]
    p = wilson.solve_params(tol=1e-10, eo=True, inner=wilson.WL_F32, graph_iters=4)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        wilson.wilson_solve_batch(hs, xs, bs, nr, p)
    clk = ClockSampler(gpu_index_for(local)).start()
    l0, b0 = wilson.wl_launch_count(), wilson.wl_algorithmic_bytes()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rc, infos = wilson.wilson_solve_batch(hs, xs, bs, nr, p)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    ms_local = e0.elapsed_time(e1)
    launches = wilson.wl_launch_count() - l0
    # algorithmic bytes of the work the systems actually did: per lattice its
    # links four times per iteration while any of its systems iterates, and
    # each system's spinor passes for the iterations it ran (the library's
    # counter charges the captured iteration graphs in full even when the
    # kernels skip converged lattices)
    from paper_1811_00893_gb300 import costs
    per_iter = costs.bicgstab_iteration_bytes("f32", "f32", eo=True)
    link_part = 4 * 8 * costs.link_bytes("f32")
    work = 0.0
    k = 0
    for m in spec:
        Vh = int(np.prod(m.dims)) // 2
        its = [infos[k + r]["iters"] for r in range(m.nrhs)]
        k += m.nrhs
        work += Vh * (max(its) * link_part + sum(its) * (per_iter - link_part))
    total_bytes, ms = aggregate(work * steps, ms_local, world, device=dev)

    # ---------------- e2e: host buffers through the same C call (each
    # lattice's b and x move on its own stream, beside the other lattices' work)
    bs_h = [t.cpu().pin_memory() for t in bs]
    xs_h = [torch.zeros_like(t).pin_memory() for t in bs_h]

    def e2e_step():
        wilson.wilson_solve_batch(hs, xs_h, bs_h, nr, p)
        torch.cuda.synchronize()

    # warm-up calls like the device timing's: the first host transfer after a
    # long stretch of device work can run several times slower
    for _ in range(max(3, args.warmup)):
        e2e_step()
    e2e_steps = max(5, steps)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    _, e2e_ms = aggregate(0.0, (time.perf_counter() - t0) * 1e3 / e2e_steps, world, device=dev)
    nbytes_io = sum(t.numel() * t.element_size() for t in bs)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3

    def per_lattice(inner, graph):
        q = wilson.solve_params(tol=1e-10, eo=True, inner=inner, graph_iters=graph)
        for g, x, b, n in zip(gs, xs, bs, nr):
            wilson.wilson_solve(g.handle, x, b, n, q)

    seq_mixed_ms = timed(lambda: per_lattice(wilson.WL_F32, 4))
    seq_fp64_ms = timed(lambda: per_lattice(wilson.WL_F64, 4))
    oracle_rec = None
    if sub and rank == 0:
        # the oracle's full solves, one right-hand side of every lattice (the
        # time for all right-hand sides extrapolated by their count)
        import oracle
        from paper_1811_00893_gb300.workloads import Workload
        t_all, t_one, its = 0.0, 0.0, []
        for m, g, b in zip(spec, gs, bs):
            w1 = Workload(4, "batch member", m.dims, m.kappa, "haar", 1, True, "fp32-defect-correction")
            Uh = fields.gauge_field(m.dims, "haar", m.gauge_seed, device=dev).cpu().numpy()
            r = oracle_solve(w1, Uh, b[0].cpu().numpy())
            t_one += r["seconds"]
            t_all += r["seconds"] * m.nrhs
            its.append(r["iters"])
        oracle_rec = {"seconds_one_rhs_per_lattice": t_one, "seconds_all_systems_extrapolated": t_all,
                      "iters": its, "cores": oracle.get_threads(),
                      "kind": "full FP64 even-odd solves of the oracle, one right-hand side per lattice"}
    out = None
    if rank == 0:
        step_ms = ms / steps
        out = {
            "metric": METRIC, "value": total_bytes / (ms / 1e3) / 1e9, "unit": UNIT,
            "n_gpus": world, "steps": steps, "warmup": max(3, args.warmup),
            "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "dtype_outer": "f64", "data": "synthetic",
            "config": {"workload": "uneven batch of 16 lattices from {8^4, 12^3x24, 16^3x32, "
                                   "16^4}, 1-8 Gaussian RHS each, kappa in [0.11, 0.124], Haar "
                                   "links; one persistent FP32 hopping kernel per operator, "
                                   "FP64 refinement to 1e-10",
                       "lattices": [list(m.dims) for m in spec], "nrhs": nr,
                       "kappa": [round(m.kappa, 5) for m in spec], "seed": 5005,
                       "l2": "batch links total 0.5 GB FP32: larger than L2"},
            "clocks": clocks,
            "e2e": {"value": total_bytes / steps / (e2e_ms / 1e3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": nbytes_io, "d2h_bytes_per_step": nbytes_io,
                    "ms_per_step": e2e_ms,
                    "timer": "wall clock around wilson_solve_batch with pinned host b and x "
                             "for every lattice"},
            "gpu_launches": launches, "launch_index_range": [l0, l0 + launches],
            # the batch's hopping and vector kernels run inside CUDA graphs,
            # which the per-launch timer does not see: the whole solve's
            # algorithmic bytes over its time
            "roofline": {"kernel": "whole batch solve (persistent batch hopping kernel, batched "
                                   "vector kernels, per-lattice FP64/df64 outer work)",
                         "bound": "hbm", "achieved": total_bytes / (ms / 1e3) / 1e9,
                         "peak": hbm_peak()[0], "peak_kind": hbm_peak()[1], "unit": "GB/s",
                         "frac": total_bytes / (ms / 1e3) / 1e9 / hbm_peak()[0], "traffic": None,
                         "bytes": "cost model over the inner iterations each system ran"},
            "solve": {"batch_ms": step_ms, "per_lattice_mixed_ms": seq_mixed_ms,
                      "per_lattice_fp64_ms": seq_fp64_ms,
                      "speedup_vs_per_lattice_fp64": seq_fp64_ms / step_ms,
                      "speedup_vs_per_lattice_mixed": seq_mixed_ms / step_ms,
                      "max_iters": max(i["iters"] for i in infos),
                      "max_true_resid": max(i["true_resid"] for i in infos),
                      "systems": len(infos)},
            "cpu_baseline": None,
        }
    for g in gs:
        g.close()
    if sub and out is not None:
        out = {k: out[k] for k in ("config", "value", "unit", "ms_per_step", "steps", "clocks", "roofline",
                                  "solve", "gpu_launches")}
        out["oracle_solve"] = oracle_rec
    return out


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world, local):
    """The oracle on the host cores: each step is one BiCGStab iteration of one
    continuing solve (the start-up, the initial residual, is timed apart and
    taken out), on the headline workload's inputs."""
    if rank != 0:
        return None
    import torch

    import oracle
    from paper_1811_00893_gb300 import costs
    from paper_1811_00893_gb300.workloads import by_index

    wl = by_index(WORKLOAD_INDEX)
    if args.dims:  # smaller runs (tests); the default is the workload's own size
        import dataclasses
        wl = dataclasses.replace(wl, dims=tuple(int(v) for v in args.dims.split(",")))
    dev = f"cuda:{local}" if torch.cuda.is_available() else "cpu"
    U, b = make_inputs(wl, 0, dev)  # same seeded inputs as the GPU arm
    U_host, b_host = U.cpu().numpy(), b[0].cpu().numpy()
    del U, b
    oracle.build()
    run, start = oracle_iterations(wl, U_host, _bsys(wl, U_host, b_host))
    run(max(3, args.warmup))  # warm-up iterations (untimed)
    dt = max(run(args.steps) - start, 1e-9)
    Vh = wl.volume // 2
    step_bytes = costs.bicgstab_iteration_bytes("f64", "f64") * Vh
    value = step_bytes * args.steps / dt / 1e9
    sample = (f"{args.steps} FP64 even-odd BiCGStab iterations of one oracle solve on the full "
              f"{'x'.join(map(str, wl.dims))} lattice, one per step, after one start-up (the initial "
              f"residual, {start:.2f} s, timed apart and taken out); bytes on the oracle's FP64 model")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(wl),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample,
                             "ms_per_iteration": dt * 1e3 / args.steps, "startup_s": start}}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world, local)
    elif args.dd:
        out = run_dd(args, rank, world, local)
    elif args.workload == BATCH_INDEX:
        out = run_batch(args, rank, world, local)
    else:
        out = run_ours(args, rank, world, local)
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
