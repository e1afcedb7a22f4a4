"""wl_cdot_noalloc, the allocation-free dot/norm entry point, against wl_cdot.

Some callers cannot allocate device memory (they run inside another
framework's memory pool, or in loops where cudaMalloc would synchronise the
device, or hold field pointers without a gauge object); wl_cdot_noalloc serves
them from a fixed built-in scratch array.  This file is collected last so a
run that stops at the first failure has already run every other test; it
also passes alone in a fresh process (its first call sets up the scratch).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import PRECS, Case
from paper_1811_00893_gb300 import wilson

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (24, 24, 24, 48)], ids=["Vh960", "Vh331776"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
def test_noalloc_matches_wl_cdot_on_two_calls(dims, prec):
    c = Case(dims, kappa=0.12, kind="haar", seed=9, precs=("f64", "f32", "f16"))
    try:
        nrhs = 3  # (df64 fields come with FP32 / FP16: the gauge object adds them)
        ia = c.to_internal(c.source(nrhs=nrhs, seed=91), 0, prec)
        ib = c.to_internal(c.source(nrhs=nrhs, seed=92), 0, prec)
        ref = torch.zeros(3 * nrhs, dtype=torch.float64, device="cuda")
        wilson.wl_cdot(c.g.handle, ref, ia, ib, PRECS[prec], nrhs)
        for _ in range(2):  # the second call reuses the scratch the first left behind
            out = torch.full((3 * nrhs,), float("nan"), dtype=torch.float64, device="cuda")
            wilson.wl_cdot_noalloc(out, ia, ib, c.Vh, PRECS[prec], nrhs)
            torch.cuda.synchronize()
            r, o = ref.view(nrhs, 3), out.view(nrhs, 3)
            scale = r[:, 2:3].expand_as(r)  # ||b||^2 ~ ||a|| ||b|| for these fields
            assert torch.all(torch.isfinite(o))
            assert torch.all((o - r).abs() <= 1e-12 * scale)
        # and against the oracle's (a, b) = sum conj(a) b on the stored values:
        # the kernel forms each site's products in the storage type's
        # arithmetic (FP32 for FP32 / FP16, relative rounding 2^-24 per term)
        # and sums in FP64
        ca = c.to_canonical(ia, 0, prec, nrhs=nrhs)
        cb = c.to_canonical(ib, 0, prec, nrhs=nrhs)
        o = out.view(nrhs, 3).cpu().numpy()
        tol = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-6, "f16": 1e-6}[prec]
        for r in range(nrhs):
            ea, eb = c.half(ca, 0, r), c.half(cb, 0, r)
            want = oracle.cdot(ea, eb)
            nb2 = oracle.cdot(eb, eb).real
            scale = float(np.sqrt(nb2 * oracle.cdot(ea, ea).real))
            assert abs(o[r, 0] - want.real) <= tol * scale
            assert abs(o[r, 1] - want.imag) <= tol * scale
            assert abs(o[r, 2] - nb2) <= tol * nb2
    finally:
        c.close()


def test_noalloc_rejects_too_many_rhs():
    c = Case((4, 4, 4, 4), kappa=0.12, kind="haar", seed=9, precs=("f64", "f32"))
    try:
        f = c.g.field("f32", 1)
        out = torch.zeros(3 * 65, dtype=torch.float64, device="cuda")
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wl_cdot_noalloc(out, f, f, c.Vh, wilson.WL_F32, 65)
        assert e.value.code == wilson.WL_ERR_ARG
    finally:
        c.close()


def test_noalloc_rejects_f16_rows_off_16_bytes():
    c = Case((4, 4, 4, 4), kappa=0.12, kind="haar", seed=9, precs=("f64", "f16"))
    try:
        f = c.g.field("f16", 2)
        out = torch.zeros(6, dtype=torch.float64, device="cuda")
        with pytest.raises(wilson.WilsonError) as e:
            wilson.wl_cdot_noalloc(out, f, f, 126, wilson.WL_F16, 1)
        assert e.value.code == wilson.WL_ERR_ARG
    finally:
        c.close()
