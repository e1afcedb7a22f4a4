"""wl_cdot_noalloc, the allocation-free dot/norm entry point, against wl_cdot.

Some callers cannot allocate device memory (they run inside another
framework's memory pool, or in loops where cudaMalloc would synchronise the
device, or hold field pointers without a gauge object); wl_cdot_noalloc serves
them from a fixed built-in scratch array.  This file is collected last so a
run that stops at the first failure has already run every other test; it
also passes alone in a fresh process (its first call sets up the scratch).
"""
import pytest
import torch

from gpu_helpers import PRECS, Case
from paper_1811_00893_gb300 import wilson

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (24, 24, 24, 48)], ids=["Vh960", "Vh331776"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_noalloc_matches_wl_cdot_on_two_calls(dims, prec):
    c = Case(dims, kappa=0.12, kind="haar", seed=9, precs=("f64", "f32", "f16"))
    try:
        nrhs = 3
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
