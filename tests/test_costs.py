"""The cost model against the paper's printed Table 1 (tests/golden)."""
import json
import os

import pytest

from paper_1811_00893_gb300 import costs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_cost_model.json")


@pytest.fixture(scope="module")
def table1():
    with open(GOLDEN) as f:
        return json.load(f)


def test_flops_per_site(table1):
    assert costs.FLOPS_D_SITE == table1["wilson"]["flop_per_site"]
    assert costs.FLOPS_HOP_SITE == 1320  # the standard Dslash count, D without 1 - kappa*


def test_bytes_per_site(table1):
    w = table1["wilson"]
    assert costs.paper_bytes_per_site(4) == w["bytes_per_site_float"]
    assert round(costs.paper_byte_per_flop(), 2) == w["byte_per_flop"]
    assert round(costs.paper_byte_per_flop(ideal_reuse=True), 3) == w["byte_per_flop_ideal"]


def test_roofline_columns(table1):
    # Table 1 divides the bandwidth by the printed (rounded) Byte/Flop values
    w, bw = table1["wilson"], table1["bandwidth_gbs"]
    bf = round(costs.paper_byte_per_flop(), 2)
    bf_ideal = round(costs.paper_byte_per_flop(ideal_reuse=True), 3)
    assert int(bw["ofp_mcdram_low"] / bf) == w["roofline_ofp_gflops"]
    assert abs(bw["ofp_mcdram_low"] / bf_ideal - w["roofline_ofp_ideal_gflops"]) < 5
    assert int(bw["ito"] / bf) == w["roofline_ito_gflops"]
    assert int(bw["ito"] / bf_ideal) == w["roofline_ito_ideal_gflops"]
    # unrounded model is within 1% of the printed columns
    assert abs(costs.roofline_gflops(bw["ito"]) / w["roofline_ito_gflops"] - 1) < 0.01


def test_hop_kernel_bytes():
    # even-odd hop: 8 links x 18 reals + 24 in + 24 out
    assert costs.hop_bytes_per_site("f32") == 768
    assert costs.hop_bytes_per_site("f64") == 1536
    assert costs.hop_bytes_per_site("f16") == 8 * 36 + 2 * 52
    # 12 RHS share one read of the links
    assert costs.hop_bytes_per_site("f32", nrhs=12) == 576 + 12 * 192
