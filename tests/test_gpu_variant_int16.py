"""The int16 fixed-point spinor build (-DWL_SPINOR16_FIXED=1) on the GPU.

The default library stores WL_F16 spinor words as binary16; a build with
WL_SPINOR16_FIXED=1 stores them as int16 fixed point of the site-scaled values
(the same 52 bytes per site).  This test builds that variant into a separate
directory and runs, in a child process loading it (WL_LIBRARY), the tests that
exercise the 16-bit spinor words: the per-component codec bound (which checks
the int16 rounding bound when wl_spinor16_format() reports 1), the FP16
hopping term, D and M_ee against the oracle, and FP16 solves.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_int16_spinor_build_passes_the_fp16_tests(tmp_path):
    from paper_1811_00893_gb300 import build
    lib = build.build(extra=("-DWL_SPINOR16_FIXED=1",), out_dir=str(tmp_path))
    env = dict(os.environ, WL_LIBRARY=lib)
    probe = subprocess.run([sys.executable, "-c",
                            "from paper_1811_00893_gb300 import wilson; print(wilson.wl_spinor16_format())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0, probe.stderr[-2000:]
    assert probe.stdout.strip() == "1"
    sel = ("codec_error_bound or (dslash_matches_oracle and f16) or (full_D_matches_oracle and f16) or "
           "(Mee_matches_oracle and f16) or (solve_schemes and fp16) or fp16_error_margins")
    out = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-k", sel,
                          "tests/test_gpu_parity.py", "tests/test_gpu_solve.py"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert " passed" in out.stdout and "failed" not in out.stdout
