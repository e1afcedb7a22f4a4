"""Planted mistakes in the oracle must be caught by the pins.

Each case copies ``oracle/wilson_oracle.c``, plants one plausible mistake by a
text substitution (a dropped term, a wrong sign, a missing adjoint, a wrong
index, a transposed operand ...), compiles it into a temporary library and
runs the pin checks through it.  At least one check must fail for every
mutant; otherwise the pins would not notice that mistake in the oracle.
"""
import os
import tempfile

import pytest

import oracle
import oracle_clover_pins as C
import oracle_pins as P

MUTANTS = {
    "forward projector sign": ("add_term(out_site, mu, -(double)d, U + (s * 4 + mu)",
                               "add_term(out_site, mu, +(double)d, U + (s * 4 + mu)"),
    "backward projector sign": ("add_term(out_site, mu, +(double)d, U + (b * 4 + mu)",
                                "add_term(out_site, mu, -(double)d, U + (b * 4 + mu)"),
    "backward link not adjoint": ("U + (b * 4 + mu) * LINK_REALS, 1,",
                                  "U + (b * 4 + mu) * LINK_REALS, 0,"),
    "backward link at wrong site": ("U + (b * 4 + mu) * LINK_REALS, 1,",
                                    "U + (s * 4 + mu) * LINK_REALS, 1,"),
    "backward phase not conjugated": ("pim = crossed ? -bc[2 * mu + 1] : 0.0;",
                                      "pim = crossed ? bc[2 * mu + 1] : 0.0;"),
    "boundary phase dropped": ("if (v >= L[mu]) { v -= L[mu]; *crossed = 1; }",
                               "if (v >= L[mu]) { v -= L[mu]; *crossed = 0; }"),
    "t direction dropped": ("for (int mu = 0; mu < 4; ++mu) {\n        int crossed;",
                            "for (int mu = 0; mu < 3; ++mu) {\n        int crossed;"),
    "link transposed": ("mre = M[2 * (a * NC + b)];\n                    mim = M[2 * (a * NC + b) + 1];",
                        "mre = M[2 * (b * NC + a)];\n                    mim = M[2 * (b * NC + a) + 1];"),
    "conjugate link": ("mim = M[2 * (a * NC + b) + 1];", "mim = -M[2 * (a * NC + b) + 1];"),
    "identity part of projector dropped": ("double re = w[sp][a][0], im = w[sp][a][1]; /* the identity part */",
                                           "double re = 0.0, im = 0.0; /* the identity part */"),
    "gamma_2 entry sign": ("{{0, 0}, {0, 0}, {0, 0}, {-1, 0}},\n     {{0, 0}, {0, 0}, {1, 0}, {0, 0}},",
                           "{{0, 0}, {0, 0}, {0, 0}, {1, 0}},\n     {{0, 0}, {0, 0}, {1, 0}, {0, 0}},"),
    "kappa sign in D": ("in[s * SITE_REALS + k] - kappa * h[k]", "in[s * SITE_REALS + k] + kappa * h[k]"),
    "kappa not squared in M_ee": ("in_e[k] - kappa * kappa * out_e[k]", "in_e[k] - kappa * out_e[k]"),
    "even-odd source sign": ("be[k] += kappa * tmp[k];", "be[k] -= kappa * tmp[k];"),
    "odd reconstruction sign": ("xo[k] = bo[k] + kappa * tmp[k];", "xo[k] = bo[k] - kappa * tmp[k];"),
    "conjugation dropped in dot": ("si += a[2 * i] * b[2 * i + 1] - a[2 * i + 1] * b[2 * i];",
                                   "si += a[2 * i] * b[2 * i + 1] + a[2 * i + 1] * b[2 * i];"),
    "half index parity": ("return parity_of(L, s) == p ? s : s + 1;",
                          "return parity_of(L, s) != p ? s : s + 1;"),
    "clover block transposed": ("M[6 * b + i][6 * b + j][1] = Fs[2 * ((b * 6 + i) * 6 + j) + 1];",
                                "M[6 * b + i][6 * b + j][1] = Fs[2 * ((b * 6 + j) * 6 + i) + 1];"),
    "clover block on the wrong spins": ("M[6 * b + i][6 * b + j][0] = Fs[2 * ((b * 6 + i) * 6 + j)];",
                                        "M[6 * (1 - b) + i][6 * (1 - b) + j][0] = Fs[2 * ((b * 6 + i) * 6 + j)];"),
    "clover product conjugated": ("im += M[i][j][0] * v[2 * j + 1] + M[i][j][1] * v[2 * j];",
                                  "im += M[i][j][0] * v[2 * j + 1] - M[i][j][1] * v[2 * j];"),
    "clover Schur without inverse": ("orc_clover_diag(F, t1, t2, L, 1, 1);",
                                     "orc_clover_diag(F, t1, t2, L, 1, 0);"),
    "clover even-odd source without inverse": ("orc_clover_diag(F, bo, t1, L, 1, 1);",
                                               "orc_clover_diag(F, bo, t1, L, 1, 0);"),
    "clover reconstruction without inverse": ("orc_clover_diag(F, t1, xo, L, 1, 1);",
                                              "orc_clover_diag(F, t1, xo, L, 1, 0);"),
    "clover solve on the Wilson matrix": ("    if (c->F) {", "    if (0) {"),
    "clover back substitution sign": ("re -= A[i][j][0] * y[2 * j] - A[i][j][1] * y[2 * j + 1];",
                                      "re += A[i][j][0] * y[2 * j] - A[i][j][1] * y[2 * j + 1];"),
}


@pytest.fixture(scope="module")
def source():
    with open(oracle.SOURCE) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, source):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "mutant.c")
        with open(src, "w") as f:
            f.write(source.replace(old, new))
        lib = oracle.compile_source(src, os.path.join(d, "libmutant.so"))
        with oracle.use_library(lib):
            failed = P.failing_checks(P.ALL_CHECKS + C.CLOVER_CHECKS)
    assert failed, f"no pin notices the planted mistake {name!r}"


def test_unmutated_source_passes_all_checks():
    assert P.failing_checks(P.ALL_CHECKS + C.CLOVER_CHECKS) == []
