"""The FP64 oracle against closed forms, invariants and brute force.

Each test runs one check from ``oracle_pins`` (its docstring lists what pins
what).  None of these checks re-types the oracle's own code: they compare it
with a dense matrix assembled independently from Eq. 1, with the free-field
closed forms, with algebraic identities the Wilson matrix must satisfy, and
with dense LU / FFT solutions.
"""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    check()
