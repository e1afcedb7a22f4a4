"""The oracle's clover operator (Eq. 2) against its pins (oracle_clover_pins)."""
import pytest

import oracle_clover_pins as C


@pytest.mark.parametrize("check", C.CLOVER_CHECKS, ids=lambda c: c.__name__)
def test_clover_pin(check):
    check()
