"""The CPU oracle against the paper's printed numbers, closed forms of
classical electrodynamics, invariants of the method and brute force."""
import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()
