"""The CPU oracle checked against brute force, closed forms, invariants and
hand-worked examples (see ``pins.py``)."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin()
