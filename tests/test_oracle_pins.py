"""The CPU oracle checked against exact arithmetic, error bounds, worked
results and the closed form of the paper's test product (no GPU)."""
import pytest

import oracle_pins as pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orl, pin):
    pin(orl)
