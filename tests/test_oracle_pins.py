"""The FP64 oracle against what the paper and the mathematics fix."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


@pytest.mark.slow
def test_wmmse_ammmse_agree():
    pins.pin_wmmse_ammmse_agree()
