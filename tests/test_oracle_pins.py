"""The FP64 oracle against its pins (CPU only)."""
import pytest

from oracle import pmace_oracle
from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(pmace_oracle)
