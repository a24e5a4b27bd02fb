"""The FP64 oracle against facts fixed by mathematics and by the paper (CPU only)."""
import pytest

import oracle_pins as pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(check):
    check()
