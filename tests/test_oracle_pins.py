"""The FP64 oracle against its pins (CPU only)."""
import pytest

import oracle.cs_oracle as O
from oracle_pins import ALL_CHECKS


@pytest.mark.parametrize("check", ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check(O)
