"""The CPU oracle against facts fixed by the paper and by mathematics
(see oracle_pins.py for each source of truth)."""
import pytest

import oracle_pins


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check()
