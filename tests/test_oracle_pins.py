"""The FP64 oracle against facts fixed outside it (hand traces from §III,
closed forms, invariants, brute force, a library special case)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check()
