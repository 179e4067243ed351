"""Pins of the learned-correction oracle (CPU only)."""
import pytest

from oracle import learned_oracle as L
from tests import learned_pins


@pytest.mark.parametrize("check", learned_pins.ALL, ids=lambda f: f.__name__)
def test_learned_oracle_pin(check):
    check(L)
