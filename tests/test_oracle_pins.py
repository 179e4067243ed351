"""The FP64 oracle against what the paper and the mathematics fix (CPU)."""
import pytest

from oracle import magpie_oracle as O
from tests import pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__[6:])
def test_oracle_pin(check):
    check(O)
