"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("name", list(P.ALL))
def test_pin(name):
    ok, detail = P.ALL[name](0)
    assert ok, detail
