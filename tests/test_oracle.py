"""The serial oracle against facts it does not compute itself (CPU only)."""
import os, sys
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import pytest

import oracle
from oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle.default())


def test_oracle_rejects_undefined_clauses():
    import numpy as np
    x = np.zeros(3, dtype=np.float32)
    for op in ["band", "bor", "bxor", "land", "lor"]:
        with pytest.raises(ValueError):
            oracle.reduce(x, op, "f32")
    with pytest.raises(ValueError):
        oracle.reduce(np.zeros(3, dtype=np.int64), "add", "i32")   # narrowing
    with pytest.raises(ValueError):
        oracle.reduce(np.zeros(3, dtype=np.int32), "add", "f64")   # int into fp
