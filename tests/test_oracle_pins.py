"""The CPU oracle, as committed, against its pins (no GPU)."""
import pytest

import oracle
import oracle_pins as pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    check(oracle.default())


def test_brute_force_helper_on_golden():
    # the pure-Python counter used as a pin agrees with the hand-worked fixtures
    import numpy as np
    for name in pins.GOLDEN_FILES:
        d = pins.load_golden(name)
        H = pins.brute_integral_histogram(d["image"], d["bins"]).astype(np.int64)
        for b, plane in d["planes"].items():
            assert np.array_equal(H[b], plane), (name, b)
