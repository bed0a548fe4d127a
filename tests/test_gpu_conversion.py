"""The int64 -> FP32 conversion of the FP32 density pass (fixed-point map ->
transform input) is done with 32-bit integer and FP32 operations; it must
equal round-to-nearest-even, bit for bit: checked against the GPU's own
conversion instruction and against the host's (numpy) on random values of
every magnitude, exact ties (both parities of the kept mantissa), the 2^24
boundary and the int64 extremes."""
import numpy as np
import pytest

from paper_2403_09070_gb300 import place3d as P

pytestmark = pytest.mark.gpu


def _values():
    rng = np.random.default_rng(11)
    v = [0, 1, -1, 2**24 - 1, 2**24, 2**24 + 1, -(2**24) - 1, 2**25 + 1, 2**25 + 3,
         2**63 - 1, -(2**63), -(2**63) + 1, 2**62 + 2**38, 2**62 + 2**38 + 1]
    for e in range(0, 63):
        lo, hi = 2**e, 2**(e + 1) - 1
        u = rng.integers(lo, hi, size=64, endpoint=True, dtype=np.uint64).astype(np.int64)
        v += list(u) + list(-u)
    for sh in range(1, 40):  # exact ties m 2^sh + 2^(sh-1), m a 24-bit mantissa of either parity
        for m in (2**23, 2**23 + 1, 2**24 - 2, 2**24 - 1, 3 * 2**21 + 7):
            t = m * 2**sh + 2**(sh - 1)
            if t < 2**63:
                v += [t, -t, t - 1, t + 1]
    return np.array(v, dtype=np.int64)


def test_ll2f_matches_round_to_nearest_even():
    vals = _values()
    out, bad = P.ll2f_selftest(vals)
    assert bad == 0
    np.testing.assert_array_equal(out.view(np.uint32), vals.astype(np.float32).view(np.uint32))
