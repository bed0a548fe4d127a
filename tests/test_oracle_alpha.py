"""Pin of the HBT penalty factor alpha (Sec. V-A): the oracle's coding, and
the library's independent coding, against values worked out by hand
(tests/golden/alpha_example.txt).  A base-10 logarithm, a wrong eta or a
dropped "- 1" in the logarithm's argument changes every nonzero row."""
import math

import pytest

from helpers import read_golden


def _rows():
    out = []
    for r in read_golden("alpha_example.txt"):
        k = r.index("|")
        args = tuple(float(v) for v in r[:k])
        eta, arg, ln, alpha = (float(v) for v in r[k + 1:])
        out.append((args, eta, arg, ln, alpha))
    return out


ROWS = _rows()


def test_golden_rows_are_consistent():
    """The hand-derived intermediates (eta, the argument, its logarithm) follow
    from the row's parameters, so each row states one reading of the formula."""
    assert len(ROWS) == 4
    for (dx, dz, beta, w, rht, rhb), eta, arg, ln, alpha in ROWS:
        assert 2.0 * w / (rht + rhb) == pytest.approx(eta, rel=1e-15)
        assert 90.0 * beta * eta - 1.0 == pytest.approx(arg, rel=1e-12, abs=1e-12)
        assert math.exp(ln) == pytest.approx(arg, rel=1e-12)


@pytest.mark.parametrize("row", range(4))
def test_oracle_alpha_matches_hand_values(row):
    from oracle import lib
    args, _, _, _, alpha = ROWS[row]
    assert lib().orc_alpha(*args) == pytest.approx(alpha, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("row", range(4))
def test_library_alpha_matches_hand_values(row):
    from paper_2403_09070_gb300 import place3d as P
    args, _, _, _, alpha = ROWS[row]
    assert P.alpha(*args) == pytest.approx(alpha, rel=1e-12, abs=1e-15)


def test_plausible_mistakes_miss_the_pin():
    """Each plausible misreading of the formula misses row (d) by far more
    than the pin's tolerance."""
    (dx, dz, beta, w, rht, rhb), _, _, _, alpha = ROWS[3]
    eta = 2.0 * w / (rht + rhb)
    wrong = [
        3.5e-3 * dx * eta * eta / dz * math.log10(90 * beta * eta - 1),      # base-10 log
        3.5e-3 * dx * (w / (rht + rhb)) ** 2 / dz * math.log(90 * beta * w / (rht + rhb) - 1),  # eta without 2
        3.5e-3 * dx * eta * eta / dz * math.log(90 * beta * eta),            # no "- 1"
        3.5e-3 * dx * eta / dz * math.log(90 * beta * eta - 1),              # eta not squared
    ]
    for v in wrong:
        assert abs(v - alpha) > 1e-6 * alpha
