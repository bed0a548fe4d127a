"""CPU checks of the C ABI: the library builds and loads, exports every entry
point include/place3d.h declares, and rejects bad problems before touching a
GPU."""
import os
import re

import numpy as np
import pytest

from helpers import problem
from paper_2403_09070_gb300 import place3d as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(place3d_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = P.load_library()
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert set(P.EXPORTS) <= declared


def test_alpha_helper():
    # the library's alpha and the oracle's alpha are two independent codings
    from oracle import lib as olib
    for args in ((200.0, 6.25, 10.0, 1.0, 0.8, 1.0), (6700.0, 52.3, 5.0, 0.5, 0.768, 1.4)):
        assert P.alpha(*args) == pytest.approx(olib().orc_alpha(*args), rel=1e-15)


def _bad(**kw):
    p = problem([(1.0, 1.0, 0.8, 0.8)] * 4, nets=[[0, 1], [2, 3]], die=(0, 0, 8, 8), grid=(4, 4, 2))
    p.update(kw)
    return p


@pytest.mark.parametrize("mut,code", [
    (dict(net_start=np.array([0, 2, 3], np.int32)), -2),                 # last != n_pin
    (dict(net_start=np.array([0, 3, 2], np.int32)), -2),                 # decreasing
    (dict(pin_inst=np.array([0, 1, 2, 9], np.int32)), -2),               # out of range
    (dict(pin_inst=np.array([0, 0, 2, 3], np.int32)), -2),               # instance twice on a net
    (dict(nx=0), -1), (dict(nz=17), -1), (dict(xh=-1.0), -1), (dict(gamma=0.0), -1),
])
def test_create_rejects_bad_problems(mut, code):
    with pytest.raises(P.Place3DError) as ei:
        P.Place3D(_bad(**mut), precision="fp64")
    assert ei.value.code == code


def test_create_rejects_unknown_precision():
    with pytest.raises(P.Place3DError) as ei:
        P.Place3D(_bad(), precision=7)
    assert ei.value.code == -1
