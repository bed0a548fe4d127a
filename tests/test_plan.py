"""The wirelength launch-plan logic of the autotuner (host code in
csrc/plan.h), compiled with g++ into a small driver and checked against
brute force: every split of the degree classes into runs of at most `span`
adjacent classes, each run with its fastest fitting form."""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ is not available")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_harness")
    subprocess.run([gxx, "-std=c++17", "-O1", "-o", exe, os.path.join(HERE, "plan_harness.cpp")], check=True)
    return exe


def _run(exe, t, span, lanes, tol):
    nd, _, nf = t.shape
    lines = [f"{nd} {nf} {span} {tol}", " ".join(str(v) for v in lanes)]
    lines += [" ".join(repr(float(v)) for v in t[i, j]) for i in range(nd) for j in range(nd)]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    return [tuple(int(v) for v in ln.split()) for ln in out.splitlines()]


def _ties(t, lanes, tol):
    """Of the forms within (1 + tol) of a run's fastest: the fewest lanes, then the faster."""
    t = t.copy()
    nd, _, nf = t.shape
    for i in range(nd):
        for j in range(i, nd):
            row = t[i, j]
            ok = [f for f in range(nf) if row[f] >= 0]
            if not ok:
                continue
            tmin = min(row[f] for f in ok)
            near = [f for f in ok if row[f] <= np.float32(1 + tol) * tmin]
            keep = min(near, key=lambda f: (lanes[f], row[f], f))
            for f in range(nf):
                if f != keep:
                    row[f] = -1
    return t


def _brute(t, span):
    """Least total time over every split into runs of at most `span` classes."""
    nd = t.shape[0]
    best = None
    for cuts in itertools.product([0, 1], repeat=max(nd - 1, 0)):
        bounds = [0] + [k + 1 for k, c in enumerate(cuts) if c] + [nd]
        runs = list(zip(bounds[:-1], bounds[1:]))
        if any(b - a > span for a, b in runs):
            continue
        total = 0.0
        for a, b in runs:
            ok = [v for v in t[a, b - 1] if v >= 0]
            if not ok:
                total = None
                break
            total += float(min(ok))
        if total is not None and (best is None or total < best):
            best = total
    return best


def _check_split(t, runs, span):
    nd = t.shape[0]
    assert runs[0][0] == 0 and runs[-1][1] == nd - 1
    for (a, b, f), nxt in zip(runs, runs[1:] + [None]):
        assert b - a + 1 <= span and t[a, b, f] >= 0
        if nxt:
            assert nxt[0] == b + 1
    return sum(float(t[a, b, f]) for a, b, f in runs)


@pytest.mark.parametrize("seed", range(12))
def test_best_split_matches_brute_force(driver, seed):
    rng = np.random.default_rng(seed)
    nd, nf = int(rng.integers(1, 8)), 5
    lanes = [1, 2, 4, 8, 16]
    t = rng.uniform(1.0, 20.0, (nd, nd, nf)).astype(np.float32)
    t[rng.random((nd, nd, nf)) < 0.3] = -1
    for i in range(nd):  # every class fits at least its own single-class run
        t[i, i, int(rng.integers(nf))] = np.float32(rng.uniform(5, 30))
    for span in sorted({1, 2, nd}):
        for tol in (-1.0, 0.03, 0.2):
            tt = _ties(t, lanes, tol) if tol >= 0 else t
            runs = _run(driver, t, span, lanes, tol)
            total = _check_split(tt, runs, span)
            assert total == pytest.approx(_brute(tt, span), rel=1e-12), (span, tol)


def test_near_ties_go_to_fewer_lanes(driver):
    lanes = [16, 4]
    t = np.array([[[10.0, 10.2]]], np.float32)
    assert _run(driver, t, 1, lanes, 0.03) == [(0, 0, 1)]  # 2 % slower, 4 lanes: kept
    assert _run(driver, t, 1, lanes, -1) == [(0, 0, 0)]    # without the rule: the fastest
    t = np.array([[[10.0, 10.5]]], np.float32)
    assert _run(driver, t, 1, lanes, 0.03) == [(0, 0, 0)]  # 5 % slower: not a tie
    t = np.array([[[10.2, 10.0]]], np.float32)
    assert _run(driver, t, 1, [4, 4], 0.03) == [(0, 0, 1)]  # equal lanes: the faster


def test_uncoverable_class_gives_no_plan(driver):
    t = np.full((2, 2, 2), -1, np.float32)
    t[0, 0, 0] = 3.0  # class 1 fits no form, alone or with class 0
    assert _run(driver, t, 2, [1, 2], -1) == []


def test_span_limits_the_runs(driver):
    # one long run is cheapest, but span 2 forbids it
    nd = 4
    t = np.full((nd, nd, 1), 10.0, np.float32)
    t[0, 3, 0] = 1.0
    assert _run(driver, t, nd, [1], -1) == [(0, 3, 0)]
    runs = _run(driver, t, 2, [1], -1)
    assert all(b - a + 1 <= 2 for a, b, _ in runs) and _check_split(t, runs, 2) == 20.0
