"""The C ABI used from plain C: paper_2403_09070_gb300/examples/place3d_minimal.c
compiles with gcc -Wall -Wextra -Werror against include/place3d.h and links
against libplace3d.so (CPU); on a GPU its objective and gradient equal the
oracle's for the same problem (FP64, 1e-9)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from helpers import problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2403_09070_gb300")
SRC = os.path.join(PKG, "examples", "place3d_minimal.c")


def _compile(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no C compiler")
    from paper_2403_09070_gb300 import place3d as P
    P.load_library()  # builds libplace3d.so if it is missing
    exe = str(tmp_path / "place3d_minimal")
    cmd = [gcc, "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
           "-L", PKG, "-lplace3d", "-Wl,-rpath," + PKG, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_compiles_and_links(tmp_path):
    _compile(tmp_path)


def _same_problem():
    # the problem place3d_minimal.c builds
    wb = [1, 2, 3, 1, 2, 4, 6]
    hb = [1, 1, 1, 1, 1, 1, 6]
    sizes = [(w, h, 0.8 * w, 0.8 * h) for w, h in zip(wb, hb)]
    nets = [[0, 1, 6], [2, 3], [1, 4, 5, 6]]
    obx = [0.2, -0.3, 1.0, 0.0, 0.1, 0.2, -0.4, 0.3, -1.5]
    oby = [0.1, 0.2, -1.0, 0.3, -0.2, 0.0, 0.1, -0.3, 2.0]
    off = np.array([(a, b, 0.8 * a, 0.8 * b) for a, b in zip(obx, oby)])
    p = problem(sizes, nets=nets, offsets=off, die=(0.0, 0.0, 32.0, 32.0), grid=(16, 16, 2), macros=[6],
                gamma=8.0, lam=1e-3)
    x = np.array([5, 9, 14, 18, 22, 26, 12], np.float64)
    y = np.array([6, 11, 20, 24, 8, 15, 16], np.float64)
    z = np.array([2.7, 1.2, 2.9, 1.4, 2.5, 1.1, 2.0])
    return p, x, y, z


@pytest.mark.gpu
def test_c_example_matches_the_oracle(tmp_path):
    from gpu_harness import rel_max
    from oracle import Oracle
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    vals, grads = {}, {}
    for line in r.stdout.splitlines():
        f = line.split()
        if f[0] == "grad":
            grads[int(f[1])] = [float(v) for v in f[2:5]]
        else:
            vals[f[0]] = float(f[1])
    p, x, y, z = _same_problem()
    ref = Oracle(p).eval(x, y, z, density_mode=1)
    for k in ("obj", "wl_bi", "wl_z", "energy", "hpwl_d2d"):
        assert vals[k] == pytest.approx(ref[k], rel=1e-9), k
    assert vals["n_cross"] == ref["n_cross"]
    g = np.array([grads[i] for i in range(p["n_inst"])])
    for c, k in enumerate(("gx", "gy", "gz")):
        assert rel_max(g[:, c], ref[k]) < 1e-9, k
