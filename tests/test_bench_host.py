"""Host logic of bench.py (no GPU): the algorithmic bytes per stage it
divides by the measured times match the per-unit formulas stated for the
1M-cell workload, and the profiled-traffic lookup refuses stale captures."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2403_09070_gb300 import synth  # noqa: E402


def test_algorithmic_bytes_at_1m_cells():
    p = synth.make_problem("cells_1m")
    a = bench.algorithmic(p, "fp32_tc")["bytes"]
    n, P, E = p["n_inst"], p["n_pin"], p["n_net"]
    B = p["nx"] * p["ny"] * p["nz"]
    assert a["wirelength"] == 12 * n + 20 * P + 4 * E + 12 * n
    assert a["scatter"] == 28 * n + 8 * B
    assert a["final"] == 28 * n + 12 * B + 12 * n
    assert a["wirelength"] == pytest.approx(116.7e6, rel=2e-3)
    assert a["scatter"] == pytest.approx(36.4e6, rel=2e-3)
    assert a["final"] == pytest.approx(52.6e6, rel=2e-3)
    # FP64 doubles the real-valued terms
    b = bench.algorithmic(p, "fp64")["bytes"]
    assert b["wirelength"] == 24 * n + 36 * P + 4 * E + 24 * n


def test_profiled_traffic_is_keyed_to_the_sources(tmp_path, monkeypatch):
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    e = t["cells_1m"]["fp32_tc"]["wirelength"]
    assert set(e["sources"]) and e["bytes_per_eval"] > 0
    # a copy of the repository layout whose entry is keyed to the copied
    # sources: the lookup returns the bytes; one listed source changed: None
    import hashlib
    prof = tmp_path / "profiles"
    prof.mkdir()
    for path in e["sources"]:
        dst = tmp_path / path
        dst.parent.mkdir(parents=True, exist_ok=True)
        data = open(os.path.join(ROOT, path), "rb").read()
        dst.write_bytes(data)
        e["sources"][path] = hashlib.sha256(data).hexdigest()
    (prof / "traffic.json").write_text(json.dumps(t))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profiled_traffic("wirelength", "cells_1m", "fp32_tc") == e["bytes_per_eval"]
    first = next(iter(e["sources"]))
    with open(tmp_path / first, "ab") as f:
        f.write(b"\n// changed\n")
    assert bench._profiled_traffic("wirelength", "cells_1m", "fp32_tc") is None
