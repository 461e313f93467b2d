"""configs/traffic_from_ncu.py: the DRAM/algorithmic ratio of the batched CG stencil from an
ncu CSV, keeping only launches that move the bytes of a k-RHS product, one entry per
(stencil sources, variant, link form)."""
import csv
import importlib.util
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load():
    spec = importlib.util.spec_from_file_location("traffic_from_ncu", os.path.join(ROOT, "configs", "traffic_from_ncu.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _csv(path, launches):
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value", "Extra"])
        for i, (rd, wr) in enumerate(launches):
            w.writerow([str(i), "k", "dram__bytes_read.sum", "byte", str(rd), "x"])
            w.writerow([str(i), "k", "dram__bytes_write.sum", "Mbyte", str(wr / 1e6), "x"])
            w.writerow([str(i), "k", "gpu__time_duration.sum", "ns", "1000", "x"])


def test_ratio_filter_and_entries(tmp_path, monkeypatch):
    m = _load()
    monkeypatch.setattr(m, "ROOT", str(tmp_path))
    os.makedirs(tmp_path / "configs")
    monkeypatch.setattr(m, "stencil_sha1", lambda: "abc")
    alg = m.cg_algorithmic_bytes(1000, 16, 12)
    assert alg == 1000 * (4 * 48 + 16 * 3 * 96)
    path = str(tmp_path / "c.csv")
    # two single-RHS launches (dropped) and two 16-RHS launches at 0.9 and 1.1 of alg
    _csv(path, [(1000, 500), (0.6 * alg, 0.3 * alg), (0.5 * alg, 0.6 * alg), (2000, 10)])
    for variant in (4, 4, 12):
        monkeypatch.setattr(sys, "argv", ["x", path, "--sites", "1000", "--k", "16", "--links", "12",
                                          "--variant", str(variant)])
        m.main()
    data = json.load(open(tmp_path / "configs" / "traffic.json"))["dslash_cg_f32_k16"]
    assert [(e["variant"], e["link_reals"]) for e in data] == [(4, 12), (12, 12)]  # re-capture replaced
    assert data[0]["launches_captured"] == 2
    assert data[0]["dram_over_algorithmic"] == pytest.approx(1.0)
    # no k-RHS launch at all: refused
    _csv(path, [(1000, 500)])
    monkeypatch.setattr(sys, "argv", ["x", path, "--sites", "1000", "--k", "16", "--variant", "6"])
    with pytest.raises(SystemExit):
        m.main()
