"""Host logic of bench.py and of the serving-mix generators (no GPU).

- the ncu traffic lookup returns a stored figure only while the kernel's
  sources are unchanged (source hash), and null once they change;
- the serving mix draws nside, kind and tolerance in the stated proportions,
  reproducibly for a seed; Poisson arrivals have the stated mean rate."""
import json
import os
import shutil
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_lookup_follows_the_kernel_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1801_05358_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in ["dm_ring.cu", "dm_fft.cuh", "dm_internal.h"]:
        shutil.copy(os.path.join(ROOT, "paper_1801_05358_gb300", "csrc", fn), csrc / fn)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    h = bench.kernel_source_hash("k_ring_iter")
    tab = {"k_ring_iter@w": {"dram_bytes_per_launch": 123.0, "source_hash": h}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(tab))
    assert bench.traffic_for("k_ring_iter", "w") == 123.0
    assert bench.traffic_for("k_ring_iter", "other") is None
    with open(csrc / "dm_ring.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench.kernel_source_hash("k_ring_iter") != h
    assert bench.traffic_for("k_ring_iter", "w") is None


def test_serving_stream_proportions_and_reproducibility():
    n = 4000
    a = W.serving_stream(n, 7)
    b = W.serving_stream(n, 7)
    assert a == b
    assert W.serving_stream(n, 8) != a
    nsides = [r["nside"] for r in a]
    assert set(nsides) == {64, 128, 256, 512, 1024}
    for ns in set(nsides):
        assert abs(nsides.count(ns) / n - 0.2) < 4 * np.sqrt(0.2 * 0.8 / n)
    wf = sum(1 for r in a if r["kind"] == 0) / n
    assert abs(wf - 0.7) < 4 * np.sqrt(0.7 * 0.3 / n)
    tols = [r["tol"] for r in a]
    assert set(tols) == {1e-5, 1e-8}
    assert abs(tols.count(1e-5) / n - 0.5) < 4 * np.sqrt(0.25 / n)
    assert all(r["lmax"] == 2 * r["nside"] for r in a)
    assert len({r["seed"] for r in a}) == n


def test_poisson_arrivals_rate():
    t = W.poisson_arrivals(20000, 2.5, 3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert gaps.mean() == pytest.approx(1 / 2.5, rel=0.03)
    assert gaps.std() == pytest.approx(1 / 2.5, rel=0.05)  # exponential gaps


def test_whole_job_value_and_schedule_split():
    assert bench.whole_job_value(64, 256, 2, 1000.0) == pytest.approx(64 * 256 * 2 / 1.0)
    for k in [1, 7, 10, 256]:
        s = bench.iters_split(k)
        assert sum(s) == k and max(s) - min(s) <= 1 and len(s) == 10


def test_single_thread_baseline_leg():
    """The bench's single-core oracle leg: one iteration at a quarter of the
    nside (here the nside 16 floor) in a child process with one OpenMP
    thread, scaled by the ratio of (l, m, ring pair) triples."""
    out = bench.single_thread_baseline(32, 64)
    assert "error" not in out, out
    assert out["cores"] == 1
    assert out["seconds_per_iteration_sample"] > 0.0
    ns, lm = 16, 32
    triples = lambda n, l: (l + 1) * (l + 2) // 2 * 2 * n  # noqa: E731
    scale = triples(32, 64) / triples(ns, lm)
    assert out["value_extrapolated"] == pytest.approx(1.0 / (out["seconds_per_iteration_sample"] * scale))
    assert "nside 16, lmax 32" in out["sample"]
