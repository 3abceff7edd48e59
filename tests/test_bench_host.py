"""Host-side logic of bench.py on the CPU: the serving leg's bookkeeping against a
fake server, and the lookup of DRAM traffic in the committed ncu summary."""
import hashlib
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeServer:
    """Answers every request at once: 2 ms latency, a fixed result, and a skip count of
    n (so that evaluated pairs = n(n-1) - n)."""

    def __init__(self, **kw):
        self.reqs = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def submit(self, x, prec):
        self.reqs.append((x.size, prec))
        return len(self.reqs) - 1

    def poll(self, t, timeout_ms=0):
        n, prec = self.reqs[t]
        res = {"status": 0, "psi6": -1.0, "psi4": 1.0, "h": 0.1, "g2": 0.2}
        tm = {"t_submit_ns": 1000 * t, "t_admit_ns": 1000 * t + 10, "t_done_ns": 1000 * t + 2_000_000,
              "skipped6": n, "skipped4": 0}
        return res, tm


@pytest.fixture()
def fake_kde(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    return types.SimpleNamespace(Server=_FakeServer, KDE_FP32=0, KDE_FP64=1)


def test_serving_leg_counts_evaluated_pairs_and_writes_each_replay(fake_kde, tmp_path):
    import synthdata
    count = 40
    out = bench.serve_leg(fake_kde, 4e14, count, [0.5, 0.8], "also", str(tmp_path / "s"), fp64_random=3)
    ns = [s.n for s in synthdata.server_specs()[:count]]
    for load in ("0.5", "0.8"):
        s = out["fp32"][f"load_{load}"]
        assert s["requests"] == count and s["status_ok"] == count
        assert s["pair_evals"] == sum(n * (n - 1) - n for n in ns)
        assert s["pairs_skipped"] == sum(ns)
        assert abs(s["latency_ms"]["p50"] - 2.0) < 1e-6
        rec = json.load(open(tmp_path / f"s.fp32_load{load}.json"))
        assert len(rec["requests"]) == count and rec["summary"]["pair_evals"] == s["pair_evals"]
    sub = out["fp64_subset"]
    small = sum(n <= 65536 for n in ns)
    assert sub["requests"] == small + min(3, count - small)
    assert "fp32_same_requests_in_the_fp32_replay" in sub
    assert os.path.exists(tmp_path / "s.fp64_subset_load0.5.json")


def test_serving_leg_fp64_only_skips_the_fp32_replays(fake_kde, tmp_path):
    out = bench.serve_leg(fake_kde, 4e14, 30, [0.8], "only", None, fp64_random=0)
    assert out["fp32"] == {}
    assert "fp32_same_requests_in_the_fp32_replay" not in out["fp64_subset"]
    assert out["fp64_subset"]["selection"].startswith("n <= 65536 plus 0 random")


def test_traffic_lookup_follows_the_kernel_source_hash():
    text = open(bench.TRAFFIC_FILE).read()
    recorded = [line for line in text.splitlines() if line.startswith("- kernel_source_sha256:")][0]
    current = hashlib.sha256(open(bench.KERNEL_SOURCE, "rb").read()).hexdigest()
    if current in recorded:
        assert bench.measured_traffic(2) == 12731392.0
        assert bench.measured_traffic(0) is None          # not captured with this source
        assert bench.measured_traffic(7) is None          # no such configuration recorded
    else:                                                 # kernel changed since the capture
        assert bench.measured_traffic(2) is None
