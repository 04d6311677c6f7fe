"""Host-side pieces of bench.py, on the CPU: the one-sided timing statistic
of Sec. 2.1 (reading R-10: sigma_L^2 = sum over t_i < T of (t_i - T)^2 /
(n/2 - 1), likewise sigma_H above the mean), and the DRAM traffic record's
guards (it is reported only for the kernel sources and the workload it was
taken on)."""

import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_one_sided_sigma_symmetric_sample():
    # four below the mean at distance 1, four above at distance 1: n = 8,
    # n/2 - 1 = 3, sigma_L = sigma_H = sqrt(4 / 3)
    ts = [9.0] * 4 + [11.0] * 4
    T, lo, hi = bench.one_sided_sigma(ts)
    assert T == 10.0
    assert math.isclose(lo, math.sqrt(4 / 3)) and math.isclose(hi, math.sqrt(4 / 3))


def test_one_sided_sigma_skewed_sample():
    # one slow outlier: the deviation shows above the mean only
    ts = [1.0] * 9 + [11.0]
    T, lo, hi = bench.one_sided_sigma(ts)
    assert math.isclose(T, 2.0)
    d = 10 / 2 - 1
    assert math.isclose(lo, math.sqrt(9 * 1.0 / d))
    assert math.isclose(hi, math.sqrt(81.0 / d))
    assert hi > lo


def test_traffic_record_guards(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    alg = rec["alg_bytes_per_launch"]
    # the record's own fields are consistent
    assert rec["traffic_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert rec["hashed_sources"] == bench.FX_KERNEL_SOURCES
    # another workload, or other sources, give no traffic figure
    assert bench.committed_traffic(alg + 8) is None
    fake = dict(rec, source_hash="0" * 16)
    root = tmp_path
    os.makedirs(root / "profiles")
    json.dump(fake, open(root / "profiles" / "traffic.json", "w"))
    real = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: real)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.committed_traffic(alg) is None
