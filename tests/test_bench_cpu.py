"""Host logic of the benchmark (no GPU): the kernel-evaluation count of a fit
against the oracle's own plan, the clock sampler's matching of samples to the
timed region, and the rule that a stored ncu traffic figure is dropped once
its kernel source changed."""

import datetime
import json
import os

import numpy as np
import pytest

import bench
from oracle import kkm_oracle as O


@pytest.mark.parametrize("N,B,C,s", [(60000, 4, 10, 0.2), (1001, 3, 5, 0.5), (500000, 20, 8, 0.05), (7, 7, 1, 1.0)])
def test_fit_evals_matches_the_oracle_plan(N, B, C, s):
    """Per mini-batch |L| x N_i block entries (Eq. 18 landmarks) plus the two
    C-column blocks (Eq. 8, Eq. 12), and C - 1 k-means++ columns over the first
    mini-batch; mini-batch sizes from the oracle's stride partition."""
    sizes = [len(g) for g in O.minibatch_indices(N, B)]
    want = sum(n * O.n_landmarks(n, s) + 2 * n * C for n in sizes) + (C - 1) * sizes[0]
    assert bench.fit_evals(N, B, C, s) == want


def _line(t, sm, reasons=("Not Active",) * 4):
    ts = t.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, 0, {sm}, 2070, 900.0, 0x0, " + ", ".join(reasons) + "\n"


def test_clock_sampler_keeps_the_timed_region(tmp_path):
    c = bench.ClockSampler(0)
    c.proc = True                     # as if nvidia-smi were running
    c.path = str(tmp_path / "clocks.csv")
    t0 = datetime.datetime.now()
    with open(c.path, "w") as f:
        f.write(_line(t0 - datetime.timedelta(seconds=2), 1000,
                      ("Active", "Not Active", "Not Active", "Not Active")))   # warm-up: slowed, outside
        for dt, sm in ((0.05, 2070), (0.15, 2060), (0.25, 2070)):
            f.write(_line(t0 + datetime.timedelta(seconds=dt), sm))
        f.write(_line(t0 + datetime.timedelta(seconds=3), 500))               # after the region
    c.t0, c.t1 = t0, t0 + datetime.timedelta(seconds=0.3)
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["reasons"] == []
    assert s["window"] == "timed region"
    # no sample inside the region: every sample is used, and the run says so
    c.t0, c.t1 = t0 + datetime.timedelta(seconds=10), t0 + datetime.timedelta(seconds=11)
    s = c.summary()
    assert s["samples"] == 5 and "hw_slowdown" in s["reasons"] and s["window"].startswith("whole run")


def test_ncu_traffic_dropped_when_the_source_changes(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1710_03013_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"bytes_per_launch": 1.5e6, "sources": ["k.cu"], "source_hash": bench.source_hash(["k.cu"])}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"k@w": entry}))
    assert bench.ncu_traffic("k", "w") == 1.5e6
    assert bench.ncu_traffic("k", "other") is None
    (csrc / "k.cu").write_text("kernel v2\n")
    assert bench.ncu_traffic("k", "w") is None


def test_ncu_traffic_region_hash(tmp_path, monkeypatch):
    """A figure keyed to one kernel's part of a file survives edits elsewhere
    in the file and is dropped when that part changes."""
    csrc = tmp_path / "paper_1710_03013_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "two.cu"
    src.write_text("// A\nkernel a v1\n// B\nkernel b v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    reg = ["// A", "// B"]
    entry = {"bytes_per_launch": 2e6, "sources": ["two.cu"], "region": reg,
             "source_hash": bench.source_hash(["two.cu"], reg)}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"a@w": entry}))
    assert bench.ncu_traffic("a", "w") == 2e6
    src.write_text("// A\nkernel a v1\n// B\nkernel b v2\n")       # the other kernel changed
    assert bench.ncu_traffic("a", "w") == 2e6
    src.write_text("// A\nkernel a v2\n// B\nkernel b v2\n")       # this kernel changed
    assert bench.ncu_traffic("a", "w") is None
    src.write_text("kernel a v1\n")                                  # markers gone
    assert bench.ncu_traffic("a", "w") is None


def test_committed_traffic_entries_name_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        data = json.load(f)
    for key, ent in data.items():
        assert "@" in key and ent["bytes_per_launch"] > 0
        for src in ent["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_1710_03013_gb300", "csrc", src)), (key, src)
        assert np.isfinite(ent["bytes_per_launch"])


def test_batched_slice_is_a_prefix_of_the_workload():
    """--problems N fits the first N problems of the batched workload: the
    same shapes and data as those problems of the full batch."""
    full = dict(bench.WORKLOADS["batched"], n_problems=12)
    cut = dict(full, take=5)
    shapes_f, data_f = bench.batched_data(full)
    shapes_c, data_c = bench.batched_data(cut)
    assert len(shapes_c) == 5 and shapes_c == shapes_f[:5]
    assert all(np.array_equal(a, b) for a, b in zip(data_c, data_f[:5]))
