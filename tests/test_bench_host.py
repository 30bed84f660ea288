"""Host-side logic of bench.py and the tuner that needs no GPU: the
profile figures apply only to the kernel source they were taken on, the
reference arm reads the depth the GPU arm runs, and the algorithmic work
of a launch is the sum of its events' costs (CPU only)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1811_03374_gb300 import flops as FL  # noqa: E402
from paper_1811_03374_gb300 import tune as T  # noqa: E402


def test_profile_figures_follow_the_kernel_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    key, files = bench.TRAFFIC[4]
    good = {key: {"source_hash": bench.source_hash(files), "dram_bytes_per_launch": 123,
                  "warp_inst_per_launch": 456}}
    (prof / "traffic.json").write_text(json.dumps(good))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is taken from the package sources, which stay where they are
    monkeypatch.setattr(bench, "source_hash", lambda f: good[key]["source_hash"])
    assert bench.profiled(4) == 123 and bench.profiled(4, "warp_inst_per_launch") == 456
    assert bench.profiled(2) is None  # no figures for the warp variant
    monkeypatch.setattr(bench, "source_hash", lambda f: "another")
    assert bench.profiled(4) is None  # taken on another version of the kernel


def test_reference_depth_is_the_tuned_one(tmp_path, monkeypatch):
    cache = tmp_path / "tune_cache.json"
    cache.write_text(json.dumps({"NVIDIA GB300|seg=10|ray=20|pair=30": {"depth": 17}}))
    monkeypatch.setattr(T, "CACHE", str(cache))
    assert T.cached_depth(10, 20, 30) == 17
    assert T.cached_depth(10, 20, 31) == T.DEFAULT["depth"]


def test_work_per_launch_is_the_sum_of_event_costs():
    c = dict(nodes=100, descents=30, backtracks=5, tests=1000, hits=7)
    root = c["nodes"] - c["descents"] - c["backtracks"]
    assert FL.alg_flops(c, 50) == (FL.PER_RAY * 50 + FL.PER_BOUND * 1000 + FL.PER_ROOT * root
                                   + FL.PER_NODE * 35 + FL.PER_DESCENT * 30 + FL.PER_BACKTRACK * 5 + FL.PER_HIT * 7)
    # the paper's algorithm sets up and root-tests every candidate: never less work
    assert FL.method_flops(c, 50) > FL.alg_flops(c, 50)
    assert FL.fp32_peak_tflops(152, 2070.0) == 152 * 128 * 2 * 2070e6 / 1e12
    # per-unit estimates: every candidate set up and root-tested as a node
    assert FL.estimate_flops(c, 50) == (FL.EST_RAY * 50 + FL.EST_SETUP * 1000 + FL.EST_NODE * (1000 + 35)
                                        + FL.EST_BACKTRACK * 5 + FL.EST_HIT * 7)


def test_clock_sampler_reports_or_stays_silent():
    # NVML where it loads (read-only queries from a thread), nvidia-smi
    # otherwise; without either (a machine with no GPU) the record is None,
    # never an error.  A record names its source and its reasons.
    c = bench.clock_sampler(0)
    rec = c.stop(0.5)
    if rec is not None:
        assert rec["source"] in ("nvml", "nvidia-smi")
        assert rec["samples"] >= 1 and rec["sm_mhz"] > 0 and isinstance(rec["reasons"], list)
        assert abs(rec["kcycles_per_step_at_median"] - 0.5 * rec["sm_mhz"]) < 1e-9
