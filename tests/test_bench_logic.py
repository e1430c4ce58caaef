"""Host arithmetic of bench.py's roofline line, on CPU with a stand-in workload.

The roofline reports the stage with the largest share of the frame: its algorithmic work per
launch (bytes for the HBM-bound stages; for the composite 10 flop per pixel-Gaussian
evaluation plus 5 per blend) over the measured launch time, against the measured HBM
bandwidth or the FP32 peak derived from the SM count, lanes and clock.  A composite timed
as a replayed graph takes its launch time and its share from the graph-timed frame.
"""
import json
import os
import types

import pytest

import bench
from paper_2507_04147_gb300 import synth


def _workload(n=1000, sh_degree=3, width=1280, height=1280):
    scene = types.SimpleNamespace(n=n, sh_degree=sh_degree)
    cams = [synth.pinhole_camera(width, height), synth.pinhole_camera(width, height)]
    return types.SimpleNamespace(scene=scene, cameras=lambda f: cams)


def _stats(evals_per_frame, staged_per_frame, frames, instances=4000):
    return {"instances": instances, "evaluations": evals_per_frame * frames,
            "records_staged": staged_per_frame * frames}


def test_composite_dominant_reports_alu_fraction():
    w = _workload()
    st = _stats(evals_per_frame=1.0e8, staged_per_frame=2.0e5, frames=10)
    stage_ms = {"preprocess": 0.05, "depth_sort": 0.07, "bin": 0.05, "emit": 0.06,
                "composite": 0.16}
    r = bench.roofline(w, st, stage_ms, n_frames=10, eyes=2, tile=32, blends=3.0e7 * 10)
    assert r["kernel"] == "composite" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["work_per_launch"] == pytest.approx(10.0 * 1.0e8 + 5.0 * 3.0e7)
    assert r["achieved"] == pytest.approx(r["work_per_launch"] / 0.16e-3 / 1e12)
    peaks, _ = bench.measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    assert r["peak"] == pytest.approx(152 * 128 * 2 * mhz * 1e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["share_of_frame"] == pytest.approx(0.16 / 0.39)
    assert r["work"]["blends_per_frame"] == pytest.approx(3.0e7)
    # algorithmic bytes of the composite: 52 B per staged record + 12 B per pixel
    px = 2 * 1280 * 1280
    assert r["composite_hbm"]["bytes_per_launch"] == pytest.approx(2.0e5 * 52 + px * 12)


def test_composite_in_graph_mode_takes_graph_time_and_share():
    w = _workload()
    st = _stats(evals_per_frame=1.0e8, staged_per_frame=2.0e5, frames=10)
    stage_ms = {"preprocess": 0.05, "depth_sort": 0.07, "bin": 0.05, "emit": 0.06,
                "composite": 0.16}
    g = {"precompute": 0.21, "composite": 0.17}
    r = bench.roofline(w, st, stage_ms, n_frames=10, eyes=2, tile=32, blends=0, graph_ms=g)
    assert r["launch_ms"] == 0.17 and r["launch_ms_direct"] == 0.16
    assert r["achieved"] == pytest.approx(1.0e9 / 0.17e-3 / 1e12)
    assert r["share_of_frame"] == pytest.approx(0.17 / 0.38)
    assert "graph" in r["launch"] and "graph" in r["share_basis"]


def test_hbm_stage_dominant_uses_measured_bandwidth():
    w = _workload(n=500000, sh_degree=3)
    st = _stats(evals_per_frame=1.0e6, staged_per_frame=1.0e3, frames=1)
    stage_ms = {"preprocess": 0.5, "depth_sort": 0.07, "bin": 0.05, "emit": 0.06,
                "composite": 0.16}
    r = bench.roofline(w, st, stage_ms, n_frames=1, eyes=2, tile=32)
    assert r["kernel"] == "preprocess" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # parameters once (3 + 3 + 4 + 1 + 48 floats) + per eye 48 + 8 + 4 + 4 bytes
    want = 500000 * 4 * 59 + 2 * 500000 * 64
    assert r["work_per_launch"] == want
    assert r["achieved"] == pytest.approx(want / 0.5e-3 / 1e9)
    peaks, _ = bench.measured_peaks()
    assert r["peak"] == pytest.approx(float(peaks["hbm_gbs"]))


def test_traffic_only_while_sources_are_unchanged(tmp_path, monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        doc = json.load(f)
    comp = next(e for e in doc["entries"] if e["stage"] == "composite")
    wl = comp["workload"]
    if comp["source_hash"] == bench.source_hash(*comp["sources"]):
        assert bench.ncu_traffic("composite", wl) == comp["dram_bytes_per_launch"]
    # another workload's capture is not this workload's traffic
    assert bench.ncu_traffic("composite", wl + " (another workload)") is None
    # a stale hash reads as no measurement
    comp["source_hash"] = "0" * 16
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(doc))
    src = tmp_path / "paper_2507_04147_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in comp["sources"]:
        with open(os.path.join(bench.ROOT, "paper_2507_04147_gb300", "csrc", name), "rb") as f:
            (src / name).write_bytes(f.read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("composite", wl) is None
    assert bench.ncu_traffic("no_such_kernel", wl) is None
