"""The roofline arithmetic of bench.py on CPU: algorithmic bytes from the device counters
of the timed launches, divided by the launches' event time, against the peak; the
dominant kernel is the one with the most time; traffic is scaled per member from the
recorded capture only while the kernel source is unchanged."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats(ms, launches, cand, members, nodes, tests, pairs, walks):
    return {"search_ms": ms, "search_launches": launches, "candidates": cand, "members": members,
            "nodes_tested": nodes, "pair_tests": tests, "pairs": pairs, "walks": walks}


def test_roofline_picks_the_slower_kernel_and_divides_bytes_by_time():
    dens = _stats(10.0, 2, 1_000_000, 100_000, 50_000, 5_000_000, 800_000, 10_000)
    hyd = _stats(30.0, 1, 2_000_000, 100_000, 40_000, 9_000_000, 1_600_000, 10_000)
    roof, detail = bench.roofline([{"density": dens, "hydro": hyd}], 8000.0, {"sm_mhz": 2000.0})
    assert roof["kernel"] == "k_group (hydro)"
    b = 2_000_000 * bench.B_CAND["hydro"] + 100_000 * bench.B_MEMBER["hydro"] + 40_000 * bench.B_NODE
    assert roof["bytes_per_launch"] == pytest.approx(b)
    assert roof["launch_ms"] == pytest.approx(30.0)
    assert roof["achieved"] == pytest.approx(b / 30e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 8000.0)
    assert roof["alu"]["peak_tflops"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    flops = 10.0 * 9_000_000 + 25.0 * 1_600_000
    assert roof["alu"]["achieved_tflops"] == pytest.approx(flops / 30e-3 / 1e12)
    # per-step detail: density ran two launches of 5 ms each
    assert detail["density"]["launches_per_step"] == 2
    assert detail["density"]["candidates_per_member"] == pytest.approx(10.0)
    assert detail["density"]["members_per_walk"] == pytest.approx(10.0)


def test_density_passes_of_the_last_step_are_reported():
    dens = _stats(10.0, 2, 1_000_000, 100_000, 50_000, 5_000_000, 800_000, 10_000)
    hyd = _stats(3.0, 1, 2_000_000, 100_000, 40_000, 9_000_000, 1_600_000, 10_000)
    first = [{"members": 100, "ms": 4.0}, {"members": 80, "ms": 3.0}]
    last = [{"members": 100, "ms": 6.0}, {"members": 70, "ms": 4.0}]
    recs = [{"density": dens, "hydro": hyd, "density_passes": first},
            {"density": dens, "hydro": hyd, "density_passes": last}]
    _, detail = bench.roofline(recs, 8000.0)
    assert detail["density"]["passes_of_last_step"] == last
    # records without the per-pass list (an optional field) leave it out
    _, detail = bench.roofline([{"density": dens, "hydro": hyd}], 8000.0)
    assert "passes_of_last_step" not in detail["density"]


def test_launch_gbs_counts_candidates_members_and_nodes():
    e = {"candidates": 1000, "members": 10, "nodes": 5, "ms": 1e-3}
    assert bench.launch_gbs(e, 48, 92) == pytest.approx((1000 * 48 + 10 * 92 + 5 * bench.B_NODE) / 1e-6 / 1e9)


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    import hashlib

    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel source")
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"kernel_source": "k.cu", "kernel_source_sha256_16": hashlib.sha256(b"kernel source").hexdigest()[:16],
           "density_dram_bytes_per_member": 75.0}
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("density", 1000) == pytest.approx(75_000.0)
    assert bench.measured_traffic("hydro", 1000) is None
    src.write_bytes(b"kernel source, changed")
    assert bench.measured_traffic("density", 1000) is None



def test_individual_form_takes_its_own_traffic_record(tmp_path, monkeypatch):
    import hashlib

    src = tmp_path / "k.cu"
    src.write_bytes(b"kernels")
    (tmp_path / "profiles").mkdir()
    rec = {"kernel_source": "k.cu", "kernel_source_sha256_16": hashlib.sha256(b"kernels").hexdigest()[:16],
           "hydro_dram_bytes_per_member": 266.0, "indiv_hydro_dram_bytes_per_member": 240.0}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec_step = {"density": _stats(1.0, 1, 10, 10, 1, 10, 1, 1), "hydro": _stats(5.0, 1, 10, 10, 1, 10, 1, 1)}
    g, _ = bench.roofline([rec_step], 8000.0)
    i, _ = bench.roofline([rec_step], 8000.0, form="individual")
    assert g["kernel"] == "k_group (hydro)" and g["traffic"] == pytest.approx(2660.0)
    assert i["kernel"] == "k_indiv (hydro)" and i["traffic"] == pytest.approx(2400.0)
