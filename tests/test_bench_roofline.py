"""The benchmark's roofline record, computed on CPU from a synthetic profile.

achieved = algorithmic bytes (or flops) per launch / mean launch time; the
dominant class is the one with the most time; CUDA-core classes go against
the FP32 FFMA peak derived from the SM count and clock, streaming classes
against the measured HBM copy rate; `traffic` comes from profiles/traffic.json
only while the kernel sources hash to the recorded value and the workload
matches.
"""
import json

import bench

PEAKS = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}


def prof(name, launches, ms, nbytes, flops):
    return {name: {"launches": launches, "ms": ms, "bytes": nbytes, "flops": flops}}


def test_alu_class_against_the_ffma_peak():
    p = prof("whalf", 10, 4.0, 10 * 88e6, 10 * 4.8e9)
    p.update(prof("il_pass", 10, 1.0, 10 * 66e6, 10 * 1e8))
    r = bench.roofline(p, PEAKS, "measured", "some_workload")
    assert r["kernel"] == "whalf" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    peak = 152 * 128 * 2 * 2000e6 / 1e12
    assert abs(r["peak"] - peak) < 1e-9
    assert abs(r["achieved"] - 4.8e9 / 0.4e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12


def test_streaming_class_against_the_hbm_peak():
    p = prof("il_pass", 100, 2.6, 100 * 66.3e6, 100 * 1e8)
    r = bench.roofline(p, PEAKS, "measured", "some_workload")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6000.0
    assert abs(r["achieved"] - 66.3e6 / 26e-6 / 1e9) < 1e-6
    assert abs(r["algorithmic_bytes_per_launch"] - 66.3e6) < 1e-3


def test_traffic_only_for_matching_sources(tmp_path, monkeypatch):
    p = prof("whalf", 10, 4.0, 10 * 88e6, 10 * 4.8e9)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    # the hash of this tree's kernel sources (none here) is a fixed value
    (tmp_path / "paper_1711_02037_gb300" / "csrc").mkdir(parents=True)
    h = bench.kernel_source_hash()
    rec = {"whalf": {"source_hash": h, "workload": "w1", "dram_bytes_per_launch": 50e6}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.roofline(p, PEAKS, "measured", "w1")["traffic"] == 50e6
    assert bench.roofline(p, PEAKS, "measured", "w2")["traffic"] is None
    rec["whalf"]["source_hash"] = "0" * 16
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.roofline(p, PEAKS, "measured", "w1")["traffic"] is None


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d = tmp_path / "paper_1711_02037_gb300" / "csrc"
    d.mkdir(parents=True)
    f = d / "k.cu"
    f.write_text("// a kernel\n__global__ void k(float *x) { x[0] = 1.f; /* one */ }\n")
    h0 = bench.kernel_source_hash()
    f.write_text("// the same kernel, reworded\n__global__ void k(float *x)\n{\n  x[0] = 1.f;  // one\n}\n")
    assert bench.kernel_source_hash() == h0
    f.write_text("__global__ void k(float *x) { x[0] = 2.f; }\n")
    assert bench.kernel_source_hash() != h0
