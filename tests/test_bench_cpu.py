"""Host-side bookkeeping of the benchmark, on CPU.

The roofline's `traffic` figure comes from a committed ncu table
(profiles/dram_traffic.json) keyed by the kernel's source-file hash: it must
be reported only while the kernel source is the one the counters were taken
on, and be null otherwise.  The algorithmic byte counts follow their stated
formulas.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _table(tmp_path, rel_src, digest, read=1000, write=24):
    prof = tmp_path / "profiles"
    prof.mkdir(exist_ok=True)
    (prof / "dram_traffic.json").write_text(json.dumps({"kernels": {"mc_emit": {
        "cuda_kernel": "k_emit", "source": rel_src, "sha256_16": digest, "dram_bytes_read": read,
        "dram_bytes_write": write}}}))


def test_traffic_reported_while_source_unchanged(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k_emit() {}\n")
    _table(tmp_path, "k.cu", hashlib.sha256(src.read_bytes()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("mc_emit") == 1024
    assert bench.load_traffic("diam_pairs_fp32") is None  # no entry for it


def test_traffic_null_once_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k_emit() {}\n")
    _table(tmp_path, "k.cu", hashlib.sha256(src.read_bytes()).hexdigest()[:16])
    src.write_text("__global__ void k_emit() { /* changed */ }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("mc_emit") is None


def test_traffic_null_without_table(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("mc_emit") is None


def test_committed_table_entries_name_existing_sources():
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return
    for name, e in json.load(open(path))["kernels"].items():
        assert os.path.exists(os.path.join(ROOT, e["source"])), (name, e["source"])
        assert int(e["dram_bytes_read"]) > 0 and int(e["dram_bytes_write"]) >= 0


def test_kernel_work_formulas():
    ctx = dict(nvox=1000, bitset_bytes=400, N=10, T=20, rows=30, pairs_evaluated=5)
    assert bench.kernel_work("mc_pack_u8", ctx) == ("hbm", 1400)
    assert bench.kernel_work("mc_count", ctx) == ("hbm", 400 + 16 * 30)
    assert bench.kernel_work("mc_emit", ctx) == ("hbm", 18 * 10 + 12 * 20)
    assert bench.kernel_work("diam_pairs_fp32", ctx) == ("alu", 8 * 5)
    assert bench.kernel_work("assemble", ctx) == (None, None)
    kernels = {k: {"total_ms": 1.0} for k in bench.MESH_KERNELS}
    r = bench.mesh_stage_roofline(kernels, ctx, 1000.0, steps=2)
    assert r["ms"] == 2.0 and r["algorithmic_bytes"] == 1000 + 180 + 240


def test_fp32_filter_entry():
    """25M pairs x 8 flops in 0.01 ms per launch (two launches, 0.02 ms in
    all) is 20 TFLOP/s: a quarter of an 80 TFLOP/s peak."""
    kernels = {"diam_pairs_fp32": {"launches": 2, "total_ms": 0.02}}
    e = bench.fp32_filter_entry(kernels, 25e6, 80.0, 100.0)
    assert abs(e["launch_ms"] - 0.01) < 1e-15
    assert abs(e["achieved_tflops"] - 20.0) < 1e-9
    assert abs(e["frac_of_derived"] - 0.25) < 1e-12 and abs(e["frac_of_measured"] - 0.2) < 1e-12
    assert bench.fp32_filter_entry({}, 25e6, 80.0, 100.0) is None
    assert bench.fp32_filter_entry({"diam_pairs_fp32": {"launches": 0, "total_ms": 0.0}}, 1, 1.0, 1.0) is None

