"""Host-side bookkeeping of the benchmark, on CPU.

The roofline's `traffic` figure comes from a committed ncu table keyed by the
kernel's source-file hash: it must be reported only while the kernel source
is the one the counters were taken on, and be null otherwise.
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _table(tmp_path, rel_src, digest, read=1000, write=24):
    prof = tmp_path / "profiles"
    prof.mkdir(exist_ok=True)
    (prof / "dram_traffic_ct512.md").write_text(
        "| bench kernel | CUDA kernel | source | sha256[:16] | dram__bytes_read.sum | dram__bytes_write.sum |\n"
        "|---|---|---|---|---|---|\n"
        f"| mc_emit | k_emit | {rel_src} | {digest} | {read} | {write} |\n")


def test_traffic_reported_while_source_unchanged(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k_emit() {}\n")
    _table(tmp_path, "k.cu", hashlib.sha256(src.read_bytes()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("mc_emit") == 1024
    assert bench.load_traffic("diam_pairs_fp32") is None  # no row for it


def test_traffic_null_once_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k_emit() {}\n")
    _table(tmp_path, "k.cu", hashlib.sha256(src.read_bytes()).hexdigest()[:16])
    src.write_text("__global__ void k_emit() { /* changed */ }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("mc_emit") is None


def test_committed_table_rows_name_existing_sources():
    path = os.path.join(ROOT, "profiles", "dram_traffic_ct512.md")
    rows = [line for line in open(path) if line.startswith("| ") and line.count("|") == 7]
    rows = [r for r in rows if not r.startswith("| bench kernel") and not r.startswith("|---")]
    assert rows
    for r in rows:
        cells = [c.strip() for c in r.strip().strip("|").split("|")]
        assert os.path.exists(os.path.join(ROOT, cells[2])), cells[2]
        assert int(cells[4]) > 0 and int(cells[5]) >= 0
