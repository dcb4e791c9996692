"""CPU checks of the C-ABI library: it loads without a GPU and exports every
function declared in include/rad.h; the generated marching-cubes tables are
well formed.  No compute call is made here."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rad_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_all_declared_symbols():
    from paper_2510_02894_gb300 import rad
    lib_path = rad.LIB_PATH
    if not os.path.exists(lib_path):
        from paper_2510_02894_gb300 import build
        build.build()
    lib = rad.lib()
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(rad.EXPORTS) <= set(names)


def test_status_strings_without_gpu():
    from paper_2510_02894_gb300 import rad
    lib = rad.lib()
    for code, name in rad.STATUS.items():
        assert lib.rad_status_str(code).decode() == name


def test_generated_tables_well_formed(tmp_path):
    out = tmp_path / "t.inc"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "paper_2510_02894_gb300", "csrc", "gen_mc_tables.py"),
                        str(out)], capture_output=True, text=True, check=True)
    info = eval(r.stdout.strip())
    assert info["max_loop"] == 7 and info["max_tri"] <= 5
    sys.path.insert(0, os.path.join(ROOT, "paper_2510_02894_gb300", "csrc"))
    import gen_mc_tables as g
    for case in range(256):
        loops = g.case_loops(case)
        if case in (0, 255):
            assert loops == []
            continue
        edges = sorted(e for l in loops for e in l)
        crossing = sorted(e for e, (c, a) in enumerate(g.EDGES)
                          if ((case >> c) & 1) != ((case >> (c | (1 << a))) & 1))
        assert edges == crossing, case


def _header_layout(tmp_path):
    """Sizes and field offsets of the ABI structs and the enum values, as a C
    compiler lays them out from include/rad.h (host gcc; no CUDA needed)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {
        "rad_features_t": ["MeshVolume", "SurfaceArea", "VoxelVolume", "Maximum3DDiameter", "n_vertices",
                           "argmax3d", "argmax_row", "status", "Sphericity", "Flatness"],
        "rad_mesh_t": ["n_vertices", "n_triangles", "vtx_idx2", "tri"],
        "rad_tuning_t": ["tile", "threads", "ctas_per_sm", "cell_shift"],
        "rad_kernel_stat_t": ["name", "launches", "total_ms"],
        "rad_call_stats_t": ["h2d_bytes", "d2h_bytes", "pairs_evaluated", "coarse_pairs"],
    }
    enums = ["RAD_OK", "RAD_ERR_INVALID_ARG", "RAD_ERR_TIMEOUT", "RAD_FP64_EQUAL_LOAD", "RAD_FP64_BLOCK_ATOMICS",
             "RAD_FP64_SHARED_2D", "RAD_FP64_THREAD_LOCAL", "RAD_FP64_PLAIN_1D", "RAD_FP64_CULLED",
             "RAD_PROBE_FP32", "RAD_PROBE_FP32X2", "RAD_PROBE_FP64"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rad.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    for e in enums:
        lines.append(f'  printf("enum {e} %d\\n", (int){e});')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        a, b, c = line.split()
        layout[(a, b)] = int(c)
    return layout


def test_binding_matches_header_layout(tmp_path):
    """The ctypes mirrors of the ABI structs have the header's sizes and field
    offsets, and the binding's constants the header's enum values."""
    import ctypes
    from paper_2510_02894_gb300 import rad
    lay = _header_layout(tmp_path)
    mirrors = {"rad_features_t": rad.Features, "rad_mesh_t": rad.MeshT, "rad_tuning_t": rad.Tuning,
               "rad_kernel_stat_t": rad.KernelStat, "rad_call_stats_t": rad.CallStats}
    for st, cls in mirrors.items():
        assert ctypes.sizeof(cls) == lay[(st, "size")], st
        for (name, field), off in lay.items():
            if name == st and field != "size":
                assert getattr(cls, field).offset == off, (st, field)
    assert lay[("enum", "RAD_OK")] == 0 and lay[("enum", "RAD_ERR_INVALID_ARG")] == 1
    assert lay[("enum", "RAD_ERR_TIMEOUT")] == 4
    assert [lay[("enum", k)] for k in ("RAD_FP64_EQUAL_LOAD", "RAD_FP64_BLOCK_ATOMICS", "RAD_FP64_SHARED_2D",
                                       "RAD_FP64_THREAD_LOCAL", "RAD_FP64_PLAIN_1D", "RAD_FP64_CULLED")] == [
        rad.FP64_EQUAL_LOAD, rad.FP64_BLOCK_ATOMICS, rad.FP64_SHARED_2D, rad.FP64_THREAD_LOCAL, rad.FP64_PLAIN_1D,
        rad.FP64_CULLED]
    assert [lay[("enum", k)] for k in ("RAD_PROBE_FP32", "RAD_PROBE_FP32X2", "RAD_PROBE_FP64")] == [
        rad.PROBE_FP32, rad.PROBE_FP32X2, rad.PROBE_FP64]
