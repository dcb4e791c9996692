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
