"""CPU check of the marching-cubes tables the CUDA kernels are built with
(paper_2510_02894_gb300/csrc/gen_mc_tables.py), against the brute force of
tests/test_oracle_triangulation.py: for every corner configuration the
generator's loops must be the face rule's loops, wound about the outward
normal, and each loop's candidate list must be exactly the set of its
admissible triangulations (the kernels choose among the candidates per
spacing or per cube, so a missing or extra candidate would change meshes)."""
import os
import sys

from tests import test_oracle_triangulation as bf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_2510_02894_gb300", "csrc"))
import gen_mc_tables as gen  # noqa: E402


def canonical(tris):
    out = []
    for t in tris:
        r = min(range(3), key=lambda s: t[s])
        out.append(tuple(t[r:] + t[:r]))
    return tuple(sorted(out))


def same_cycle(a, b):
    if len(a) != len(b) or set(a) != set(b):
        return False
    k = b.index(a[0])
    return list(a) == list(b[k:]) + list(b[:k])


def test_edge_numbering_agrees():
    assert [(c, a) for c, _, a in bf.EDGES] == gen.EDGES


def test_generated_loops_and_candidates_match_brute_force():
    tables = gen.build()
    n_multi = 0
    for case in range(256):
        inside = [bool((case >> c) & 1) for c in range(8)]
        pos = bf.positions([int(v) for v in inside], (1.0, 1.0, 1.0), soft=False)
        mine = [bf.oriented(lp, pos, inside) for lp in bf.cube_loops(inside)]
        theirs = tables[case]
        assert len(mine) == len(theirs), case
        for loop, cands in theirs:
            match = [lp for lp in mine if set(lp) == set(loop)]
            assert len(match) == 1, (case, loop)
            lp = match[0]
            assert same_cycle(list(loop), lp), (case, loop, lp)  # same winding
            expect = {canonical(tr) for tr in bf.triangulations(lp) if bf.admissible(tr, lp)}
            got = {tuple(tuple(t) for t in c) for c in cands}
            assert got == expect, (case, loop)
            assert [list(map(list, c)) for c in sorted(got)] == [list(map(list, c)) for c in cands]  # ascending
            n_multi += len(cands) > 1
    assert n_multi >= 100  # loops with a real choice among candidates
