"""Generate the marching-cubes tables used by the CUDA kernels.

The paper (Sec. 2, "Marching cubes fused parallel kernels") uses a
brute-force marching cubes over every cube of the mask but prints no table.
This script derives one from the rule statement alone -- no published table
is copied:

  * corners c = cx + 2 cy + 4 cz; an edge is (corner with the axis bit clear,
    axis); local edge ids follow (cz, cy, cx, axis), the canonical global
    vertex order restricted to one cube;
  * a corner is inside iff its value passes the iso level;
  * on every cube face the crossing points are joined by segments; where the
    two inside corners of a face are diagonal they are separated (each cut
    off on its own);
  * seen from outside the cube, each segment runs with the outside corners
    of its face on its left, so chained loops wind counter-clockwise about
    the outward normal;
  * each loop is closed by its own disk; a loop of k vertices becomes k - 2
    triangles.

For every loop the script lists all admissible triangulations (no diagonal
may join two vertices lying on one cube face), each as its canonical list:
triangles rotated to start at their smallest local edge id, sorted ascending.
Candidates are stored in ascending lexicographic order of that list.  The
choice among them (minimum area, then maximum enclosed volume, then the first
in list order) needs the vertex positions, so the kernels make it: once per
spacing for a binary mask, per cube for a soft map.

Usage: python gen_mc_tables.py OUTPUT.inc
"""
import math
import sys


def corner_pos(c):
    return (c & 1, (c >> 1) & 1, (c >> 2) & 1)


EDGES = [(c, a) for c in range(8) for a in range(3) if not (c >> a) & 1]
EDGE_ID = {e: i for i, e in enumerate(EDGES)}


def edge_id(c1, c2):
    d = c1 ^ c2
    a = d.bit_length() - 1
    lo = c2 if (c1 >> a) & 1 else c1
    return EDGE_ID[(lo, a)]


def edge_mid(e):
    c, a = EDGES[e]
    p = list(corner_pos(c))
    p[a] += 0.5
    return p


def sub(p, q):
    return [p[i] - q[i] for i in range(3)]


def cross(p, q):
    return [p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]]


def dot(p, q):
    return sum(p[i] * q[i] for i in range(3))


def faces():
    """Six faces as (normal, cyclic corner list); cyclic order by angle about
    the face centre."""
    out = []
    for axis in range(3):
        for side in (0, 1):
            cs = [c for c in range(8) if corner_pos(c)[axis] == side]
            u, v = [k for k in range(3) if k != axis]
            cs.sort(key=lambda c: math.atan2(corner_pos(c)[v] - 0.5, corner_pos(c)[u] - 0.5))
            normal = [0, 0, 0]
            normal[axis] = 1 if side else -1
            out.append((normal, cs))
    return out


FACES = faces()


def on_common_face(e1, e2):
    """Both edge midpoints lie in one face plane (coordinate 0 or 1 on an
    axis along which neither edge runs)."""
    p, q = edge_mid(e1), edge_mid(e2)
    for k in range(3):
        if p[k] == q[k] and p[k] in (0, 1):
            return True
    return False


def case_loops(case):
    inside = [(case >> c) & 1 for c in range(8)]
    succ = {}
    for normal, cs in FACES:
        ring = [(cs[i], cs[(i + 1) % 4]) for i in range(4)]
        crossing = [i for i in range(4) if inside[ring[i][0]] != inside[ring[i][1]]]
        pairs = []
        if len(crossing) == 2:
            pairs.append((crossing[0], crossing[1]))
        elif len(crossing) == 4:
            # separated inside corners: cut each one off with the two ring
            # edges that meet at it
            for i in range(4):
                c = ring[i][0]
                if inside[c]:
                    pairs.append(((i + 3) % 4, i))
        elif crossing:
            raise RuntimeError("odd crossing count")
        outside = [c for c in cs if not inside[c]]
        for (i1, i2) in pairs:
            e1, e2 = edge_id(*ring[i1]), edge_id(*ring[i2])
            p1, p2 = edge_mid(e1), edge_mid(e2)
            side = 0.0
            for o in outside:
                side = dot(normal, cross(sub(p2, p1), sub(corner_pos(o), p1)))
                if side != 0:
                    break
            a, b = (e1, e2) if side > 0 else (e2, e1)
            if a in succ:
                raise RuntimeError("edge leaves twice")
            succ[a] = b
    loops = []
    seen = set()
    for e in sorted(succ):
        if e in seen:
            continue
        loop = []
        x = e
        while x not in seen:
            seen.add(x)
            loop.append(x)
            x = succ[x]
        if x != e:
            raise RuntimeError("open chain")
        loops.append(loop)
    return loops


def polygon_triangulations(k):
    """All triangulations of a convex k-gon as lists of position triples
    (i, m, j), i < m < j, which keep the polygon's orientation."""
    memo = {}

    def rec(i, j):
        if j - i < 2:
            return [[]]
        key = (i, j)
        if key not in memo:
            res = []
            for m in range(i + 1, j):
                for left in rec(i, m):
                    for right in rec(m, j):
                        res.append([(i, m, j)] + left + right)
            memo[key] = res
        return memo[key]

    return rec(0, k - 1)


def canonical(loop, tri):
    out = []
    for (i, m, j) in tri:
        t = (loop[i], loop[m], loop[j])
        r = min(range(3), key=lambda s: t[s])
        out.append(t[r:] + t[:r])
    return sorted(out)


def admissible(loop, tri):
    k = len(loop)
    for (i, m, j) in tri:
        for (x, y) in ((i, m), (m, j), (i, j)):
            if (y - x) % k in (1, k - 1):
                continue
            if on_common_face(loop[x], loop[y]):
                return False
    return True


def build():
    cases = []
    for case in range(256):
        loops = case_loops(case)
        entries = []
        for loop in loops:
            cands = [canonical(loop, t) for t in polygon_triangulations(len(loop)) if admissible(loop, t)]
            if not cands:
                raise RuntimeError(f"no admissible triangulation for case {case}")
            uniq = sorted({tuple(c) for c in cands})
            entries.append((loop, [list(c) for c in uniq]))
        cases.append(entries)
    return cases


def emit(path):
    cases = build()
    loop_k, loop_verts, loop_cand_begin = [], [], []
    cand_tri_begin, triples = [], []
    case_loop_begin, case_ntri, case_edges = [], [], []
    max_loop = max_tri = max_cand = 0
    for case, entries in enumerate(cases):
        case_loop_begin.append(len(loop_k))
        nt = 0
        emask = 0
        for loop, cands in entries:
            k = len(loop)
            max_loop = max(max_loop, k)
            max_cand = max(max_cand, len(cands))
            nt += k - 2
            for e in loop:
                emask |= 1 << e
            loop_k.append(k)
            loop_verts.append(loop + [255] * (8 - k))
            loop_cand_begin.append(len(cand_tri_begin))
            for c in cands:
                cand_tri_begin.append(len(triples))
                triples.extend(c)
        case_ntri.append(nt)
        case_edges.append(emask)
        max_tri = max(max_tri, nt)
    case_loop_begin.append(len(loop_k))
    loop_cand_begin.append(len(cand_tri_begin))
    cand_tri_begin.append(len(triples))

    def arr(name, ctype, vals, per_line=16):
        body = ",\n  ".join(", ".join(str(v) for v in vals[i:i + per_line]) for i in range(0, len(vals), per_line))
        return f"__device__ const {ctype} {name}[{len(vals)}] = {{\n  {body}\n}};\n"

    with open(path, "w") as f:
        f.write("// Generated by gen_mc_tables.py from the rule statement in its docstring.\n")
        f.write("// Do not edit.\n#pragma once\n")
        f.write(f"#define MC_MAX_LOOP {max_loop}\n#define MC_MAX_TRI {max_tri}\n#define MC_MAX_CAND {max_cand}\n")
        f.write(f"#define MC_NUM_LOOPS {len(loop_k)}\n#define MC_NUM_CANDS {len(cand_tri_begin) - 1}\n")
        f.write(f"#define MC_NUM_TRIPLES {len(triples)}\n")
        f.write(arr("MC_EDGE_CORNER", "unsigned char", [c for c, a in EDGES]))
        f.write(arr("MC_EDGE_AXIS", "unsigned char", [a for c, a in EDGES]))
        f.write(arr("MC_CASE_NTRI", "unsigned char", case_ntri))
        f.write(arr("MC_CASE_EDGES", "unsigned short", case_edges))
        f.write(arr("MC_CASE_LOOP_BEGIN", "unsigned short", case_loop_begin))
        f.write(arr("MC_LOOP_K", "unsigned char", loop_k))
        f.write(arr("MC_LOOP_VERTS", "unsigned char", [v for lv in loop_verts for v in lv]))
        f.write(arr("MC_LOOP_CAND_BEGIN", "unsigned short", loop_cand_begin))
        f.write(arr("MC_CAND_TRI_BEGIN", "unsigned short", cand_tri_begin))
        f.write(arr("MC_CAND_TRIPLES", "unsigned char", [v for t in triples for v in t]))
        # host copy of the per-case triangle counts for capacity bounds
        f.write("static const unsigned char MC_CASE_NTRI_HOST[256] = {\n  " +
                ", ".join(str(v) for v in case_ntri) + "\n};\n")
    return dict(max_loop=max_loop, max_tri=max_tri, max_cand=max_cand, loops=len(loop_k),
                cands=len(cand_tri_begin) - 1, triples=len(triples))


if __name__ == "__main__":
    print(emit(sys.argv[1]))
