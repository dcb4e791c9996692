"""Pin of the oracle's convex-hull shortlist (oracle.diameter_hull) against the
oracle's brute force over all pairs (paper Sec. 2, "Parallel diameter
calculation": the maximum over every vertex pair).

The hull route decides the parity of the largest masks (512^3), where the
brute force is out of reach.  Its shortlist comes from Qhull, whose merge
tolerances decide which points survive; the half-integer vertex lattice is
full of exactly coplanar, collinear and cospherical points, which is where a
shortlist could drop a tied extreme point and move the tie-broken argmax.
So the result (d2, i, j) must equal the brute force bit for bit, for the 3D
diameter and for every plane family, on meshes chosen for those degeneracies:
boxes and cubes (large tied sets), one-voxel slabs and lines (flat and
collinear plane sets, which take the QhullError fallback), single voxels,
hollow boxes, spheres, rotated ellipsoids and the batch crops at all three
spacings.  Meshes stay below ~12k vertices so the brute force is quick.
"""
import numpy as np
import pytest

import oracle
from paper_2510_02894_gb300 import synth

SPACINGS = ((1.0, 1.0, 1.0), (0.7, 0.7, 2.5), (0.8, 0.8, 3.0), (0.5, 0.5, 1.0))
MAX_NV = 12000


def _box(a, b, c, pad=1):
    m = np.zeros((c + 2 * pad, b + 2 * pad, a + 2 * pad), np.uint8)
    m[pad:pad + c, pad:pad + b, pad:pad + a] = 1
    return m


def _hollow(a, b, c):
    m = _box(a, b, c)
    m[2:-2, 2:-2, 2:-2] = 0
    return m


def _two_cubes():
    m = np.zeros((16, 16, 30), np.uint8)
    m[1:6, 1:6, 1:6] = 1
    m[9:14, 9:14, 23:28] = 1
    return m


def _cases():
    out = []
    boxes = [(1, 1, 1), (5, 5, 5), (10, 10, 10), (12, 7, 5), (20, 3, 9), (16, 16, 1), (60, 60, 1), (100, 1, 1),
             (1, 90, 1), (1, 1, 70), (25, 25, 2), (9, 30, 17), (1, 70, 70)]
    for k, abc in enumerate(boxes):
        out.append((f"box{abc[0]}x{abc[1]}x{abc[2]}", _box(*abc), SPACINGS[k % len(SPACINGS)]))
    for k, sp in enumerate(SPACINGS[:3]):
        out.append((f"voxel_sp{k}", _box(1, 1, 1, pad=2), sp))
    out.append(("hollow14", _hollow(14, 14, 14), (1.0, 1.0, 1.0)))
    out.append(("hollow_aniso", _hollow(18, 11, 9), (0.7, 0.7, 2.5)))
    out.append(("two_cubes", _two_cubes(), (1.0, 1.0, 1.0)))
    # cospherical: a sphere on an isotropic grid
    out.append(("sphere", synth.ellipsoid((26, 26, 26), (12.5, 12.5, 12.5), (11.0, 11.0, 11.0)).astype(np.uint8),
                (1.0, 1.0, 1.0)))
    rng = np.random.default_rng(11)
    for k in range(5):
        semi = rng.uniform(4.0, 12.0, size=3)
        shape = tuple(int(2 * s + 6) for s in semi[::-1])
        centre = [(shape[2] - 1) / 2.0, (shape[1] - 1) / 2.0, (shape[0] - 1) / 2.0]
        m = synth.ellipsoid(shape, centre, semi, synth.random_rotation(rng)).astype(np.uint8)
        out.append((f"ellipsoid{k}", m, SPACINGS[k % len(SPACINGS)]))
    # batch crops: the first small ones of each spacing
    per_sp = {sp: 0 for sp in synth.SPACINGS_BATCH}
    for i, (m, sp) in enumerate(synth.batch_256(3, n=60)):
        if per_sp[sp] >= 4 or m.size > 125000:
            continue
        out.append((f"crop{i}", m, sp))
        per_sp[sp] += 1
    return out


CASES = _cases()


def test_case_list_covers_the_degeneracies():
    assert len(CASES) >= 30
    sps = {sp for name, _, sp in CASES if name.startswith("crop")}
    assert sps == set(synth.SPACINGS_BATCH)


@pytest.mark.parametrize("name,mask,sp", CASES, ids=[c[0] for c in CASES])
def test_diameter_hull_matches_bruteforce(name, mask, sp):
    mesh = oracle.OracleMesh(mask, sp)
    if mesh.nv > MAX_NV:
        pytest.skip(f"{mesh.nv} vertices: brute force too slow for the CPU suite")
    ref = oracle.diameters_bruteforce(mesh.u, sp)
    for q, axis in ((0, None), (1, 2), (2, 1), (3, 0)):
        got = oracle.diameter_hull(mesh.u, sp, axis)
        # bit-exact: the same pinned d2, the same tie-broken (i, j)
        assert (got[0], int(got[1]), int(got[2])) == ref[q], (name, q, got, ref[q])


def test_hull_fallback_path_is_taken():
    """The collinear plane sets of a long one-voxel line go through the
    QhullError fallback (more than 64 collinear points in one plane)."""
    mesh = oracle.OracleMesh(_box(100, 1, 1), (1.0, 1.0, 1.0))
    u = mesh.u
    grp = np.flatnonzero(u[:, 2] == 0.5)  # z-edge vertices below the line (voxels at z = 1): collinear along x
    assert grp.size > 64
    P = u[grp][:, [0, 1]]
    cand = oracle._extreme_candidates(P)
    xs = P[cand, 0]
    assert xs.min() == P[:, 0].min() and xs.max() == P[:, 0].max()
