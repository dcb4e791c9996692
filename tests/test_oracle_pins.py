"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, invariants, brute force on tiny masks (paper Sec. 2 names the
features; the closed forms follow from the geometry of the iso-surface).

Each test is chosen so that a plausible slip in the oracle (a dropped term,
a flipped orientation, a wrong axis or index in a diameter, a wrong face rule)
fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def box_mask(a, b, c, pad=2):
    m = np.zeros((c + 2 * pad, b + 2 * pad, a + 2 * pad), np.uint8)
    m[pad:pad + c, pad:pad + b, pad:pad + a] = 1
    return m


def directed_edges_ok(tri):
    """Closed, consistently oriented: every directed edge once, and its
    reverse once."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    fwd = {tuple(x) for x in e.tolist()}
    if len(fwd) != len(e):
        return False
    return all((b, a) in fwd for (a, b) in fwd)


def sign_change_count(mask):
    p = np.pad(mask != 0, 1)
    n = 0
    for ax in range(3):
        a = np.take(p, range(0, p.shape[ax] - 1), axis=ax)
        b = np.take(p, range(1, p.shape[ax]), axis=ax)
        n += int(np.count_nonzero(a != b))
    return n


def test_single_voxel_golden():
    g = json.load(open(os.path.join(GOLDEN, "single_voxel.json")))
    m = np.zeros(g["mask_shape_zyx"], np.uint8)
    m[tuple(g["inside_voxel_zyx"])] = 1
    f, me = oracle.features(m, g["spacing"])
    assert me.nv == g["n_vertices"] and me.nt == g["n_triangles"]
    for k in ("MeshVolume", "SurfaceArea", "VoxelVolume", "Maximum3DDiameter", "Maximum2DDiameterSlice",
              "Maximum2DDiameterColumn", "Maximum2DDiameterRow"):
        assert f[k] == pytest.approx(g[k], rel=1e-15, abs=1e-15), k
    assert directed_edges_ok(me.tri)


BOXES = [(1, 1, 1), (2, 1, 1), (1, 3, 1), (1, 1, 4), (3, 2, 1), (4, 3, 2), (2, 5, 3), (5, 5, 5), (7, 3, 4)]


@pytest.mark.parametrize("abc", BOXES)
def test_box_closed_forms_isotropic(abc):
    a, b, c = abc
    f, me = oracle.features(box_mask(a, b, c), (1.0, 1.0, 1.0))
    p, q, r = a - 1, b - 1, c - 1
    N = 2 * (a * b + b * c + c * a)
    assert me.nv == N
    assert me.nt == 2 * N - 4
    V = p * q * r + (p * q + q * r + r * p) + (p + q + r) / 2 + 1 / 6
    A = 2 * (p * q + q * r + r * p) + 2 * math.sqrt(2) * (p + q + r) + math.sqrt(3)
    assert f["MeshVolume"] == pytest.approx(V, rel=1e-13)
    assert f["SurfaceArea"] == pytest.approx(A, rel=1e-13)
    assert f["d2"][0] == p * p + q * q + r * r + 2 * max(p, q, r) + 1
    assert f["d2"][1] == p * p + q * q + 2 * max(p, q) + 1          # Slice: equal z
    assert f["d2"][2] == p * p + r * r + 2 * max(p, r) + 1          # Column: equal y
    assert f["d2"][3] == q * q + r * r + 2 * max(q, r) + 1          # Row: equal x
    assert f["VoxelVolume"] == a * b * c
    assert directed_edges_ok(me.tri)


@pytest.mark.parametrize("abc,sp", [((4, 3, 2), (0.7, 0.7, 2.5)), ((2, 5, 3), (0.6, 0.9, 1.2)),
                                    ((6, 2, 3), (1.0, 0.5, 0.25))])
def test_box_closed_forms_anisotropic(abc, sp):
    a, b, c = abc
    sx, sy, sz = sp
    f, me = oracle.features(box_mask(a, b, c), sp)
    p, q, r = a - 1, b - 1, c - 1
    L = (p * sx, q * sy, r * sz)
    ext = ((2 * p + 1) * sx * sx, (2 * q + 1) * sy * sy, (2 * r + 1) * sz * sz)
    V = (p * q * r + (p * q + q * r + r * p) + (p + q + r) / 2 + 1 / 6) * sx * sy * sz
    assert f["MeshVolume"] == pytest.approx(V, rel=1e-13)
    assert f["d2"][0] == pytest.approx(L[0] ** 2 + L[1] ** 2 + L[2] ** 2 + max(ext), rel=1e-14)
    assert f["d2"][1] == pytest.approx(L[0] ** 2 + L[1] ** 2 + max(ext[0], ext[1]), rel=1e-14)
    assert f["d2"][2] == pytest.approx(L[0] ** 2 + L[2] ** 2 + max(ext[0], ext[2]), rel=1e-14)
    assert f["d2"][3] == pytest.approx(L[1] ** 2 + L[2] ** 2 + max(ext[1], ext[2]), rel=1e-14)
    assert f["VoxelVolume"] == pytest.approx(a * b * c * sx * sy * sz, rel=1e-15)


def test_all_2x2x2_masks():
    """Exhaustive: all 256 masks of a 2x2x2 block (every corner configuration
    of the central cube, plus the padding cubes around it)."""
    for case in range(256):
        m = np.zeros((2, 2, 2), np.uint8)
        for c in range(8):
            if (case >> c) & 1:
                m[(c >> 2) & 1, (c >> 1) & 1, c & 1] = 1
        f, me = oracle.features(m, (1.0, 1.0, 1.0))
        assert me.nv == sign_change_count(m), case
        if case == 0:
            assert me.nt == 0 and f["MeshVolume"] == 0.0
            continue
        assert directed_edges_ok(me.tri), case
        assert f["MeshVolume"] > 0, case
        # Euler characteristic of a closed surface: V - E + F, E = 3F/2, is even
        chi = me.nv - me.nt // 2
        assert me.nt % 2 == 0 and chi % 2 == 0, case


def test_random_small_masks():
    rng = np.random.default_rng(1)
    for it in range(1500):
        n = 3 if it % 2 else 4
        m = (rng.random((n, n, n)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        f, me = oracle.features(m, (1.0, 1.0, 1.0))
        assert me.nv == sign_change_count(m)
        assert me.nvox == int(m.sum())
        if me.nt:
            assert directed_edges_ok(me.tri), it
            assert f["MeshVolume"] > 0, it


def test_volume_independent_of_origin():
    """A closed, consistently oriented mesh encloses the same volume from any
    tetrahedron apex: recompute V from the oracle's own triangles with the
    apex at a grid corner and at a far point."""
    rng = np.random.default_rng(2)
    m = (rng.random((9, 8, 7)) < 0.55).astype(np.uint8)
    sp = (0.8, 0.8, 3.0)
    f, me = oracle.features(m, sp)
    P = me.rel_positions()
    for apex in (np.array([0.0, 0.0, 0.0]), np.array([-3.0, 7.5, 11.0]), np.array([100.0, -40.0, 2.0])):
        a, b, c = P[me.tri[:, 0]] - apex, P[me.tri[:, 1]] - apex, P[me.tri[:, 2]] - apex
        V = float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c)))) / 6.0
        assert V == pytest.approx(f["MeshVolume"], rel=1e-12)


def test_translation_invariance():
    rng = np.random.default_rng(3)
    core = (rng.random((6, 7, 8)) < 0.5).astype(np.uint8)
    sp = (0.7, 0.7, 2.5)
    big1 = np.zeros((12, 12, 12), np.uint8)
    big2 = np.zeros((12, 12, 12), np.uint8)
    big1[1:7, 2:9, 0:8] = core
    big2[5:11, 3:10, 4:12] = core
    f1, m1 = oracle.features(big1, sp)
    f2, m2 = oracle.features(big2, sp)
    assert (m1.nv, m1.nt, m1.nvox) == (m2.nv, m2.nt, m2.nvox)
    assert f1["d2"] == f2["d2"]  # bit-exact: differences of half-integers
    for k in ("argmax3d", "argmax_slice", "argmax_column", "argmax_row"):
        assert f1[k] == f2[k]  # canonical order is translation invariant
    assert f1["MeshVolume"] == pytest.approx(f2["MeshVolume"], rel=1e-12)
    assert f1["SurfaceArea"] == pytest.approx(f2["SurfaceArea"], rel=1e-12)


def test_mirror_and_permutation_invariance():
    """Mirrors and axis permutations (spacing permuted with the axes): counts
    exact, squared diameters equal, V and A equal up to rounding (the
    minimum-area triangulation commutes with the symmetries; a fixed fan
    triangulation would not)."""
    rng = np.random.default_rng(4)
    m = (rng.random((5, 6, 7)) < 0.5).astype(np.uint8)
    sp = np.array([0.8, 1.1, 1.7])
    f0, m0 = oracle.features(m, tuple(sp))
    names = {0: 3, 1: 2, 2: 1}  # axis -> index of its planar diameter in d2
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            mm = m
            for ax in range(3):  # array axes are (z, y, x)
                if flips[ax]:
                    mm = np.flip(mm, axis=2 - ax)
            # permute spatial axes: new axis k is old axis perm[k]
            mm = np.ascontiguousarray(np.transpose(mm, [2 - perm[2 - i] for i in range(3)]))
            spp = tuple(sp[list(perm)])
            f1, m1 = oracle.features(mm, spp)
            assert (m1.nv, m1.nt, m1.nvox) == (m0.nv, m0.nt, m0.nvox)
            assert f1["d2"][0] == pytest.approx(f0["d2"][0], rel=1e-15)
            for k in range(3):
                assert f1["d2"][names[k]] == pytest.approx(f0["d2"][names[perm[k]]], rel=1e-15)
            assert f1["MeshVolume"] == pytest.approx(f0["MeshVolume"], rel=1e-12)
            assert f1["SurfaceArea"] == pytest.approx(f0["SurfaceArea"], rel=1e-12)


def test_ellipsoid_genus_zero():
    from paper_2510_02894_gb300 import synth
    for seed in range(3):
        m, sp = synth.ellipsoid_32(seed)
        f, me = oracle.features(m, sp)
        assert me.nt == 2 * me.nv - 4  # Euler: one genus-0 component
        assert directed_edges_ok(me.tri)
        # the mesh lies within half a voxel of the voxel set: V within the
        # band between the digitised voxel volume and its surface layer
        assert abs(f["MeshVolume"] - f["VoxelVolume"]) < 0.5 * f["SurfaceArea"]


def test_diameter_bruteforce_is_max():
    """Brute-force pins: the reported pair attains the maximum of an explicit
    scan, and no pair with a smaller (i, j) attains it."""
    rng = np.random.default_rng(5)
    m = (rng.random((7, 6, 8)) < 0.5).astype(np.uint8)
    sp = (0.7, 0.9, 2.5)
    f, me = oracle.features(m, sp, method="brute")
    U = me.u * np.array(sp)
    D2 = ((U[:, None, :] - U[None, :, :]) ** 2).sum(-1)
    n = me.nv
    iu = np.triu_indices(n, 1)
    for q, ax in ((0, None), (1, 2), (2, 1), (3, 0)):
        sel = np.ones(len(iu[0]), bool) if ax is None else (me.u[iu[0], ax] == me.u[iu[1], ax])
        vals = D2[iu][sel]
        d2, i, j = f["d2"][q], *[f[k] for k in ("argmax3d", "argmax_slice", "argmax_column", "argmax_row")][q]
        assert d2 == pytest.approx(vals.max(), rel=1e-14)
        assert i < j
        if ax is not None:
            assert me.u[i, ax] == me.u[j, ax]
        # exact pinned value of the reported pair
        assert oracle.pair_d2(me.u, i, j, sp) == d2


def test_fast_diameters_match_bruteforce():
    from paper_2510_02894_gb300 import synth
    for seed in range(2):
        for m, sp in synth.batch_256(seed, n=3):
            mesh = oracle.OracleMesh(m, sp)
            if mesh.nv > 6000:
                continue
            ref = oracle.diameters_bruteforce(mesh.u, sp)
            d3, kept = oracle.diameter3d_pruned(mesh.u, sp)
            assert d3 == ref[0] and kept <= mesh.nv
            for q, ax in ((1, 2), (2, 1), (3, 0)):
                assert oracle.diameter2d(mesh.u, sp, ax) == ref[q]


def test_empty_and_full_masks():
    f, me = oracle.features(np.zeros((4, 5, 6), np.uint8), (1, 1, 1))
    assert me.nv == 0 and me.nt == 0 and f["MeshVolume"] == 0 and f["Maximum3DDiameter"] == 0
    assert f["argmax3d"] == (-1, -1)
    f, me = oracle.features(np.ones((3, 4, 5), np.uint8), (1, 1, 1))
    assert me.nv == 2 * (3 * 4 + 4 * 5 + 5 * 3) and me.nt == 2 * me.nv - 4
