"""Pins of the oracle's soft (probability-map) path: linearly interpolated
iso-0.5 vertices and the analytic FP64 gradient of area, volume and maximum
3D diameter.

A 0/1 map must reproduce the binary mesh bit for bit; one voxel of value v
among zeros gives an octahedron of radius r = 1 - 1/(2v) whose features and
derivatives have closed forms; elsewhere the gradient is checked against FP64
central finite differences of the oracle's own forward pass.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2510_02894_gb300 import synth


def soft_forward(vals, sp):
    f, m = oracle.features(vals, sp)
    return f, m


def test_binary_float_map_equals_mask():
    rng = np.random.default_rng(7)
    for it in range(20):
        m = (rng.random((6, 5, 7)) < 0.5).astype(np.uint8)
        sp = (0.8, 0.8, 3.0)
        fb, mb = oracle.features(m, sp)
        fs, ms = oracle.features(m.astype(np.float32), sp)
        assert np.array_equal(mb.u, ms.u) and np.array_equal(mb.tri, ms.tri)
        assert fb["MeshVolume"] == fs["MeshVolume"] and fb["SurfaceArea"] == fs["SurfaceArea"]
        assert fb["d2"] == fs["d2"]
        for k in ("argmax3d", "argmax_slice", "argmax_column", "argmax_row"):
            assert fb[k] == fs[k]


@pytest.mark.parametrize("v", [0.6, 0.75, 0.93, 1.0])
def test_soft_single_voxel_closed_forms(v):
    vals = np.zeros((3, 3, 3), np.float64)
    vals[1, 1, 1] = v
    f, m = oracle.features(vals, (1.0, 1.0, 1.0))
    r = 1.0 - 1.0 / (2.0 * v)
    assert m.nv == 6 and m.nt == 8
    assert f["MeshVolume"] == pytest.approx(4.0 / 3.0 * r ** 3, rel=1e-14)
    assert f["SurfaceArea"] == pytest.approx(4.0 * math.sqrt(3.0) * r * r, rel=1e-14)
    assert f["Maximum3DDiameter"] == pytest.approx(2.0 * r, rel=1e-15)
    # gradients: dV/dv = 2 r^2 / v^2, dA/dv = 4 sqrt(3) r / v^2, dD/dv = 1 / v^2
    gV = oracle.soft_grad(m, 0.0, 1.0, 0.0)
    gA = oracle.soft_grad(m, 1.0, 0.0, 0.0)
    gD = oracle.soft_grad(m, 0.0, 0.0, 1.0, f["argmax3d"])
    assert gV[1, 1, 1] == pytest.approx(2 * r * r / v ** 2, rel=1e-13)
    assert gA[1, 1, 1] == pytest.approx(4 * math.sqrt(3) * r / v ** 2, rel=1e-13)
    assert gD[1, 1, 1] == pytest.approx(1.0 / v ** 2, rel=1e-13)
    # a zero 6-neighbour moves one radius: dr/dn = (v - 1/2) / v^2;
    # dV/dr_one = (2/3) r^2, dA/dr_one = 4 r / sqrt(3)
    drn = (v - 0.5) / v ** 2
    for (z, y, x) in ((1, 1, 0), (1, 1, 2), (1, 0, 1), (1, 2, 1), (0, 1, 1), (2, 1, 1)):
        assert gV[z, y, x] == pytest.approx(2.0 / 3.0 * r * r * drn, rel=1e-13)
        assert gA[z, y, x] == pytest.approx(4.0 * r / math.sqrt(3.0) * drn, rel=1e-13)
    # diameter: the tie-broken argmax pair lies on one axis; only its two
    # neighbours (and the centre) move it
    i, j = f["argmax3d"]
    ax = int(np.flatnonzero(m.u[i] != m.u[j])[0])
    for (z, y, x) in ((1, 1, 0), (1, 1, 2), (1, 0, 1), (1, 2, 1), (0, 1, 1), (2, 1, 1)):
        off = np.array([x - 1, y - 1, z - 1])
        expect = drn if off[ax] != 0 else 0.0
        assert gD[z, y, x] == pytest.approx(expect, rel=1e-13, abs=1e-15)
    # far voxels carry no gradient
    assert gV[0, 0, 0] == 0.0 and gA[2, 2, 2] == 0.0


def _loss(vals, sp, w):
    f, m = oracle.features(vals, sp)
    return w[0] * f["SurfaceArea"] + w[1] * f["MeshVolume"] + w[2] * f["Maximum3DDiameter"], f, m


@pytest.mark.parametrize("seed", [0, 1])
def test_soft_gradient_finite_differences(seed):
    """Central differences (h = 1e-4) of the FP64 forward on 24 band voxels
    drawn at random, plus zero-gradient checks on far voxels.  Voxels whose
    perturbation changes the mesh topology, the triangulation choice or the
    argmax pair are skipped (the loss is only piecewise smooth)."""
    vals, sp = synth.soft_160(seed, n=36)
    vals = vals.astype(np.float64)
    rng = np.random.default_rng(100 + seed)
    w = (0.7, 0.3, 1.3)
    L0, f0, m0 = _loss(vals, sp, w)
    g = oracle.soft_grad(m0, w[0], w[1], w[2], f0["argmax3d"])
    band = np.argwhere(g != 0.0)
    assert len(band) > 50
    h = 1e-4
    checked = 0
    for idx in rng.permutation(len(band))[:60]:
        z, y, x = band[idx]
        vp = vals.copy(); vp[z, y, x] += h
        vm = vals.copy(); vm[z, y, x] -= h
        Lp, fp, mp = _loss(vp, sp, w)
        Lm, fm, mm = _loss(vm, sp, w)
        if not (np.array_equal(mp.tri, m0.tri) and np.array_equal(mm.tri, m0.tri)):
            continue
        if fp["argmax3d"] != f0["argmax3d"] or fm["argmax3d"] != f0["argmax3d"]:
            continue
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(g[z, y, x], rel=1e-5, abs=1e-7), (z, y, x)
        checked += 1
        if checked == 24:
            break
    assert checked >= 12
    # far from the surface the loss does not move
    far = np.argwhere((np.abs(vals - 0.5) > 0.45))
    for idx in rng.permutation(len(far))[:5]:
        z, y, x = far[idx]
        if g[z, y, x] != 0.0:
            continue
        vp = vals.copy(); vp[z, y, x] += h
        Lp, _, _ = _loss(vp, sp, w)
        assert Lp == L0


def _loss4(vals, sp, w):
    f, m = oracle.features(vals, sp)
    D = ("Maximum3DDiameter", "Maximum2DDiameterSlice", "Maximum2DDiameterColumn", "Maximum2DDiameterRow")
    return w[0] * f["SurfaceArea"] + w[1] * f["MeshVolume"] + sum(w[2 + q] * f[D[q]] for q in range(4)), f, m


ARGS4 = ("argmax3d", "argmax_slice", "argmax_column", "argmax_row")


@pytest.mark.parametrize("seed", [0, 3])
def test_soft_planar_gradient_finite_differences(seed):
    """The planar-diameter terms of the gradient (each argmax pair held
    fixed) against central differences of the oracle's FP64 forward pass, on
    band voxels whose perturbation keeps the mesh and all four argmax pairs."""
    vals, sp = synth.soft_160(seed, n=30)
    vals = vals.astype(np.float64)
    rng = np.random.default_rng(200 + seed)
    w = (0.4, -0.2, 0.0, 1.3, -0.9, 0.7)  # A, V, D3, Slice, Column, Row
    L0, f0, m0 = _loss4(vals, sp, w)
    pairs = [f0[k] for k in ARGS4]
    g = oracle.soft_grad_planes(m0, w[0], w[1], w[2:], pairs)
    # the planar argmax vertices carry a gradient of their own
    gp = oracle.soft_grad_planes(m0, 0.0, 0.0, (0.0, 1.0, 1.0, 1.0), pairs)
    assert np.count_nonzero(gp) >= 4
    band = np.argwhere(gp != 0.0)
    h = 1e-4
    checked = 0
    for idx in rng.permutation(len(band)):
        z, y, x = band[idx]
        vp = vals.copy(); vp[z, y, x] += h
        vm = vals.copy(); vm[z, y, x] -= h
        Lp, fp, mp = _loss4(vp, sp, w)
        Lm, fm, mm = _loss4(vm, sp, w)
        if not (np.array_equal(mp.tri, m0.tri) and np.array_equal(mm.tri, m0.tri)):
            continue
        if any(fp[k] != f0[k] or fm[k] != f0[k] for k in ARGS4):
            continue
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(g[z, y, x], rel=1e-5, abs=1e-7), (z, y, x)
        checked += 1
    assert checked >= 4


def test_soft_grad_planes_reduces_to_3d_term():
    vals, sp = synth.soft_160(1, n=24)
    f, m = oracle.features(vals, sp)
    a = oracle.soft_grad(m, 0.3, 0.6, 1.7, f["argmax3d"])
    b = oracle.soft_grad_planes(m, 0.3, 0.6, (1.7, 0.0, 0.0, 0.0), [f[k] for k in ARGS4])
    assert np.array_equal(a, b)


def _numpy_planar(u, sp, axis):
    """Max pinned d2 over the pairs with exactly equal coordinate on `axis`,
    smallest (i, j) on ties: an explicit numpy scan, independent of the C code."""
    best = (0.0, -1, -1)
    n = u.shape[0]
    s = np.asarray(sp, np.float64)
    for i in range(n - 1):
        j = np.arange(i + 1, n)
        j = j[u[j, axis] == u[i, axis]]
        if j.size == 0:
            continue
        d = (u[i] - u[j]) * s
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        k = int(np.argmax(d2))  # first maximum: the smallest j for this i
        if d2[k] > best[0] or best[1] < 0:
            best = (float(d2[k]), i, int(j[k]))
    return best


@pytest.mark.parametrize("case", ["layered", "soft20"])
def test_soft_planes_by_exact_coordinate(case):
    """Planar diameters of soft meshes: planes are sets of exactly equal FP64
    coordinates, on the grid planes or off them (vertices of edges along the
    axis whose interpolated coordinates coincide)."""
    if case == "layered":
        n = 14
        vals = np.zeros((n, n, n), np.float32)
        z = np.arange(n)
        prof = (0.95 - 0.05 * np.abs(z - n / 2.0)).astype(np.float32)
        vals[:, 2:n - 2, 3:n - 4] = prof[:, None, None]
        vals[n // 2, 4:7, 5:8] = 0.5
        sp = (1.0, 1.0, 1.0)
    else:
        vals, sp = synth.soft_160(9, n=20)
    m = oracle.OracleMesh(vals, sp)
    ref = oracle.diameters_bruteforce(m.u, sp)
    for q, ax in ((1, 2), (2, 1), (3, 0)):
        want = _numpy_planar(m.u, sp, ax)
        assert ref[q] == want, (case, ax, ref[q], want)
        assert oracle.diameter2d(m.u, sp, ax) == want
    if case == "layered":  # off-grid planes of many vertices exist
        zc = m.u[:, 2]
        frac = zc[zc != np.floor(zc)]
        assert np.unique(frac, return_counts=True)[1].max() >= 8
