"""Pins of the oracle's derived Shape features (the closed forms in V and A,
and the principal axes of the voxel-coordinate covariance) against facts that
do not come from the oracle: a hand-evaluated single voxel, the covariance of
a solid box of voxel centres (a discrete uniform grid: variance (a^2 - 1)/12
per axis), a two-voxel line, and invariance under translation and axis
permutation."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def box(a, b, c, pad=2):
    m = np.zeros((c + 2 * pad, b + 2 * pad, a + 2 * pad), np.uint8)
    m[pad:pad + c, pad:pad + b, pad:pad + a] = 1
    return m


def test_single_voxel_golden():
    g = json.load(open(os.path.join(GOLDEN, "single_voxel_derived.json")))
    m = np.zeros(g["mask_shape_zyx"], np.uint8)
    m[tuple(g["inside_voxel_zyx"])] = 1
    f, _ = oracle.features(m, g["spacing"])
    for k in oracle.DERIVED_NAMES:
        assert f[k] == pytest.approx(g[k], rel=1e-14, abs=1e-15), k


@pytest.mark.parametrize("abc,sp", [((5, 3, 2), (1.0, 1.0, 1.0)), ((7, 4, 9), (0.7, 0.7, 2.5)),
                                    ((12, 2, 5), (0.8, 0.8, 3.0)), ((1, 6, 3), (0.5, 0.5, 1.0))])
def test_box_principal_axes(abc, sp):
    a, b, c = abc
    f, _ = oracle.features(box(a, b, c), sp)
    lam = sorted([(n * n - 1) / 12.0 * s * s for n, s in zip(abc, sp)], reverse=True)
    assert f["MajorAxisLength"] == pytest.approx(4 * math.sqrt(lam[0]), rel=1e-12)
    assert f["MinorAxisLength"] == pytest.approx(4 * math.sqrt(lam[1]), rel=1e-12, abs=1e-12)
    assert f["LeastAxisLength"] == pytest.approx(4 * math.sqrt(lam[2]), rel=1e-12, abs=1e-6)
    assert f["Elongation"] == pytest.approx(math.sqrt(lam[1] / lam[0]), rel=1e-12, abs=1e-12)
    assert f["Flatness"] == pytest.approx(math.sqrt(lam[2] / lam[0]), rel=1e-12, abs=1e-6)
    # closed forms of the box mesh (pinned in test_oracle_pins.py for V and A)
    V, A = f["MeshVolume"], f["SurfaceArea"]
    assert f["SurfaceVolumeRatio"] == pytest.approx(A / V, rel=1e-15)
    assert f["Sphericity"] * f["SphericalDisproportion"] == pytest.approx(1.0, rel=1e-14)
    assert f["Compactness2"] == pytest.approx(f["Sphericity"] ** 3, rel=1e-13)


def test_two_voxel_line():
    m = np.zeros((3, 3, 4), np.uint8)
    m[1, 1, 1:3] = 1
    f, _ = oracle.features(m, (0.6, 1.0, 1.0))
    assert f["MajorAxisLength"] == pytest.approx(4 * 0.3, rel=1e-14)  # variance (0.6/2)^2
    assert f["MinorAxisLength"] == 0.0 and f["LeastAxisLength"] == 0.0
    assert f["Elongation"] == 0.0 and f["Flatness"] == 0.0


def test_invariance():
    rng = np.random.default_rng(3)
    m = (rng.random((7, 9, 11)) < 0.4).astype(np.uint8)
    sp = (0.7, 0.9, 2.5)
    f, _ = oracle.features(m, sp)
    g, _ = oracle.features(np.pad(m, ((2, 1), (0, 3), (4, 0))), sp)  # translation
    h, _ = oracle.features(np.ascontiguousarray(m.transpose(1, 0, 2)), (sp[0], sp[2], sp[1]))  # swap y and z
    for k in ("MajorAxisLength", "MinorAxisLength", "LeastAxisLength", "Elongation", "Flatness"):
        assert g[k] == pytest.approx(f[k], rel=1e-12), k
        assert h[k] == pytest.approx(f[k], rel=1e-12), k


def test_solid_ellipsoid_moments():
    """A large digitised solid ellipsoid: the covariance eigenvalues approach
    the continuous solid's a_k^2 / 5 (within the digitisation error)."""
    from paper_2510_02894_gb300 import synth
    semi = (30.0, 20.0, 12.0)
    m = synth.ellipsoid((30, 46, 66), (32.5, 22.5, 14.5), semi).astype(np.uint8)
    f, _ = oracle.features(m, (1.0, 1.0, 1.0))
    for name, a in zip(("MajorAxisLength", "MinorAxisLength", "LeastAxisLength"), semi):
        assert f[name] == pytest.approx(4 * a / math.sqrt(5.0), rel=0.02), name
