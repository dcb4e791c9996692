"""Parity of the FP64 diameter variants (paper Sec. 3, optimisation steps
(1)-(5) of the accumulation-pattern study, and the culled FP64 search) with
the FP64 CPU oracle, through rad_shape_fp64_variant.

Every variant evaluates the pinned FP64 d2 and breaks ties by the smallest
(i, j), so diameters and argmax pairs are bit-exact, like rad_shape.  The
cases cover ties (boxes), a single voxel, empty masks, meshes of several
256-vertex tiles with a ragged tail, planar problems, and a soft-map mesh
(vertices off the half-integer lattice)."""
import numpy as np
import pytest

import oracle
from paper_2510_02894_gb300 import synth
from tests.helpers import ARGS, FEATS, assert_features

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2510_02894_gb300 import rad

VARIANTS = (1, 2, 3, 4, 5, 6)


def _box(a, b, c, pad=2):
    m = np.zeros((c + 2 * pad, b + 2 * pad, a + 2 * pad), np.uint8)
    m[pad:pad + c, pad:pad + b, pad:pad + a] = 1
    return m


def _cases():
    rng = np.random.default_rng(5)
    out = [("voxel", _box(1, 1, 1), (1.0, 1.0, 1.0)),
           ("box7x3x4", _box(7, 3, 4), (0.6, 0.9, 1.2)),
           ("box12x12x12", _box(12, 12, 12), (1.0, 1.0, 1.0)),
           ("slab40x40x1", _box(40, 40, 1), (0.7, 0.7, 2.5))]
    for seed in range(2):
        m, sp = synth.ellipsoid_32(seed)
        out.append((f"ellipsoid32_{seed}", m, sp))
    out.append(("blob20x30x40", (synth._noise_blob(rng, (20, 30, 40), 2.0) > 0.5).astype(np.uint8), (0.8, 0.8, 3.0)))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,mask,sp", CASES, ids=[c[0] for c in CASES])
def test_variants_match_oracle(name, mask, sp):
    ref, _ = oracle.features(mask, sp)
    m = rad.mesh(torch.from_numpy(np.ascontiguousarray(mask)).cuda(), sp)
    assert m.n_vertices > 0
    base = rad.shape(m)
    for v in VARIANTS:
        got = rad.shape_fp64_variant(m, v)
        assert_features(got, ref)
        for k in FEATS[3:] + ARGS:  # identical to the FP32-filter engine
            assert got[k] == base[k], (name, v, k)


def test_variants_empty_mask():
    m = rad.mesh(torch.zeros((4, 5, 6), dtype=torch.uint8, device="cuda"), (1.0, 1.0, 1.0))
    for v in VARIANTS:
        got = rad.shape_fp64_variant(m, v)
        assert got["Maximum3DDiameter"] == 0.0 and tuple(got["argmax3d"]) == (-1, -1)


def test_variants_soft_mesh():
    """Vertices off the half-integer lattice (soft map, t in (0, 1)): the
    all-pairs variants give every category; the culled engine (like
    rad_shape on a soft mesh) the 3D diameter."""
    prob, sp = synth.soft_160(0, n=40)
    ref, _ = oracle.features(prob, sp)
    m = rad.soft_mesh(torch.from_numpy(prob).cuda(), sp)
    assert m.n_vertices == ref["n_vertices"]
    for v in VARIANTS:
        got = rad.shape_fp64_variant(m, v)
        keys = (FEATS[3:] + ARGS) if v <= 5 else (FEATS[3], ARGS[0])
        for k in keys:
            assert (tuple(got[k]) if k in ARGS else got[k]) == (tuple(ref[k]) if k in ARGS else ref[k]), (v, k)


def test_unknown_variant_rejected():
    m = rad.mesh(torch.from_numpy(_box(2, 2, 2)).cuda(), (1.0, 1.0, 1.0))
    for v in (0, 7, -1):
        with pytest.raises(rad.RadError):
            rad.shape_fp64_variant(m, v)
