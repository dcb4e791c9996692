"""Pins of the preprocessing oracle (crop to the ROI's bounding box, nearest-
neighbour resampling; oracle/preprocess.py) against what the definitions fix
independently of its code: boxes from np.argwhere, plain slicing for the
crop, strided slicing for integer downsampling, the closed-form index map of
2x upsampling, and a brute-force nearest-centre search on small random
cases."""
import numpy as np
import pytest

from oracle import preprocess as pp


def _random_mask(rng, shape, fill=0.05, labels=(1,)):
    m = np.zeros(shape, np.uint8)
    k = max(1, int(fill * m.size))
    idx = rng.choice(m.size, size=k, replace=False)
    m.flat[idx] = rng.choice(np.array(labels, np.uint8), size=k)
    return m


def _argwhere_box(inside):
    zyx = np.argwhere(inside)
    lo = zyx.min(axis=0)[::-1]
    hi = zyx.max(axis=0)[::-1]
    return tuple(int(v) for v in lo), tuple(int(v) for v in hi)


@pytest.mark.parametrize("seed", range(6))
def test_bbox_and_crop_equal_argwhere_and_slicing(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(3, 30, size=3))
    m = _random_mask(rng, shape, fill=rng.uniform(0.001, 0.05), labels=(1, 2, 7))
    for label in (None, 2):
        inside = (m == label) if label is not None else (m != 0)
        if not inside.any():
            assert pp.roi_bbox(m, label) is None
            continue
        lo, hi = _argwhere_box(inside)
        assert pp.roi_bbox(m, label) == (lo, hi)
        out, olo, osp = pp.crop_resample(m, (0.7, 0.8, 2.0), label=label)
        ref = inside[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1].astype(np.uint8)
        assert olo == lo and osp == (0.7, 0.8, 2.0)
        assert np.array_equal(out, ref)


def test_pad_widens_and_clamps():
    m = np.zeros((10, 12, 14), np.uint8)
    m[1, 5:7, 10:13] = 1
    out, lo, _ = pp.crop_resample(m, (1, 1, 1), pad=3)
    assert lo == (7, 2, 0)
    assert out.shape == (1 + 3 + 1, 2 + 6, 13 - 7 + 1)  # z clamped below at 0, x clamped above at 13
    assert np.array_equal(out, m[0:5, 2:10, 7:14])


def test_empty_roi():
    out, lo, sp = pp.crop_resample(np.zeros((4, 5, 6), np.uint8), (1, 1, 1), new_spacing=(2, 2, 2))
    assert out.shape == (0, 0, 0) and lo == (0, 0, 0) and sp == (2.0, 2.0, 2.0)


@pytest.mark.parametrize("k", [2, 3, 5])
def test_integer_downsampling_is_strided_slicing(k):
    rng = np.random.default_rng(10 + k)
    m = _random_mask(rng, (17, 23, 29), fill=0.2)
    s = (0.6, 0.9, 1.7)
    out, lo, osp = pp.crop_resample(m, s, new_spacing=tuple(k * v for v in s))
    lo_b, hi_b = _argwhere_box(m != 0)
    crop = (m != 0)[lo_b[2]:hi_b[2] + 1, lo_b[1]:hi_b[1] + 1, lo_b[0]:hi_b[0] + 1]
    assert np.array_equal(out, crop[::k, ::k, ::k].astype(np.uint8))


def test_twofold_upsampling_index_map():
    """s' = s / 2: output i samples floor(i / 2 + 1/2) = (i + 1) // 2."""
    for m in (1, 2, 5, 16):
        r = pp.index_map(m, 1.0, 0.5)
        i = np.arange(2 * (m - 1) + 1)
        assert np.array_equal(r, np.minimum((i + 1) // 2, m - 1))


@pytest.mark.parametrize("seed", range(8))
def test_nearest_centre_brute_force(seed):
    """Each output voxel takes the input voxel whose centre is nearest to it
    (positions relative to the box's first voxel centre): brute force over
    all input centres, ties and near-ties (1e-9) skipped."""
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(1, 40))
    s = float(rng.uniform(0.3, 3.0))
    s_new = float(rng.uniform(0.3, 3.0))
    r = pp.index_map(m, s, s_new)
    n = pp.output_size(m, s, s_new)
    assert len(r) == n
    assert (n - 1) * s_new <= (m - 1) * s + 1e-9 and n * s_new > (m - 1) * s - 1e-9
    centres = np.arange(m) * s
    for i in range(n):
        d = np.abs(centres - i * s_new)
        order = np.argsort(d, kind="stable")
        if m > 1 and d[order[1]] - d[order[0]] < 1e-9:
            continue
        assert r[i] == order[0], (i, r[i], order[0])


def test_resampled_box_spans_the_original_centres():
    """A solid box stays solid, and its output voxel centres span the input
    centres' extent to within one output spacing."""
    m = np.zeros((20, 30, 40), np.uint8)
    m[4:16, 5:25, 6:36] = 1
    s = (0.7, 0.7, 2.5)
    out, lo, osp = pp.crop_resample(m, s, new_spacing=(1.0, 1.0, 1.0))
    assert out.all() and lo == (6, 5, 4)
    span_in = [29 * 0.7, 19 * 0.7, 11 * 2.5]
    span_out = [out.shape[2] - 1, out.shape[1] - 1, out.shape[0] - 1]
    for a, b in zip(span_in, span_out):
        assert b <= a + 1e-9 and a < b + 1.0
