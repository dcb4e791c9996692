"""GPU crop-to-ROI and nearest-neighbour resampling (rad_crop_resample)
against the preprocessing oracle, bit for bit: boxes, padding, labels,
down-, up- and non-integer resampling, rows that allow 16-byte loads and rows
that do not, an empty ROI, the capacity protocol, and the full CT-sized mask.
Cropping keeps a mask's shape features exactly (the mesh only moves)."""
import numpy as np
import pytest

from oracle import preprocess as pp
from paper_2510_02894_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2510_02894_gb300 import rad


def _check(mask, sp, **kw):
    ws = rad.Workspace()
    out, lo, osp = rad.crop_resample(torch.from_numpy(np.ascontiguousarray(mask)).cuda(), sp, ws, **kw)
    ref, rlo, rsp = pp.crop_resample(mask, sp, label=kw.get("label"), pad=kw.get("pad", 0),
                                     new_spacing=kw.get("new_spacing"))
    assert lo == tuple(rlo) and tuple(osp) == tuple(rsp)
    assert tuple(out.shape) == ref.shape
    assert np.array_equal(out.cpu().numpy(), ref)
    return out


CASES = [
    dict(),
    dict(pad=2),
    dict(pad=50),
    dict(label=2),
    dict(new_spacing=(1.0, 1.0, 1.0)),
    dict(new_spacing=(0.35, 0.45, 0.8), pad=1),
    dict(new_spacing=(2.1, 1.3, 5.0), label=1),
]


@pytest.mark.parametrize("kw", CASES, ids=[str(c) for c in CASES])
@pytest.mark.parametrize("shape", [(20, 33, 47), (24, 40, 64)])  # byte rows / 16-byte rows
def test_matches_oracle(kw, shape):
    rng = np.random.default_rng(sum(shape))
    m = np.zeros(shape, np.uint8)
    z0, y0, x0 = (int(v) for v in rng.integers(1, 6, size=3))
    m[z0:shape[0] - 3, y0:shape[1] - 4, x0:shape[2] - 5] = rng.choice(np.array([0, 1, 2], np.uint8),
                                                                        size=(shape[0] - 3 - z0, shape[1] - 4 - y0,
                                                                              shape[2] - 5 - x0), p=[0.6, 0.3, 0.1])
    _check(m, (0.7, 0.9, 2.5), **kw)


def test_single_voxel_and_corners():
    m = np.zeros((9, 10, 17), np.uint8)
    m[8, 0, 16] = 1
    _check(m, (1.0, 1.0, 1.0))
    _check(m, (1.0, 1.0, 1.0), pad=3, new_spacing=(0.5, 0.5, 0.5))
    m[0, 9, 0] = 1
    _check(m, (1.0, 1.0, 1.0), new_spacing=(3.0, 3.0, 3.0))


def test_empty_roi_and_capacity():
    ws = rad.Workspace()
    z = torch.zeros((5, 6, 7), dtype=torch.uint8, device="cuda")
    out, lo, _ = rad.crop_resample(z, (1.0, 1.0, 1.0), ws)
    assert tuple(out.shape) == (0, 0, 0) and lo == (0, 0, 0)
    m = torch.zeros((5, 6, 7), dtype=torch.uint8, device="cuda")
    m[1:3, 2:5, 1:6] = 1
    small = torch.empty(3, dtype=torch.uint8, device="cuda")
    with pytest.raises(rad.RadError):
        rad.crop_resample(m, (1.0, 1.0, 1.0), ws, out=small)
    big = torch.full((64,), 9, dtype=torch.uint8, device="cuda")
    out, lo, _ = rad.crop_resample(m, (1.0, 1.0, 1.0), ws, out=big)
    assert tuple(out.shape) == (2, 3, 5) and out.all() and lo == (1, 2, 1)
    assert (big[30:] == 9).all()  # nothing written past the output


def test_ct_mask_full_size():
    mask, sp = synth.ct_512(0)
    _check(mask, sp, new_spacing=(1.0, 1.0, 1.0))
    _check(mask, sp, pad=4)


def test_crop_keeps_the_shape_features():
    """The mesh of the cropped mask is the original's moved by the box
    corner: counts, volume, area, diameters and argmax pairs are equal."""
    mask, sp = synth.ct_512(0)
    dev = torch.from_numpy(mask).cuda()
    ws = rad.Workspace()
    crop, lo, _ = rad.crop_resample(dev, sp, ws)
    assert crop.numel() < mask.size
    a = rad.extract(dev, sp, rad.Workspace())
    b = rad.extract(crop.contiguous(), sp, rad.Workspace())
    for k in ("n_vertices", "n_triangles", "n_voxels", "MeshVolume", "SurfaceArea", "Maximum3DDiameter",
              "Maximum2DDiameterSlice", "Maximum2DDiameterColumn", "Maximum2DDiameterRow", "argmax3d",
              "argmax_slice", "argmax_column", "argmax_row"):
        assert a[k] == b[k], k
