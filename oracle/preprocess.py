"""FP64 CPU oracle of the preprocessing step the paper leaves open (Sec. 3,
"Discussion of the results": reading, cleaning and re-laying out the data
before the features, named as work that could move to the GPU): crop a mask
to the bounding box of its region of interest and resample it to a new voxel
spacing.  Test infrastructure only, like the rest of oracle/.

The paper fixes neither operation, so this module states the definitions
the GPU path is held to (readings):

  ROI voxels      value == label, or value != 0 when no label is given.
  Bounding box    lo_k = min, hi_k = max of the ROI voxels' index on axis k
                  (x, y, z); widened by `pad` voxels per side and clamped to
                  the grid.  An empty ROI gives an empty output.
  Crop            the box's m_k = hi_k - lo_k + 1 voxels per axis.
  Resample        to spacing s'_k (s_k the input spacing), nearest neighbour
                  with the first output voxel centred on the box's first
                  voxel: n'_k = floor((m_k - 1) * s_k / s'_k) + 1 output
                  voxels, output voxel i taking input voxel
                  lo_k + min(m_k - 1, floor(i * s'_k / s_k + 1/2))
                  (a tie goes to the larger index).  Every value above is an
                  FP64 expression evaluated left to right, each operation
                  rounded to nearest, so both sides take the same integer
                  decisions.
  Output          1 where the sampled input voxel is an ROI voxel, else 0
                  (uint8), with spacing s' (s when not resampling) and the
                  box's lo as the input index of output voxel 0.
"""
import numpy as np


def roi_inside(mask, label=None):
    arr = np.asarray(mask)
    return arr == label if label is not None else arr != 0


def roi_bbox(mask, label=None):
    """((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z)) of the ROI voxels of a
    [nz][ny][nx] mask, from the per-axis projections; None when empty."""
    inside = roi_inside(mask, label)
    zs = np.flatnonzero(inside.any(axis=(1, 2)))
    ys = np.flatnonzero(inside.any(axis=(0, 2)))
    xs = np.flatnonzero(inside.any(axis=(0, 1)))
    if zs.size == 0:
        return None
    return (int(xs[0]), int(ys[0]), int(zs[0])), (int(xs[-1]), int(ys[-1]), int(zs[-1]))


def output_size(m, s, s_new):
    """n' = floor((m - 1) * s / s') + 1, in FP64 left to right."""
    return int(np.floor((float(m - 1) * float(s)) / float(s_new))) + 1


def index_map(m, s, s_new):
    """Input offset (within the box) of every output voxel along one axis."""
    n = output_size(m, s, s_new)
    i = np.arange(n, dtype=np.float64)
    r = np.floor((i * float(s_new)) / float(s) + 0.5).astype(np.int64)
    return np.minimum(r, m - 1)


def crop_resample(mask, spacing, label=None, pad=0, new_spacing=None):
    """(out uint8 [nz'][ny'][nx'], lo (x, y, z), out_spacing) by the
    definitions in the module docstring."""
    arr = np.asarray(mask)
    nz, ny, nx = arr.shape
    sp = tuple(float(v) for v in spacing)
    out_sp = sp if new_spacing is None else tuple(float(v) for v in new_spacing)
    box = roi_bbox(arr, label)
    if box is None:
        return np.zeros((0, 0, 0), np.uint8), (0, 0, 0), out_sp
    n = (nx, ny, nz)
    lo = tuple(max(0, box[0][k] - pad) for k in range(3))
    hi = tuple(min(n[k] - 1, box[1][k] + pad) for k in range(3))
    m = tuple(hi[k] - lo[k] + 1 for k in range(3))
    if new_spacing is None:
        maps = [np.arange(m[k], dtype=np.int64) for k in range(3)]
    else:
        maps = [index_map(m[k], sp[k], out_sp[k]) for k in range(3)]
    inside = roi_inside(arr, label)
    zi = lo[2] + maps[2]
    yi = lo[1] + maps[1]
    xi = lo[0] + maps[0]
    out = inside[zi[:, None, None], yi[None, :, None], xi[None, None, :]].astype(np.uint8)
    return np.ascontiguousarray(out), lo, out_sp
