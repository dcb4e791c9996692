"""Shared helpers of the parity tests (comparison logic only)."""
import numpy as np

FEATS = ("MeshVolume", "SurfaceArea", "VoxelVolume", "Maximum3DDiameter", "Maximum2DDiameterSlice",
         "Maximum2DDiameterColumn", "Maximum2DDiameterRow")
ARGS = ("argmax3d", "argmax_slice", "argmax_column", "argmax_row")
REL_TOL = 1e-9  # volume and area: FP64 sums in a different order


def canon_tris(tri):
    """Rotate each triangle (keeping orientation) to start at its smallest id,
    then sort the rows: a representation independent of emission order."""
    tri = np.asarray(tri, np.int64)
    if len(tri) == 0:
        return tri.reshape(0, 3)
    r = np.argmin(tri, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    rot = np.take_along_axis(tri, idx, axis=1)
    order = np.lexsort((rot[:, 2], rot[:, 1], rot[:, 0]))
    return rot[order]


def assert_features(got, ref, planes=True, rel=REL_TOL):
    assert got["n_vertices"] == ref["n_vertices"], (got["n_vertices"], ref["n_vertices"])
    assert got["n_triangles"] == ref["n_triangles"], (got["n_triangles"], ref["n_triangles"])
    assert got["n_voxels"] == ref["n_voxels"]
    for k in ("MeshVolume", "SurfaceArea"):
        assert abs(got[k] - ref[k]) <= rel * max(abs(ref[k]), 1e-300), (k, got[k], ref[k])
    assert got["VoxelVolume"] == ref["VoxelVolume"]
    names = FEATS[3:] if planes else FEATS[3:4]
    args = ARGS if planes else ARGS[:1]
    for k in names:  # the FP64 confirmation makes the diameters bit-exact
        assert got[k] == ref[k], (k, got[k], ref[k])
    for k in args:
        assert tuple(got[k]) == tuple(ref[k]), (k, got[k], ref[k])
    assert_derived(got, ref, rel)


CLOSED_FORM = ("Sphericity", "SurfaceVolumeRatio", "Compactness1", "Compactness2", "SphericalDisproportion")
AXES = ("MajorAxisLength", "MinorAxisLength", "LeastAxisLength")


def assert_derived(got, ref, rel=REL_TOL):
    """Derived Shape features: closed forms in V and A within rel; principal
    axes from the covariance eigenvalues within rel of the major axis (small
    eigenvalues carry rounding relative to the largest)."""
    if "Sphericity" not in ref or "Sphericity" not in got:
        return
    for k in CLOSED_FORM:
        assert abs(got[k] - ref[k]) <= rel * max(abs(ref[k]), 1e-300), (k, got[k], ref[k])
    major = ref["MajorAxisLength"]
    for k in AXES:
        assert abs(got[k] - ref[k]) <= rel * max(abs(ref[k]), 1e-300) + 1e-6 * major, (k, got[k], ref[k])
    for k in ("Elongation", "Flatness"):
        assert abs(got[k] - ref[k]) <= 1e-6, (k, got[k], ref[k])
