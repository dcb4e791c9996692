"""FP64 CPU oracle for the shape-feature path (arXiv 2510.02894, Sec. 2).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the bench's CPU-baseline
and reference legs are the only callers.  The product library never imports,
links or runs anything here, and this package imports nothing from it.

The C library (rad_oracle.c) holds all arithmetic; this module only marshals
numpy arrays through ctypes.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        lib.orc_mesh_build.restype = P
        lib.orc_mesh_build.argtypes = [P, ctypes.c_int, I64, I64, I64, P, ctypes.POINTER(ctypes.c_int)]
        lib.orc_mesh_free.argtypes = [P]
        for name in ("orc_mesh_nv", "orc_mesh_nt", "orc_mesh_nvox", "orc_mesh_n_ties"):
            getattr(lib, name).restype = I64
            getattr(lib, name).argtypes = [P]
        for name in ("orc_mesh_volume", "orc_mesh_area"):
            getattr(lib, name).restype = D
            getattr(lib, name).argtypes = [P]
        lib.orc_mesh_max_loop.restype = ctypes.c_int
        lib.orc_mesh_max_loop.argtypes = [P]
        lib.orc_mesh_copy.argtypes = [P, P, P, P, P, P]
        lib.orc_diameters_bruteforce.argtypes = [P, I64, P, P, P, P]
        lib.orc_diameter3d_pruned.argtypes = [P, I64, P, P, P, P, P]
        lib.orc_diameter2d_grouped.argtypes = [P, I64, P, ctypes.c_int, P, P, P]
        lib.orc_soft_grad.argtypes = [P, D, D, D, I64, I64, P]
        lib.orc_soft_grad4.argtypes = [P, D, D, P, P, P]
        lib.orc_subset_max.argtypes = [P, P, I64, P, P, P, P]
        lib.orc_pair_d2.restype = D
        lib.orc_pair_d2.argtypes = [P, I64, I64, P]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleMesh:
    """Mesh of one mask: vertices in canonical (z, y, x, axis) order.

    owner: (N, 3) int32 lower grid point of each crossing edge
    axis:  (N,) int32 edge axis;  t: (N,) float64 crossing parameter
    u:     (N, 3) float64 index-space position (owner + t along axis)
    tri:   (T, 3) int32 vertex ids, outward counter-clockwise
    """

    def __init__(self, data, spacing):
        lib = _load()
        arr = np.ascontiguousarray(data)
        if arr.ndim != 3:
            raise ValueError("mask must be 3-D [nz][ny][nx]")
        if arr.dtype == np.uint8 or arr.dtype == np.bool_:
            arr = arr.astype(np.uint8, copy=False)
            kind = 0
        elif arr.dtype == np.float32:
            kind = 1
        elif arr.dtype == np.float64:
            kind = 2
        else:
            raise TypeError(f"unsupported dtype {arr.dtype}")
        nz, ny, nx = arr.shape
        self.dims = (nx, ny, nz)
        self.spacing = tuple(float(s) for s in spacing)
        sp = np.array(self.spacing, dtype=np.float64)
        st = ctypes.c_int(0)
        h = lib.orc_mesh_build(_ptr(arr), kind, nx, ny, nz, _ptr(sp), ctypes.byref(st))
        if not h:
            raise RuntimeError(f"oracle mesh failed with status {st.value}")
        try:
            self.nv = int(lib.orc_mesh_nv(h))
            self.nt = int(lib.orc_mesh_nt(h))
            self.nvox = int(lib.orc_mesh_nvox(h))
            self.volume = float(lib.orc_mesh_volume(h))
            self.area = float(lib.orc_mesh_area(h))
            self.max_loop = int(lib.orc_mesh_max_loop(h))
            self.n_ties = int(lib.orc_mesh_n_ties(h))
            self.owner = np.zeros((self.nv, 3), np.int32)
            self.axis = np.zeros(self.nv, np.int32)
            self.t = np.zeros(self.nv, np.float64)
            self.u = np.zeros((self.nv, 3), np.float64)
            self.tri = np.zeros((self.nt, 3), np.int32)
            lib.orc_mesh_copy(h, _ptr(self.owner), _ptr(self.axis), _ptr(self.t), _ptr(self.u), _ptr(self.tri))
            self._h = h
            self._arr = arr
        except Exception:
            lib.orc_mesh_free(h)
            raise

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_mesh_free(h)
            self._h = None

    @property
    def idx2(self):
        """Doubled index coordinates (exact integers for a binary mask)."""
        return np.rint(2.0 * self.u).astype(np.int64)

    def rel_positions(self):
        """O-relative physical positions, O = centre of the padded box."""
        base = self.owner.astype(np.float64) - (np.array(self.dims, np.float64) - 1.0) * 0.5
        tt = np.zeros((self.nv, 3))
        tt[np.arange(self.nv), self.axis] = self.t
        return (base + tt) * np.array(self.spacing)


def pair_d2(u, i, j, spacing):
    u = np.ascontiguousarray(u, dtype=np.float64)
    sp = np.array(spacing, dtype=np.float64)
    return float(_load().orc_pair_d2(_ptr(u), int(i), int(j), _ptr(sp)))


def diameters_bruteforce(u, spacing):
    """All pairs: returns [(d2, i, j)] for 3D, Slice, Column, Row."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    sp = np.array(spacing, dtype=np.float64)
    d2 = np.zeros(4)
    ii = np.zeros(4, np.int64)
    jj = np.zeros(4, np.int64)
    lib.orc_diameters_bruteforce(_ptr(u), u.shape[0], _ptr(sp), _ptr(d2), _ptr(ii), _ptr(jj))
    return [(float(d2[q]), int(ii[q]), int(jj[q])) for q in range(4)]


def diameter3d_pruned(u, spacing):
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    sp = np.array(spacing, dtype=np.float64)
    d2 = ctypes.c_double(0)
    i = ctypes.c_int64(0)
    j = ctypes.c_int64(0)
    kept = ctypes.c_int64(0)
    lib.orc_diameter3d_pruned(_ptr(u), u.shape[0], _ptr(sp), ctypes.byref(d2), ctypes.byref(i),
                              ctypes.byref(j), ctypes.byref(kept))
    return (d2.value, i.value, j.value), kept.value


def diameter2d(u, spacing, axis):
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    sp = np.array(spacing, dtype=np.float64)
    d2 = ctypes.c_double(0)
    i = ctypes.c_int64(0)
    j = ctypes.c_int64(0)
    lib.orc_diameter2d_grouped(_ptr(u), u.shape[0], _ptr(sp), int(axis), ctypes.byref(d2), ctypes.byref(i),
                               ctypes.byref(j))
    return (d2.value, i.value, j.value)


def subset_max(u, ids, spacing):
    """Pinned brute force over the pairs of a vertex subset."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    ids = np.ascontiguousarray(np.unique(np.asarray(ids, np.int64)))
    sp = np.array(spacing, dtype=np.float64)
    d2 = ctypes.c_double(0)
    i = ctypes.c_int64(0)
    j = ctypes.c_int64(0)
    lib.orc_subset_max(_ptr(u), _ptr(ids), ids.size, _ptr(sp), ctypes.byref(d2), ctypes.byref(i), ctypes.byref(j))
    return (d2.value, i.value, j.value)


def _extreme_candidates(P):
    """Indices of points that include every extreme point of their convex
    hull: Qhull's vertices plus the points it reports as coplanar ('Qc'),
    or, for sets of lower dimension, the per-coordinate extremes together
    with a hull of the remaining coordinates."""
    from scipy.spatial import ConvexHull
    from scipy.spatial import QhullError
    n, dim = P.shape
    if n <= 64:
        return np.arange(n)
    try:
        h = ConvexHull(P, qhull_options="Qc")
        cand = [h.vertices]
        if h.coplanar.size:
            cand.append(h.coplanar[:, 0])
        return np.unique(np.concatenate(cand))
    except QhullError:
        # flat (or collinear) set: drop a constant coordinate and retry
        spread = P.max(axis=0) - P.min(axis=0)
        keep = np.flatnonzero(spread > 0)
        if keep.size < dim and keep.size >= 2:
            return _extreme_candidates(P[:, keep])
        ext = [np.flatnonzero(P[:, k] == P[:, k].min()) for k in range(dim)]
        ext += [np.flatnonzero(P[:, k] == P[:, k].max()) for k in range(dim)]
        return np.unique(np.concatenate(ext))


def diameter_hull(u, spacing, axis=None):
    """Exact maximum (d2, i, j) for very large vertex sets.

    Every pair attaining the maximum consists of extreme points of the
    convex hull (|p - q|^2 is strictly convex in p, so its maximum over the
    hull is attained only at extreme points).  Qhull only shortlists them
    (vertices plus coplanar points, a superset); the pinned FP64 brute force
    over the shortlist decides.  axis None: 3D; 0/1/2: pairs of equal x/y/z,
    one plane at a time (2D hull of the other two coordinates)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    sp = np.asarray(spacing, np.float64)
    if axis is None:
        cand = _extreme_candidates(u * sp)
        return subset_max(u, cand, spacing)
    other = [k for k in range(3) if k != axis]
    order = np.lexsort((np.arange(len(u)), u[:, axis]))
    keys = u[order, axis]
    cuts = np.flatnonzero(np.diff(keys)) + 1
    best = (0.0, -1, -1)
    for grp in np.split(order, cuts):
        if grp.size < 2:
            continue
        loc = _extreme_candidates(u[grp][:, other] * sp[other])
        d2, i, j = subset_max(u, grp[loc], spacing)
        if i < 0:
            continue
        if best[1] < 0 or d2 > best[0] or (d2 == best[0] and (i, j) < (best[1], best[2])):
            best = (d2, i, j)
    return best


def all_diameters(u, spacing, method="auto"):
    """[(d2, i, j)] for 3D, Slice, Column, Row.

    method "brute": one all-pairs pass; "fast": pruned 3D + grouped planes;
    "hull": convex-hull shortlists + pinned brute force (very large sets);
    "auto" picks by size.  The brute force is pinned by explicit numpy scans
    and closed forms (tests/test_oracle_pins.py); "fast" is compared with it
    bit for bit in test_fast_diameters_match_bruteforce (same file), and
    "hull" in tests/test_oracle_hull.py (3D and every plane family, on boxes,
    slabs, lines, single voxels, hollow boxes, spheres, ellipsoids and batch
    crops)."""
    n = u.shape[0]
    if method == "brute" or (method == "auto" and n <= 20000):
        return diameters_bruteforce(u, spacing)
    if method == "hull" or (method == "auto" and n > 1500000):
        return [diameter_hull(u, spacing), diameter_hull(u, spacing, 2), diameter_hull(u, spacing, 1),
                diameter_hull(u, spacing, 0)]
    d3, _ = diameter3d_pruned(u, spacing)
    return [d3, diameter2d(u, spacing, 2), diameter2d(u, spacing, 1), diameter2d(u, spacing, 0)]


FEATURE_NAMES = ("MeshVolume", "SurfaceArea", "VoxelVolume", "Maximum3DDiameter",
                 "Maximum2DDiameterSlice", "Maximum2DDiameterColumn", "Maximum2DDiameterRow")


def features(data, spacing, method="auto"):
    """All shape features of one mask, with argmax pairs and counts."""
    m = OracleMesh(data, spacing)
    sp = m.spacing
    diam = all_diameters(m.u, sp, method) if m.nv >= 2 else [(0.0, -1, -1)] * 4
    out = {
        "MeshVolume": m.volume,
        "SurfaceArea": m.area,
        "VoxelVolume": m.nvox * sp[0] * sp[1] * sp[2],
        "Maximum3DDiameter": float(np.sqrt(diam[0][0])),
        "Maximum2DDiameterSlice": float(np.sqrt(diam[1][0])),
        "Maximum2DDiameterColumn": float(np.sqrt(diam[2][0])),
        "Maximum2DDiameterRow": float(np.sqrt(diam[3][0])),
        "n_vertices": m.nv,
        "n_triangles": m.nt,
        "n_voxels": m.nvox,
        "argmax3d": diam[0][1:],
        "argmax_slice": diam[1][1:],
        "argmax_column": diam[2][1:],
        "argmax_row": diam[3][1:],
        "d2": [d[0] for d in diam],
    }
    out.update(derived_features(m.volume, m.area, data, sp))
    return out, m


DERIVED_NAMES = ("Sphericity", "SurfaceVolumeRatio", "Compactness1", "Compactness2", "SphericalDisproportion",
                 "MajorAxisLength", "MinorAxisLength", "LeastAxisLength", "Elongation", "Flatness")


def derived_features(volume, area, mask, spacing):
    """The rest of the Shape class (paper Sec. 2 names the Shape class the
    method accelerates), written from the standard definitions in plain FP64:

      Sphericity             = (36 pi V^2)^(1/3) / A
      SurfaceVolumeRatio     = A / V
      Compactness1           = V / (sqrt(pi) A^(3/2))
      Compactness2           = 36 pi V^2 / A^3
      SphericalDisproportion = A / (36 pi V^2)^(1/3)

    with V the mesh volume and A the surface area, and, from the eigenvalues
    l1 >= l2 >= l3 of the covariance (1/N normalisation) of the physical
    coordinates of the N inside voxel centres,

      Major/Minor/LeastAxisLength = 4 sqrt(l1), 4 sqrt(l2), 4 sqrt(l3)
      Elongation = sqrt(l2 / l1),  Flatness = sqrt(l3 / l1).

    Readings: a feature with a zero denominator is 0; eigenvalues below 0
    (rounding) count as 0."""
    V, A = float(volume), float(area)
    out = {}
    k = (36.0 * np.pi * V * V) ** (1.0 / 3.0)
    out["Sphericity"] = k / A if A > 0 else 0.0
    out["SurfaceVolumeRatio"] = A / V if V > 0 else 0.0
    out["Compactness1"] = V / (np.sqrt(np.pi) * A ** 1.5) if A > 0 else 0.0
    out["Compactness2"] = 36.0 * np.pi * V * V / A ** 3 if A > 0 else 0.0
    out["SphericalDisproportion"] = A / k if k > 0 else 0.0
    lam = covariance_eigenvalues(mask, spacing)
    l1, l2, l3 = (max(float(x), 0.0) for x in lam)
    out["MajorAxisLength"] = 4.0 * np.sqrt(l1)
    out["MinorAxisLength"] = 4.0 * np.sqrt(l2)
    out["LeastAxisLength"] = 4.0 * np.sqrt(l3)
    out["Elongation"] = float(np.sqrt(l2 / l1)) if l1 > 0 else 0.0
    out["Flatness"] = float(np.sqrt(l3 / l1)) if l1 > 0 else 0.0
    return out


def covariance_eigenvalues(mask, spacing):
    """Eigenvalues (descending) of sum (p - m)(p - m)^T / N over the inside
    voxel centres p = (x sx, y sy, z sz) of a [nz][ny][nx] mask, m their mean."""
    arr = np.asarray(mask)
    sp = np.asarray(spacing, np.float64)
    slab = 16  # z-slices per step: large masks stay within memory

    def points(z0):
        part = arr[z0:z0 + slab]
        inside = part > 0.5 if arr.dtype.kind == "f" else part != 0
        zyx = np.argwhere(inside)
        zyx[:, 0] += z0
        return zyx[:, ::-1].astype(np.float64) * sp

    n, total = 0, np.zeros(3)
    for z0 in range(0, arr.shape[0], slab):  # first pass: the mean
        P = points(z0)
        n += P.shape[0]
        total += P.sum(axis=0)
    if n == 0:
        return np.zeros(3)
    mean = total / n
    C = np.zeros((3, 3))
    for z0 in range(0, arr.shape[0], slab):  # second pass: sum of (p - m)(p - m)^T
        D = points(z0) - mean
        C += D.T @ D
    return np.sort(np.linalg.eigvalsh(C / n))[::-1]


def soft_grad(mesh, gA, gV, gD, argmax3d=(-1, -1)):
    """Analytic FP64 gradient of gA*A + gV*V + gD*D3 w.r.t. every voxel."""
    lib = _load()
    nx, ny, nz = mesh.dims
    grad = np.zeros((nz, ny, nx), np.float64)
    lib.orc_soft_grad(mesh._h, float(gA), float(gV), float(gD), int(argmax3d[0]), int(argmax3d[1]), _ptr(grad))
    return grad


def soft_grad_planes(mesh, gA, gV, gD4, pairs4):
    """Analytic FP64 gradient of gA*A + gV*V + sum_q gD4[q]*D_q w.r.t. every
    voxel, D_q the 3D, Slice, Column and Row diameters with their argmax
    pairs pairs4[q] (each pair held fixed: the 3D term's formula per pair)."""
    lib = _load()
    nx, ny, nz = mesh.dims
    grad = np.zeros((nz, ny, nx), np.float64)
    g = np.array([float(x) for x in gD4], np.float64)
    pr = np.array([int(v) for pq in pairs4 for v in pq], np.int64)
    lib.orc_soft_grad4(mesh._h, float(gA), float(gV), _ptr(g), _ptr(pr), _ptr(grad))
    return grad


def num_threads():
    return int(_load().orc_num_threads())
