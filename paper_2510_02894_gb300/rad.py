"""Thin Python binding of librad (include/rad.h): argument marshalling only.

Every step of the shape-feature path runs in the library's CUDA kernels; this
module passes device pointers of torch tensors, the current CUDA stream and
plain structs through ctypes.  There is no CPU fallback: if librad.so is
missing the first call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librad.so")

RAD_OK = 0
STATUS = {0: "RAD_OK", 1: "RAD_ERR_INVALID_ARG", 2: "RAD_ERR_CUDA", 3: "RAD_ERR_CAPACITY", 4: "RAD_ERR_TIMEOUT",
          5: "RAD_ERR_OOM", 6: "RAD_ERR_INTERNAL"}


class RadError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


DERIVED = ("Sphericity", "SurfaceVolumeRatio", "Compactness1", "Compactness2", "SphericalDisproportion",
           "MajorAxisLength", "MinorAxisLength", "LeastAxisLength", "Elongation", "Flatness")


class Features(ctypes.Structure):
    _fields_ = [("MeshVolume", ctypes.c_double), ("SurfaceArea", ctypes.c_double), ("VoxelVolume", ctypes.c_double),
                ("Maximum3DDiameter", ctypes.c_double), ("Maximum2DDiameterSlice", ctypes.c_double),
                ("Maximum2DDiameterColumn", ctypes.c_double), ("Maximum2DDiameterRow", ctypes.c_double),
                ("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64), ("n_voxels", ctypes.c_int64),
                ("argmax3d", ctypes.c_int32 * 2), ("argmax_slice", ctypes.c_int32 * 2),
                ("argmax_column", ctypes.c_int32 * 2), ("argmax_row", ctypes.c_int32 * 2),
                ("status", ctypes.c_int32), ("_pad", ctypes.c_int32)] + \
        [(n, ctypes.c_double) for n in DERIVED]

    def as_dict(self):
        d = {k: getattr(self, k) for k in ("MeshVolume", "SurfaceArea", "VoxelVolume", "Maximum3DDiameter",
                                           "Maximum2DDiameterSlice", "Maximum2DDiameterColumn",
                                           "Maximum2DDiameterRow", "n_vertices", "n_triangles", "n_voxels")}
        for k in ("argmax3d", "argmax_slice", "argmax_column", "argmax_row"):
            a = getattr(self, k)
            d[k] = (int(a[0]), int(a[1]))
        d["status"] = int(self.status)
        for k in DERIVED:
            d[k] = getattr(self, k)
        return d


class MeshT(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64), ("n_voxels", ctypes.c_int64),
                ("vtx_idx2", ctypes.c_void_p), ("vtx_t", ctypes.c_void_p), ("tri", ctypes.c_void_p),
                ("mesh_volume", ctypes.c_double), ("surface_area", ctypes.c_double),
                ("dims", ctypes.c_int64 * 3), ("spacing", ctypes.c_double * 3), ("soft", ctypes.c_int32),
                ("_pad", ctypes.c_int32), ("_priv", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("cell_shift", ctypes.c_int32)]


class CallStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("h2d_bytes", "d2h_bytes", "problems", "tiles", "tile_pairs",
                                               "work_items", "items_evaluated", "pairs_evaluated", "candidates",
                                               "coarse_pairs")]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None
EXPORTS = ("rad_mesh", "rad_soft_mesh", "rad_shape", "rad_shape_plain_fp64", "rad_shape_fp64_variant", "rad_extract",
           "rad_extract_host",
           "rad_workspace_free", "rad_mesh_free", "rad_mesh_copy", "rad_set_tuning", "rad_profile_enable",
           "rad_profile_read", "rad_profile_reset", "rad_launch_count", "rad_status_str", "rad_last_error",
           "rad_last_call_stats", "rad_soft_forward", "rad_soft_backward", "rad_batch_create", "rad_batch_run",
           "rad_batch_destroy", "rad_check_bounded_wait", "rad_soft_features", "rad_soft_backward_planes",
           "rad_soft_batch_forward", "rad_soft_batch_backward", "rad_crop_resample", "rad_peak_probe")


def lib():
    """Load librad.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        for name in ("rad_mesh", "rad_soft_mesh"):
            getattr(L, name).argtypes = [P, P, P, ctypes.POINTER(MeshT), P]
            getattr(L, name).restype = I
        for name in ("rad_shape", "rad_shape_plain_fp64"):
            getattr(L, name).argtypes = [ctypes.POINTER(MeshT), ctypes.POINTER(Features), P]
            getattr(L, name).restype = I
        L.rad_shape_fp64_variant.argtypes = [ctypes.POINTER(MeshT), I, ctypes.POINTER(Features), P]
        L.rad_shape_fp64_variant.restype = I
        for name in ("rad_extract", "rad_extract_host"):
            getattr(L, name).argtypes = [P, P, P, ctypes.POINTER(Features), ctypes.POINTER(P), P]
            getattr(L, name).restype = I
        L.rad_workspace_free.argtypes = [P]
        L.rad_workspace_free.restype = None
        L.rad_mesh_free.argtypes = [ctypes.POINTER(MeshT)]
        L.rad_mesh_free.restype = None
        L.rad_mesh_copy.argtypes = [ctypes.POINTER(MeshT), P, P, P, P]
        L.rad_mesh_copy.restype = I
        L.rad_set_tuning.argtypes = [ctypes.POINTER(Tuning), ctypes.POINTER(Tuning)]
        L.rad_set_tuning.restype = I
        L.rad_profile_enable.argtypes = [I]
        L.rad_profile_enable.restype = I
        L.rad_profile_read.argtypes = [ctypes.POINTER(KernelStat), I]
        L.rad_profile_read.restype = I
        L.rad_profile_reset.argtypes = []
        L.rad_profile_reset.restype = None
        L.rad_launch_count.argtypes = []
        L.rad_launch_count.restype = ctypes.c_int64
        L.rad_status_str.argtypes = [I]
        L.rad_status_str.restype = ctypes.c_char_p
        L.rad_last_call_stats.argtypes = [ctypes.POINTER(CallStats)]
        L.rad_last_call_stats.restype = I
        L.rad_soft_forward.argtypes = [P, P, P, P, P, ctypes.POINTER(P), P]
        L.rad_soft_forward.restype = I
        L.rad_soft_backward.argtypes = [P, P, P, P, P, P, ctypes.POINTER(P), P]
        L.rad_soft_backward.restype = I
        L.rad_soft_features.argtypes = [P, P, P, ctypes.POINTER(Features), ctypes.POINTER(P), P]
        L.rad_soft_features.restype = I
        L.rad_soft_backward_planes.argtypes = [P, P, P, P, P, P, ctypes.POINTER(P), P]
        L.rad_soft_backward_planes.restype = I
        L.rad_soft_batch_forward.argtypes = [I, P, P, P, P, ctypes.POINTER(P), P]
        L.rad_soft_batch_forward.restype = I
        L.rad_soft_batch_backward.argtypes = [I, P, P, P, P, P, P, ctypes.POINTER(P), P]
        L.rad_soft_batch_backward.restype = I
        L.rad_crop_resample.argtypes = [P, P, P, I, I, P, P, ctypes.c_int64, P, P, P, ctypes.POINTER(P), P]
        L.rad_crop_resample.restype = I
        L.rad_batch_create.argtypes = [I, P, P, P, ctypes.POINTER(P), P]
        L.rad_batch_create.restype = I
        L.rad_batch_run.argtypes = [P, ctypes.POINTER(Features), P]
        L.rad_batch_run.restype = I
        L.rad_batch_destroy.argtypes = [P]
        L.rad_batch_destroy.restype = None
        L.rad_last_error.argtypes = []
        L.rad_last_error.restype = ctypes.c_char_p
        L.rad_check_bounded_wait.argtypes = [P]
        L.rad_check_bounded_wait.restype = I
        L.rad_peak_probe.argtypes = [I, ctypes.POINTER(ctypes.c_double), P]
        L.rad_peak_probe.restype = I
        _lib = L
    return _lib


def _check(status):
    if status != RAD_OK:
        raise RadError(status, lib().rad_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _geometry(shape_zyx, spacing):
    nz, ny, nx = (int(v) for v in shape_zyx)
    dims = (ctypes.c_int64 * 3)(nx, ny, nz)
    sp = (ctypes.c_double * 3)(*(float(s) for s in spacing))
    return dims, sp


def _device_tensor(t, dtype_name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch.Tensor")
    if str(t.dtype) != dtype_name:
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    if t.dim() != 3 or not t.is_contiguous():
        raise ValueError("expected a contiguous [nz][ny][nx] tensor")
    return t


class Mesh:
    """A device mesh owned by the library (freed with the object)."""

    def __init__(self):
        self.m = MeshT()

    def __del__(self):
        if _lib is not None and self.m._priv:
            _lib.rad_mesh_free(ctypes.byref(self.m))

    @property
    def n_vertices(self):
        return int(self.m.n_vertices)

    @property
    def n_triangles(self):
        return int(self.m.n_triangles)

    def to_host(self, stream=None):
        """(idx2 int16 [N,3], t float64 [N] or None, tri int32 [T,3]) on the host."""
        idx2 = np.zeros((self.n_vertices, 3), np.int16)
        tri = np.zeros((self.n_triangles, 3), np.int32)
        t = np.zeros(self.n_vertices, np.float64) if self.m.soft else None
        _check(lib().rad_mesh_copy(ctypes.byref(self.m), idx2.ctypes.data_as(ctypes.c_void_p),
                                   t.ctypes.data_as(ctypes.c_void_p) if t is not None else None,
                                   tri.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return idx2, t, tri


def mesh(mask, spacing, stream=None, out=None):
    """rad_mesh on a CUDA uint8 tensor [nz][ny][nx]."""
    _device_tensor(mask, "torch.uint8")
    dims, sp = _geometry(mask.shape, spacing)
    m = out if out is not None else Mesh()
    _check(lib().rad_mesh(ctypes.c_void_p(mask.data_ptr()), dims, sp, ctypes.byref(m.m), _stream(stream)))
    return m


def soft_mesh(prob, spacing, stream=None, out=None):
    """rad_soft_mesh on a CUDA float32 tensor [nz][ny][nx]."""
    _device_tensor(prob, "torch.float32")
    dims, sp = _geometry(prob.shape, spacing)
    m = out if out is not None else Mesh()
    _check(lib().rad_soft_mesh(ctypes.c_void_p(prob.data_ptr()), dims, sp, ctypes.byref(m.m), _stream(stream)))
    return m


def shape(m, stream=None):
    f = Features()
    _check(lib().rad_shape(ctypes.byref(m.m), ctypes.byref(f), _stream(stream)))
    return f.as_dict()


def shape_plain_fp64(m, stream=None):
    f = Features()
    _check(lib().rad_shape_plain_fp64(ctypes.byref(m.m), ctypes.byref(f), _stream(stream)))
    return f.as_dict()


# FP64 diameter variants of rad_shape_fp64_variant (rad.h)
FP64_EQUAL_LOAD, FP64_BLOCK_ATOMICS, FP64_SHARED_2D, FP64_THREAD_LOCAL, FP64_PLAIN_1D, FP64_CULLED = 1, 2, 3, 4, 5, 6
FP64_VARIANTS = {"equal_load": FP64_EQUAL_LOAD, "block_atomics": FP64_BLOCK_ATOMICS, "shared_2d": FP64_SHARED_2D,
                 "thread_local": FP64_THREAD_LOCAL, "plain_1d": FP64_PLAIN_1D, "culled_fp64": FP64_CULLED}


def shape_fp64_variant(m, variant, stream=None):
    f = Features()
    _check(lib().rad_shape_fp64_variant(ctypes.byref(m.m), int(variant), ctypes.byref(f), _stream(stream)))
    return f.as_dict()


class Workspace:
    """Library-owned buffers reused by extract()/extract_host() calls."""

    def __init__(self):
        self.h = ctypes.c_void_p(None)

    def __del__(self):
        if _lib is not None and self.h.value:
            _lib.rad_workspace_free(self.h)
            self.h = ctypes.c_void_p(None)


def extract(mask, spacing, ws, stream=None, out=None):
    """Whole path (mesh + all features) for a CUDA uint8 mask.  Returns a
    dict, or, when `out` (a Features) is given, fills it and returns it (the
    rad_features_t the call wrote, no conversion; a later call with the same
    `out` overwrites it)."""
    _device_tensor(mask, "torch.uint8")
    dims, sp = _geometry(mask.shape, spacing)
    f = Features() if out is None else out
    _check(lib().rad_extract(ctypes.c_void_p(mask.data_ptr()), dims, sp, ctypes.byref(f), ctypes.byref(ws.h),
                             _stream(stream)))
    return f.as_dict() if out is None else f


def extract_host(mask_ptr, shape_zyx, spacing, ws, stream=None, out=None):
    """Whole path for a HOST mask given by address and shape [nz, ny, nx].
    Pinned memory is read in place by the device; pageable memory is copied
    inside the call.  `out` as in extract()."""
    dims, sp = _geometry(shape_zyx, spacing)
    f = Features() if out is None else out
    _check(lib().rad_extract_host(ctypes.c_void_p(int(mask_ptr)), dims, sp, ctypes.byref(f), ctypes.byref(ws.h),
                                  _stream(stream)))
    return f.as_dict() if out is None else f


def soft_forward(prob, spacing, ws, stream=None):
    """(SurfaceArea, MeshVolume, Maximum3DDiameter), argmax pair of a CUDA
    float32 probability map."""
    _device_tensor(prob, "torch.float32")
    dims, sp = _geometry(prob.shape, spacing)
    out = (ctypes.c_double * 3)()
    am = (ctypes.c_int32 * 2)()
    _check(lib().rad_soft_forward(ctypes.c_void_p(prob.data_ptr()), dims, sp, out, am, ctypes.byref(ws.h),
                                  _stream(stream)))
    return (out[0], out[1], out[2]), (int(am[0]), int(am[1]))


def soft_backward(prob, spacing, gout, argmax, grad, ws, stream=None):
    """Writes d(gout . (A, V, D3)) / d prob into `grad` (CUDA float64 tensor of
    prob's shape); the mesh is recomputed."""
    _device_tensor(prob, "torch.float32")
    _device_tensor(grad, "torch.float64")
    if tuple(grad.shape) != tuple(prob.shape):
        raise ValueError("grad must have prob's shape")
    dims, sp = _geometry(prob.shape, spacing)
    g = (ctypes.c_double * 3)(*(float(v) for v in gout))
    am = (ctypes.c_int32 * 2)(int(argmax[0]), int(argmax[1]))
    _check(lib().rad_soft_backward(ctypes.c_void_p(prob.data_ptr()), dims, sp, g, am,
                                   ctypes.c_void_p(grad.data_ptr()), ctypes.byref(ws.h), _stream(stream)))


ARGMAX_KEYS = ("argmax3d", "argmax_slice", "argmax_column", "argmax_row")


def soft_features(prob, spacing, ws, stream=None):
    """All features (dict) of a CUDA float32 probability map, planar
    diameters and their argmax pairs included."""
    _device_tensor(prob, "torch.float32")
    dims, sp = _geometry(prob.shape, spacing)
    f = Features()
    _check(lib().rad_soft_features(ctypes.c_void_p(prob.data_ptr()), dims, sp, ctypes.byref(f), ctypes.byref(ws.h),
                                   _stream(stream)))
    return f.as_dict()


def _pairs8(feats_or_pairs):
    if isinstance(feats_or_pairs, dict):
        return [int(v) for k in ARGMAX_KEYS for v in feats_or_pairs[k]]
    return [int(v) for pq in feats_or_pairs for v in pq]


def soft_backward_planes(prob, spacing, gout6, argmax, grad, ws, stream=None):
    """grad (CUDA float64, prob's shape) = d(gout6 . (A, V, D3, DSlice,
    DColumn, DRow)) / d prob; argmax: the features dict of soft_features or
    four (i, j) pairs."""
    _device_tensor(prob, "torch.float32")
    _device_tensor(grad, "torch.float64")
    if tuple(grad.shape) != tuple(prob.shape):
        raise ValueError("grad must have prob's shape")
    dims, sp = _geometry(prob.shape, spacing)
    g = (ctypes.c_double * 6)(*(float(v) for v in gout6))
    am = (ctypes.c_int32 * 8)(*_pairs8(argmax))
    _check(lib().rad_soft_backward_planes(ctypes.c_void_p(prob.data_ptr()), dims, sp, g, am,
                                          ctypes.c_void_p(grad.data_ptr()), ctypes.byref(ws.h), _stream(stream)))


def _batch_geometry(probs, spacings):
    n = len(probs)
    if n < 1 or len(spacings) != n:
        raise ValueError("need one spacing per map and at least one map")
    for p in probs:
        _device_tensor(p, "torch.float32")
    dims = (ctypes.c_int64 * (3 * n))(*[int(d) for p in probs for d in (p.shape[2], p.shape[1], p.shape[0])])
    sp = (ctypes.c_double * (3 * n))(*[float(v) for s in spacings for v in s])
    ptrs = (ctypes.c_void_p * n)(*[p.data_ptr() for p in probs])
    return n, ptrs, dims, sp


def soft_batch_forward(probs, spacings, ws, stream=None):
    """Features (list of dicts) of several soft maps in one set of launches."""
    n, ptrs, dims, sp = _batch_geometry(probs, spacings)
    out = (Features * n)()
    _check(lib().rad_soft_batch_forward(n, ptrs, dims, sp, out, ctypes.byref(ws.h), _stream(stream)))
    return [out[i].as_dict() for i in range(n)]


def soft_batch_backward(probs, spacings, gouts, argmaxes, grads, ws, stream=None):
    """Gradients of several soft maps in one set of launches: gouts[i] the six
    weights and argmaxes[i] the features dict (or four pairs) of map i."""
    n, ptrs, dims, sp = _batch_geometry(probs, spacings)
    if len(grads) != n or len(gouts) != n or len(argmaxes) != n:
        raise ValueError("one gradient, weight set and argmax set per map")
    for p, g in zip(probs, grads):
        _device_tensor(g, "torch.float64")
        if tuple(g.shape) != tuple(p.shape):
            raise ValueError("each grad must have its map's shape")
    g6 = (ctypes.c_double * (6 * n))(*[float(v) for go in gouts for v in go])
    a8 = (ctypes.c_int32 * (8 * n))(*[v for am in argmaxes for v in _pairs8(am)])
    gp = (ctypes.c_void_p * n)(*[g.data_ptr() for g in grads])
    _check(lib().rad_soft_batch_backward(n, ptrs, dims, sp, g6, a8, gp, ctypes.byref(ws.h), _stream(stream)))


STATUS_CAPACITY = 3


def crop_resample(mask, spacing, ws, label=None, pad=0, new_spacing=None, out=None, stream=None):
    """Crop a CUDA uint8 mask to its ROI's bounding box (label None: any
    non-zero value) widened by `pad`, optionally resampled to new_spacing by
    nearest neighbour.  Returns (out tensor [nz'][ny'][nx'] uint8 on the
    mask's device, box_lo (x, y, z), out_spacing); `out` may be a preallocated
    CUDA uint8 tensor with enough elements."""
    import torch
    _device_tensor(mask, "torch.uint8")
    dims, sp = _geometry(mask.shape, spacing)
    nsp = (ctypes.c_double * 3)(*new_spacing) if new_spacing is not None else None
    od = (ctypes.c_int64 * 3)()
    lo = (ctypes.c_int64 * 3)()
    osp = (ctypes.c_double * 3)()
    lab = -1 if label is None else int(label)
    L = lib()
    cap = 0 if out is None else out.numel()
    ptr = None if out is None else ctypes.c_void_p(out.data_ptr())
    st = L.rad_crop_resample(ctypes.c_void_p(mask.data_ptr()), dims, sp, lab, int(pad), nsp, ptr, cap, od, lo, osp,
                             ctypes.byref(ws.h), _stream(stream))
    if st == STATUS_CAPACITY and out is None:
        out = torch.empty(int(od[0]) * int(od[1]) * int(od[2]), dtype=torch.uint8, device=mask.device)
        st = L.rad_crop_resample(ctypes.c_void_p(mask.data_ptr()), dims, sp, lab, int(pad), nsp,
                                 ctypes.c_void_p(out.data_ptr()), out.numel(), od, lo, osp, ctypes.byref(ws.h),
                                 _stream(stream))
    _check(st)
    n = int(od[0]) * int(od[1]) * int(od[2])
    res = (out if out is not None else torch.empty(0, dtype=torch.uint8, device=mask.device))
    res = res.reshape(-1)[:n].reshape(int(od[2]), int(od[1]), int(od[0]))
    return res, (int(lo[0]), int(lo[1]), int(lo[2])), (osp[0], osp[1], osp[2])


class Batch:
    """A batch of CUDA uint8 masks (tensors [nz][ny][nx]) with their spacings,
    processed in one set of launches and replayed as one CUDA graph."""

    def __init__(self, masks, spacings, stream=None):
        if len(masks) != len(spacings) or not masks:
            raise ValueError("need one spacing per mask")
        for m in masks:
            _device_tensor(m, "torch.uint8")
        self.masks = list(masks)  # keep the tensors alive
        n = len(masks)
        ptrs = (ctypes.c_void_p * n)(*[m.data_ptr() for m in masks])
        dims = (ctypes.c_int64 * (3 * n))(*[v for m in masks for v in (m.shape[2], m.shape[1], m.shape[0])])
        sp = (ctypes.c_double * (3 * n))(*[float(v) for s in spacings for v in s])
        self.h = ctypes.c_void_p(None)
        _check(lib().rad_batch_create(n, ptrs, dims, sp, ctypes.byref(self.h), _stream(stream)))
        self.n = n

    def features_buffer(self):
        """A rad_features_t array for run(out=...)."""
        return (Features * self.n)()

    def run(self, stream=None, out=None):
        """Features of every ROI: a list of dicts, or, when `out` (from
        features_buffer()) is given, that array filled by the call (a later
        call with the same array overwrites it)."""
        buf = (Features * self.n)() if out is None else out
        if len(buf) != self.n:
            raise ValueError("out must hold one rad_features_t per ROI")
        _check(lib().rad_batch_run(self.h, buf, _stream(stream)))
        return [f.as_dict() for f in buf] if out is None else buf

    def __del__(self):
        if _lib is not None and getattr(self, "h", None) is not None and self.h.value:
            _lib.rad_batch_destroy(self.h)
            self.h = ctypes.c_void_p(None)


def check_bounded_wait(stream=None):
    """Run the library's bounded device wait on a flag that nothing sets;
    returns the status code (RAD_ERR_TIMEOUT = 4 is the expected outcome)."""
    return int(lib().rad_check_bounded_wait(_stream(stream)))


PROBE_FP32, PROBE_FP32X2, PROBE_FP64 = 0, 1, 2


def peak_probe(kind, stream=None):
    """Measured multiply-add rate of this GPU in TFLOP/s (rad_peak_probe):
    PROBE_FP32 scalar FP32, PROBE_FP32X2 packed f32x2, PROBE_FP64 FP64."""
    out = ctypes.c_double(0.0)
    _check(lib().rad_peak_probe(int(kind), ctypes.byref(out), _stream(stream)))
    return out.value


def set_tuning(tile=None, threads=None, ctas_per_sm=None, cell_shift=None):
    cur = get_tuning()
    t = Tuning(tile or cur["tile"], threads or cur["threads"], ctas_per_sm or cur["ctas_per_sm"],
               cell_shift or cur["cell_shift"])
    _check(lib().rad_set_tuning(ctypes.byref(t), None))


def get_tuning():
    t = Tuning()
    _check(lib().rad_set_tuning(None, ctypes.byref(t)))
    return {"tile": t.tile, "threads": t.threads, "ctas_per_sm": t.ctas_per_sm, "cell_shift": t.cell_shift}


def profile_enable(on=True):
    _check(lib().rad_profile_enable(1 if on else 0))


def profile_reset():
    lib().rad_profile_reset()


def profile_read():
    n = lib().rad_profile_read(None, 0)
    arr = (KernelStat * max(n, 1))()
    n = lib().rad_profile_read(arr, n)
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms)}
            for i in range(n)}


def last_call_stats():
    st = CallStats()
    _check(lib().rad_last_call_stats(ctypes.byref(st)))
    return {n: int(getattr(st, n)) for n, _ in CallStats._fields_}


def launch_count():
    return int(lib().rad_launch_count())
