"""rad_diameters_plain_fp64_noalloc: the entry point for callers that cannot
call cudaMalloc (for example when a framework owns the whole device memory
budget, or when allocation after start-up is forbidden).  It must give the
oracle's diameters and argmax pairs (and so rad_shape_plain_fp64's), call
after call, with no pair at 0 or 1 vertices, while allocating no device
memory: after a first call, device memory in use is unchanged by further
calls.

Kept in a file that pytest collects last, so that a failure here comes after
every other test has run."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2510_02894_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("Maximum3DDiameter", "Maximum2DDiameterSlice", "Maximum2DDiameterColumn", "Maximum2DDiameterRow")
ARGS = ("argmax3d", "argmax_slice", "argmax_column", "argmax_row")


def _entry():
    from paper_2510_02894_gb300 import rad
    fn = rad.lib().rad_diameters_plain_fp64_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return rad, fn


def _call(fn, mesh, spacing):
    d2 = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    pairs = torch.full((8,), -7, dtype=torch.int32, device="cuda")
    sp = (ctypes.c_double * 3)(*spacing)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(ctypes.c_void_p(mesh.m.vtx_idx2), ctypes.c_void_p(mesh.m.vtx_t), mesh.m.n_vertices, sp,
            ctypes.c_void_p(d2.data_ptr()), ctypes.c_void_p(pairs.data_ptr()), stream)
    assert st == 0
    torch.cuda.synchronize()
    return d2.cpu().numpy(), pairs.cpu().numpy().reshape(4, 2)


def _check(ref, d2, pairs):
    for q in range(4):
        assert float(np.sqrt(d2[q])) == ref[KEYS[q]], (KEYS[q], float(np.sqrt(d2[q])), ref[KEYS[q]])
        assert tuple(int(v) for v in pairs[q]) == tuple(ref[ARGS[q]])


def test_noalloc_matches_plain_entry_point_twice():
    rad, fn = _entry()
    rng = np.random.default_rng(21)
    cases = [((synth._noise_blob(rng, (30, 36, 41), 2.5) > 0.5).astype(np.uint8), (0.6, 0.6, 1.2)),
             (synth.ellipsoid_32(4)[0], (1.0, 1.0, 1.0))]
    for mask, sp in cases:
        m = rad.mesh(torch.from_numpy(mask).cuda(), sp)
        ref = rad.shape_plain_fp64(m)
        oref, _ = oracle.features(mask, sp)
        for k in KEYS + ARGS:
            assert (tuple(ref[k]) if k in ARGS else ref[k]) == (tuple(oref[k]) if k in ARGS else oref[k]), k
        for _ in range(2):  # the static scratch keeps the previous call's contents
            d2, pairs = _call(fn, m, sp)
            _check(oref, d2, pairs)


def test_noalloc_no_pair_and_no_allocation():
    rad, fn = _entry()
    mask, sp = synth.ellipsoid_32(5)
    m = rad.mesh(torch.from_numpy(mask).cuda(), sp)
    _call(fn, m, sp)  # first call: the scratch address is looked up
    d2 = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    pairs = torch.full((8,), -7, dtype=torch.int32, device="cuda")
    sp3 = (ctypes.c_double * 3)(*sp)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for nv in (0, 1, m.n_vertices):
        st = fn(ctypes.c_void_p(m.m.vtx_idx2), None, nv, sp3, ctypes.c_void_p(d2.data_ptr()),
                ctypes.c_void_p(pairs.data_ptr()), stream)
        assert st == 0
        torch.cuda.synchronize()
        if nv < 2:  # no pair: 0 and (-1, -1)
            assert d2.cpu().tolist() == [0.0] * 4 and pairs.cpu().tolist() == [-1] * 8
    # nothing allocated on the device by the calls (driver view and torch's allocator)
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_soft_mesh_and_limits():
    rad, fn = _entry()
    prob, sp = synth.soft_160(3, n=40)
    m = rad.soft_mesh(torch.from_numpy(prob).cuda(), sp)
    ref = rad.shape_plain_fp64(m)
    for _ in range(2):
        d2, pairs = _call(fn, m, sp)
        _check(ref, d2, pairs)
    # beyond the static scratch: rejected before any launch
    sp3 = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = fn(ctypes.c_void_p(m.m.vtx_idx2), None, 4096 * 256 + 1, sp3, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1
    assert b"static scratch" in rad.lib().rad_last_error()
