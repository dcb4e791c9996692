"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Counts, vertices, triangle sets and argmax pairs must be bit-exact; the
diameters are bit-exact (FP64 confirmation with the same pinned formula);
MeshVolume and SurfaceArea agree within 1e-9 relative (FP64 sums taken in a
different order)."""
import numpy as np
import pytest

import oracle
from paper_2510_02894_gb300 import synth
from tests.helpers import assert_features, canon_tris

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2510_02894_gb300 import rad


def run_both(mask, sp, method="auto", check_mesh=True):
    dev = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    m = rad.mesh(dev, sp)
    got = rad.shape(m)
    ref, om = oracle.features(mask, sp, method)
    assert_features(got, ref)
    if check_mesh:
        idx2, _, tri = m.to_host()
        assert np.array_equal(idx2.astype(np.int64), om.idx2)
        assert np.array_equal(canon_tris(tri), canon_tris(om.tri))
    return got, ref, m


def test_single_voxel():
    m = np.zeros((3, 3, 3), np.uint8)
    m[1, 1, 1] = 1
    got, ref, _ = run_both(m, (1.0, 1.0, 1.0))
    assert got["n_vertices"] == 6 and got["n_triangles"] == 8
    assert abs(got["MeshVolume"] - 1 / 6) < 1e-15 and got["Maximum3DDiameter"] == 1.0


@pytest.mark.parametrize("abc,sp", [((1, 1, 1), (1, 1, 1)), ((4, 3, 2), (1, 1, 1)), ((5, 5, 5), (0.7, 0.7, 2.5)),
                                    ((7, 3, 4), (0.6, 0.9, 1.2)), ((33, 2, 3), (1, 1, 1))])
def test_boxes(abc, sp):
    a, b, c = abc
    m = np.zeros((c + 4, b + 4, a + 4), np.uint8)
    m[2:2 + c, 2:2 + b, 2:2 + a] = 1
    run_both(m, sp)


def test_all_2x2x2_masks():
    for case in range(256):
        m = np.zeros((2, 2, 2), np.uint8)
        for c in range(8):
            if (case >> c) & 1:
                m[(c >> 2) & 1, (c >> 1) & 1, c & 1] = 1
        run_both(m, (0.8, 0.8, 3.0))


def test_random_small_masks():
    rng = np.random.default_rng(11)
    for it in range(150):
        shape = tuple(int(v) for v in rng.integers(1, 8, size=3))
        m = (rng.random(shape) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        m[m > 0] = rng.integers(1, 256, size=int(m.sum()), dtype=np.uint8)  # any non-zero value (1..255) is inside
        sp = tuple(float(v) for v in rng.choice([0.5, 0.6, 0.7, 0.8, 1.0, 1.2, 2.5, 3.0], size=3))
        run_both(m, sp)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ellipsoid_32(seed):
    m, sp = synth.ellipsoid_32(seed)
    run_both(m, sp)


def test_ragged_multi_tile():
    """Spans many tiles, several words per row and a ragged x tail."""
    rng = np.random.default_rng(5)
    m = (synth._noise_blob(rng, (33, 45, 70), 2.5) > 0.5).astype(np.uint8)
    got, ref, _ = run_both(m, (0.7, 0.7, 2.5))
    assert got["n_vertices"] > 2000


def test_wide_rows():
    """nx > 1024: rows longer than one 32-word group pass."""
    rng = np.random.default_rng(6)
    m = (rng.random((4, 3, 1100)) < 0.3).astype(np.uint8)
    run_both(m, (1.0, 1.0, 1.0))


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 1), (1, 1, 7), (6, 1, 1), (2, 3, 17), (3, 2, 16)])
def test_thin_and_degenerate(shape):
    rng = np.random.default_rng(sum(shape))
    m = (rng.random(shape) < 0.6).astype(np.uint8)
    m.reshape(-1)[0] = 1
    run_both(m, (1.0, 1.0, 1.0))


def test_empty_and_full():
    got, ref, _ = run_both(np.zeros((4, 5, 6), np.uint8), (1, 1, 1))
    assert got["n_vertices"] == 0 and got["argmax3d"] == (-1, -1) and got["Maximum3DDiameter"] == 0.0
    run_both(np.ones((3, 4, 5), np.uint8), (1, 1, 1))


def test_plain_fp64_matches():
    for seed in range(2):
        m, sp = synth.ellipsoid_32(seed)
        dev = torch.from_numpy(m).cuda()
        mm = rad.mesh(dev, sp)
        ref, _ = oracle.features(m, sp)
        assert_features(rad.shape_plain_fp64(mm), ref)
    rng = np.random.default_rng(8)
    m = (synth._noise_blob(rng, (20, 30, 40), 2.0) > 0.5).astype(np.uint8)
    mm = rad.mesh(torch.from_numpy(m).cuda(), (0.8, 0.8, 3.0))
    ref, _ = oracle.features(m, (0.8, 0.8, 3.0))
    assert_features(rad.shape_plain_fp64(mm), ref)


def test_extract_paths_agree():
    m, sp = synth.ellipsoid_32(3)
    ref, _ = oracle.features(m, sp)
    ws = rad.Workspace()
    dev = torch.from_numpy(m).cuda()
    for _ in range(3):  # the workspace is reused
        assert_features(rad.extract(dev, sp, ws), ref)
    f = rad.Features()  # the rad_features_t form, filled in place
    assert rad.extract(dev, sp, ws, out=f) is f
    assert_features(f.as_dict(), ref)
    host = torch.from_numpy(m).pin_memory()
    ws2 = rad.Workspace()
    assert_features(rad.extract_host(host.data_ptr(), m.shape, sp, ws2), ref)
    assert_features(rad.extract_host(host.data_ptr(), m.shape, sp, ws2, out=rad.Features()).as_dict(), ref)
    # pageable host memory goes through a device copy
    ws3 = rad.Workspace()
    assert_features(rad.extract_host(m.ctypes.data, m.shape, sp, ws3), ref)
    # pinned memory is read in place at every call, graph replays included:
    # new contents in the same buffer give the new features
    for seed in (4, 5, 3):
        mk, spk = synth.ellipsoid_32(seed)
        refk, _ = oracle.features(mk, spk)
        host.copy_(torch.from_numpy(mk))
        assert_features(rad.extract_host(host.data_ptr(), mk.shape, spk, ws2), refk)
    # a different mask through the same workspace (pools grow as needed)
    rng = np.random.default_rng(9)
    m2 = (synth._noise_blob(rng, (30, 40, 50), 2.0) > 0.5).astype(np.uint8)
    ref2, _ = oracle.features(m2, (0.5, 0.5, 1.0))
    assert_features(rad.extract(torch.from_numpy(m2).cuda(), (0.5, 0.5, 1.0), ws), ref2)
    # pinned masks of odd sizes and row widths, read in place at every call
    for shape in ((16, 9, 7), (17, 33, 40), (64, 20, 90)):
        mk = (synth._noise_blob(rng, shape, 1.5) > 0.5).astype(np.uint8)
        refk, _ = oracle.features(mk, (0.7, 0.9, 1.3))
        hk = torch.from_numpy(mk).pin_memory()
        wsk = rad.Workspace()
        for _ in range(2):
            assert_features(rad.extract_host(hk.data_ptr(), mk.shape, (0.7, 0.9, 1.3), wsk), refk)


@pytest.mark.parametrize("tuning", [dict(tile=64, threads=64, cell_shift=3), dict(tile=256, threads=128, cell_shift=5),
                                    dict(tile=256, threads=64, ctas_per_sm=2, cell_shift=4),
                                    dict(tile=128, threads=64, ctas_per_sm=1, cell_shift=2)])
def test_tuning_variants_same_result(tuning):
    rng = np.random.default_rng(10)
    m = (synth._noise_blob(rng, (40, 36, 44), 3.0) > 0.5).astype(np.uint8)
    old = rad.get_tuning()
    try:
        rad.set_tuning(**tuning)
        run_both(m, (0.6, 0.6, 1.2), check_mesh=False)
    finally:
        rad.set_tuning(**old)


def test_invalid_arguments():
    dev = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(rad.RadError) as e:
        rad.mesh(dev, (1.0, -1.0, 1.0))
    assert e.value.status == 1
    import ctypes
    host = np.zeros((4, 4, 4), np.uint8)
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    sp = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    mt = rad.MeshT()
    st = rad.lib().rad_mesh(ctypes.c_void_p(host.ctypes.data), dims, sp, ctypes.byref(mt), None)
    assert st == 1  # a host pointer is rejected before any launch
    big = (ctypes.c_int64 * 3)(4, 4, 20000)
    st = rad.lib().rad_mesh(ctypes.c_void_p(dev.data_ptr()), big, sp, ctypes.byref(mt), None)
    assert st == 1


def test_graph_replay_follows_new_contents():
    """From the second call the whole pass is a replayed CUDA graph bound to
    the buffer, not to its contents: new contents in the same buffer give the
    new features, and a mask with more vertices than the pools hold makes the
    call fall back, grow the pools and re-capture."""
    rng = np.random.default_rng(13)
    shape = (24, 40, 48)
    masks = [(synth._noise_blob(rng, shape, s) > 0.5).astype(np.uint8) for s in (4.0, 3.0, 1.2)]
    sp = (0.8, 0.8, 3.0)
    buf = torch.zeros(shape, dtype=torch.uint8, device="cuda")
    ws = rad.Workspace()
    for m in masks + masks[:1]:
        buf.copy_(torch.from_numpy(m))
        ref, _ = oracle.features(m, sp)
        for _ in range(3):
            assert_features(rad.extract(buf, sp, ws), ref)


def test_kernel_timing_inside_replayed_graph():
    m, sp = synth.ellipsoid_32(5)
    dev = torch.from_numpy(m).cuda()
    ws = rad.Workspace()
    rad.profile_enable(True)
    try:
        rad.extract(dev, sp, ws)
        rad.extract(dev, sp, ws)  # captured with event nodes
        rad.profile_reset()
        n0 = rad.launch_count()
        for _ in range(3):
            rad.extract(dev, sp, ws)
        prof = rad.profile_read()
        per_call = (rad.launch_count() - n0) / 3
    finally:
        rad.profile_enable(False)
    assert prof["mc_pack_u8"]["launches"] == 3 and prof["mc_pack_u8"]["total_ms"] > 0
    assert prof["diam_pairs_fp32"]["launches"] == 3 and prof["diam_pairs_fp32"]["total_ms"] > 0
    assert per_call == sum(v["launches"] for v in prof.values()) / 3
    torch.zeros(8, device="cuda").sum().item()  # no CUDA error left behind


def test_bounded_wait_reports_timeout_and_context_survives():
    """A device wait on a flag that nothing sets gives up, is reported as
    RAD_ERR_TIMEOUT, and the context keeps working afterwards."""
    import time
    t0 = time.perf_counter()
    assert rad.check_bounded_wait() == 4  # RAD_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    m = synth.ellipsoid_32(3)
    ref, _ = oracle.features(*m)
    assert_features(rad.extract(torch.from_numpy(m[0]).cuda(), m[1], rad.Workspace()), ref)


def test_peak_probe_rates_and_arguments():
    """The measured multiply-add rates (the ALU roofline's denominators) are
    finite and within the range this part can reach: scalar FP32 below the
    152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.6 TFLOP/s the units allow
    (5 % margin), FP64 below FP32.  A bad kind or a NULL output is
    rejected before any launch."""
    import ctypes
    fp32 = rad.peak_probe(rad.PROBE_FP32)
    fp32x2 = rad.peak_probe(rad.PROBE_FP32X2)
    fp64 = rad.peak_probe(rad.PROBE_FP64)
    props = torch.cuda.get_device_properties(0)
    ceiling = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12 * 1.05
    assert 1.0 < fp32 < ceiling, (fp32, ceiling)
    assert 1.0 < fp32x2 < 2.0 * ceiling, (fp32x2, ceiling)  # in case packed issue doubles the lane rate
    assert 0.0 < fp64 < fp32
    out = ctypes.c_double(0.0)
    assert rad.lib().rad_peak_probe(7, ctypes.byref(out), None) == 1  # RAD_ERR_INVALID_ARG
    assert rad.lib().rad_peak_probe(rad.PROBE_FP32, None, None) == 1
    torch.zeros(8, device="cuda").sum().item()  # no CUDA error left behind
