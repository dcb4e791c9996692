"""Parity at the full workload sizes, in the launch configuration the bench
times: the 512x512x256 CT mask, a batch of crops, one 512^3 blob mask and the
160^3 soft map.  The oracle computes everything it can exactly (its mesh in
full; the diameters with exact shortlists, see oracle.diameter_hull)."""
import numpy as np
import pytest

import oracle
from paper_2510_02894_gb300 import synth
from tests.helpers import assert_features, canon_tris

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2510_02894_gb300 import rad


def check_full(mask, sp, method="auto", tris=True):
    dev = torch.from_numpy(mask).cuda()
    m = rad.mesh(dev, sp)
    got = rad.shape(m)
    ref, om = oracle.features(mask, sp, method)
    assert_features(got, ref)
    idx2, _, tri = m.to_host()
    assert np.array_equal(idx2.astype(np.int64), om.idx2)
    if tris:
        assert np.array_equal(canon_tris(tri), canon_tris(om.tri))
    # the whole-path entry point (no host sync inside) gives the same result
    ws = rad.Workspace()
    for _ in range(2):
        assert_features(rad.extract(dev, sp, ws), ref)
    return got


def test_ct_512x512x256():
    mask, sp = synth.ct_512(0)
    got = check_full(mask, sp)
    assert got["n_vertices"] > 100000
    # from a pinned host buffer, read in place over the host link: the same features
    host = torch.from_numpy(mask).pin_memory()
    ws = rad.Workspace()
    for _ in range(2):
        h = rad.extract_host(host.data_ptr(), mask.shape, sp, ws)
        for k in got:
            if k not in ("status",):
                assert h[k] == got[k], k


def test_batch_crops():
    crops = synth.batch_256(1, n=32)
    refs = [check_full(mask, sp) for mask, sp in crops]  # one at a time: meshes and triangle sets
    # the same crops through the batch path (one set of launches), against the oracle
    b = rad.Batch([torch.from_numpy(m).cuda() for m, _ in crops], [s for _, s in crops])
    for got, (mask, sp) in zip(b.run(), crops):
        ref, _ = oracle.features(mask, sp)
        assert_features(got, ref)


def test_blob_512_cubed():
    (mask, sp), = synth.blobs_512(0, count=1)
    got = check_full(mask, sp, method="hull")
    assert got["n_vertices"] > 1000000


def test_batch_8_blobs_512_cubed():
    """The large batched configuration: 8 masks of 512^3 (about 1e6 vertices
    each) in one batch, replayed as a graph; every mask against the oracle
    (its full mesh counts, volume and area; diameters from exact shortlists)."""
    masks = synth.blobs_512(1, count=8)
    devs = [torch.from_numpy(m).cuda() for m, _ in masks]
    b = rad.Batch(devs, [sp for _, sp in masks])
    first = b.run()
    again = b.run()  # graph replay
    for (mask, sp), got, got2 in zip(masks, first, again):
        ref, _ = oracle.features(mask, sp, "hull")
        assert_features(got, ref)
        assert got2 == got
        assert got["n_vertices"] > 500000
    del b, devs
    torch.cuda.empty_cache()


def test_soft_160():
    prob, sp = synth.soft_160(0)
    dev = torch.from_numpy(prob).cuda()
    m = rad.soft_mesh(dev, sp)
    got = rad.shape(m)
    ref, om = oracle.features(prob, sp)
    assert_features(got, ref)  # planar diameters of the soft map included
    idx2, t, tri = m.to_host()
    owner = (idx2.astype(np.int64) - (idx2 & 1)) // 2
    axis = np.argmax(idx2 & 1, axis=1)
    assert np.array_equal(owner, om.owner) and np.array_equal(axis, om.axis)
    assert np.array_equal(t, om.t)  # same FP64 formula, bit for bit
    assert np.array_equal(canon_tris(tri), canon_tris(om.tri))


def test_soft_binary_map_equals_mask():
    rng = np.random.default_rng(12)
    mask = (synth._noise_blob(rng, (30, 33, 37), 2.0) > 0.5).astype(np.uint8)
    sp = (0.8, 0.8, 3.0)
    mb = rad.mesh(torch.from_numpy(mask).cuda(), sp)
    ms = rad.soft_mesh(torch.from_numpy(mask.astype(np.float32)).cuda(), sp)
    fb, fs = rad.shape(mb), rad.shape(ms)
    assert fb["n_vertices"] == fs["n_vertices"] and fb["n_triangles"] == fs["n_triangles"]
    assert fb["MeshVolume"] == pytest.approx(fs["MeshVolume"], rel=1e-12)
    assert fb["SurfaceArea"] == pytest.approx(fs["SurfaceArea"], rel=1e-12)
    assert fb["Maximum3DDiameter"] == fs["Maximum3DDiameter"] and fb["argmax3d"] == fs["argmax3d"]
    ib, _, tb = mb.to_host()
    i_s, ts, tsr = ms.to_host()
    assert np.array_equal(ib, i_s) and np.all(ts == 0.5)
    assert np.array_equal(canon_tris(tb), canon_tris(tsr))
