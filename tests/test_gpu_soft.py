"""Soft probability maps on the GPU: forward features and the hand-written
adjoint against the FP64 oracle (analytic gradient), closed forms, central
finite differences and torch autograd."""
import math

import numpy as np
import pytest

import oracle
from paper_2510_02894_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2510_02894_gb300 import rad
    from paper_2510_02894_gb300.soft import soft_shape_features


def gpu_forward(prob, sp, ws):
    return rad.soft_forward(torch.from_numpy(prob).cuda(), sp, ws)


def gpu_grad(prob, sp, gout, argmax, ws):
    dev = torch.from_numpy(prob).cuda()
    g = torch.empty(dev.shape, dtype=torch.float64, device="cuda")
    rad.soft_backward(dev, sp, gout, argmax, g, ws)
    return g.cpu().numpy()


@pytest.mark.parametrize("n", [40, 160])
def test_forward_and_gradient_match_oracle(n):
    prob, sp = synth.soft_160(1, n=n)
    ws = rad.Workspace()
    (A, V, D), am = gpu_forward(prob, sp, ws)
    ref, om = oracle.features(prob, sp)
    assert abs(A - ref["SurfaceArea"]) <= 1e-9 * ref["SurfaceArea"]
    assert abs(V - ref["MeshVolume"]) <= 1e-9 * ref["MeshVolume"]
    assert D == ref["Maximum3DDiameter"] and am == tuple(ref["argmax3d"])
    gout = (0.7, 0.3, 1.3)
    g = gpu_grad(prob, sp, gout, am, ws)
    gr = oracle.soft_grad(om, *gout, ref["argmax3d"])
    scale = np.abs(gr).max()
    assert np.all(np.abs(g - gr) <= 1e-9 * np.abs(gr) + 1e-12 * scale)
    assert np.array_equal(g != 0, gr != 0)


@pytest.mark.parametrize("v", [0.6, 0.9])
def test_single_voxel_gradient_closed_form(v):
    prob = np.zeros((3, 3, 3), np.float32)
    prob[1, 1, 1] = v
    v = float(np.float32(v))
    ws = rad.Workspace()
    (A, V, D), am = gpu_forward(prob, (1.0, 1.0, 1.0), ws)
    r = 1.0 - 1.0 / (2.0 * v)
    assert V == pytest.approx(4.0 / 3.0 * r ** 3, rel=1e-13)
    assert A == pytest.approx(4.0 * math.sqrt(3.0) * r * r, rel=1e-13)
    gV = gpu_grad(prob, (1.0, 1.0, 1.0), (0.0, 1.0, 0.0), am, ws)
    gA = gpu_grad(prob, (1.0, 1.0, 1.0), (1.0, 0.0, 0.0), am, ws)
    gD = gpu_grad(prob, (1.0, 1.0, 1.0), (0.0, 0.0, 1.0), am, ws)
    assert gV[1, 1, 1] == pytest.approx(2 * r * r / v ** 2, rel=1e-12)
    assert gA[1, 1, 1] == pytest.approx(4 * math.sqrt(3) * r / v ** 2, rel=1e-12)
    assert gD[1, 1, 1] == pytest.approx(1.0 / v ** 2, rel=1e-12)


def test_gradient_central_differences_160():
    """64 random voxels with a non-zero gradient; h = 1e-4 on the float32
    values (divided by the exactly represented step)."""
    prob, sp = synth.soft_160(2)
    ws = rad.Workspace()
    w = (0.7, 0.3, 1.3)
    (A, V, D), am = gpu_forward(prob, sp, ws)
    g = gpu_grad(prob, sp, w, am, ws)
    band = np.argwhere(g != 0.0)
    rng = np.random.default_rng(3)
    dev = torch.from_numpy(prob).cuda()
    checked = 0
    for idx in rng.permutation(len(band)):
        z, y, x = band[idx]
        v0 = dev[z, y, x].item()
        vals, feats = [], []
        for sgn in (1.0, -1.0):
            dev[z, y, x] = float(np.float32(v0 + sgn * 1e-4))
            vals.append(dev[z, y, x].item())
            feats.append(rad.soft_forward(dev, sp, ws))
        dev[z, y, x] = float(np.float32(v0))
        if feats[0][1] != am or feats[1][1] != am:
            continue  # the argmax pair moved: D3 is not differentiable here
        Lp = sum(wk * f for wk, f in zip(w, feats[0][0]))
        Lm = sum(wk * f for wk, f in zip(w, feats[1][0]))
        fd = (Lp - Lm) / (vals[0] - vals[1])
        assert fd == pytest.approx(g[z, y, x], rel=2e-4, abs=1e-5), (z, y, x, fd, g[z, y, x])
        checked += 1
        if checked == 64:
            break
    assert checked == 64


def test_autograd_function():
    prob, sp = synth.soft_160(4, n=48)
    t = torch.from_numpy(prob).cuda().requires_grad_(True)
    feats = soft_shape_features(t, sp)
    w = torch.tensor([0.5, -0.25, 2.0], dtype=torch.float64, device="cuda")
    (feats * w).sum().backward()
    ref, om = oracle.features(prob, sp)
    gr = oracle.soft_grad(om, 0.5, -0.25, 2.0, ref["argmax3d"])
    got = t.grad.double().cpu().numpy()
    assert np.allclose(got, gr, rtol=1e-6, atol=1e-9 * np.abs(gr).max())
    assert feats[2].item() == ref["Maximum3DDiameter"]


def _layered(n=24):
    """A map that varies along z only inside a box: every z-edge vertex of a
    slab has the same coordinate, so the planes off the grid planes are large;
    a patch of exact 0.5 values puts vertices exactly on grid planes (t = 0
    or t = 1)."""
    prob = np.zeros((n, n, n), np.float32)
    z = np.arange(n)
    prof = (0.95 - 0.04 * np.abs(z - n / 2.0)).astype(np.float32)
    prob[:, 3:n - 3, 4:n - 5] = prof[:, None, None]
    prob[n // 2, 6:10, 7:11] = 0.5
    return prob


@pytest.mark.parametrize("case", ["ellipsoid40", "ellipsoid96", "layered", "aniso"])
def test_soft_planar_diameters_match_oracle(case):
    """Slice, Column and Row diameters of soft maps: planes are the sets of
    vertices with exactly equal FP64 coordinates, on or off the grid planes."""
    from tests.helpers import assert_features
    if case == "ellipsoid40":
        prob, sp = synth.soft_160(5, n=40)
    elif case == "ellipsoid96":
        prob, sp = synth.soft_160(6, n=96)
    elif case == "layered":
        prob, sp = _layered(), (1.0, 1.0, 1.0)
    else:
        prob, sp = synth.soft_160(7, n=40)[0], (0.7, 0.9, 2.5)
    m = rad.soft_mesh(torch.from_numpy(prob).cuda(), sp)
    got = rad.shape(m)
    ref, _ = oracle.features(prob, sp)
    assert_features(got, ref)
    assert got["Maximum2DDiameterSlice"] > 0.0


def test_soft_layered_has_planes_off_the_grid():
    """The layered map's Slice diameter comes from z-edge vertices off the
    grid planes or from grid planes; either way the oracle's exact grouping
    is met (checked above); here the grouping itself is exercised: many
    vertices share a fractional z."""
    prob = _layered()
    om = oracle.OracleMesh(prob, (1.0, 1.0, 1.0))
    z = om.u[:, 2]
    frac = z[z != np.floor(z)]
    vals, counts = np.unique(frac, return_counts=True)
    assert counts.max() >= 16


W6 = (0.4, -0.2, 0.8, 1.3, -0.9, 0.7)  # A, V, D3, Slice, Column, Row


def test_soft_features_and_planar_gradient_match_oracle():
    """rad_soft_features and rad_soft_backward_planes against the oracle's
    features and its analytic gradient with the planar terms."""
    from tests.helpers import assert_features
    prob, sp = synth.soft_160(8, n=48)
    sp = (0.9, 0.8, 1.5)
    ws = rad.Workspace()
    dev = torch.from_numpy(prob).cuda()
    f = rad.soft_features(dev, sp, ws)
    ref, om = oracle.features(prob, sp)
    assert_features(f, ref)
    g = torch.empty(dev.shape, dtype=torch.float64, device="cuda")
    rad.soft_backward_planes(dev, sp, W6, f, g, ws)
    gr = oracle.soft_grad_planes(om, W6[0], W6[1], W6[2:], [ref[k] for k in rad.ARGMAX_KEYS])
    got = g.cpu().numpy()
    scale = np.abs(gr).max()
    assert np.all(np.abs(got - gr) <= 1e-9 * np.abs(gr) + 1e-12 * scale)
    assert np.array_equal(got != 0, gr != 0)


def _soft_batch_inputs():
    maps = [(synth.soft_160(10, n=32)[0], (1.0, 1.0, 1.0)), (synth.soft_160(11, n=40)[0], (0.7, 0.7, 2.5)),
            (_layered(20), (1.0, 1.0, 1.0)), (synth.soft_160(12, n=28)[0], (0.5, 0.6, 1.0)),
            (np.zeros((6, 7, 8), np.float32), (1.0, 1.0, 1.0))]
    return maps


def test_soft_batch_matches_single_maps_and_oracle():
    """One batch of five maps (one of them empty) against per-map calls and
    the oracle: diameters and argmax pairs bit-exact, A and V within 1e-9;
    gradients against the oracle's per map."""
    from tests.helpers import assert_features
    maps = _soft_batch_inputs()
    devs = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p, _ in maps]
    sps = [s for _, s in maps]
    ws = rad.Workspace()
    feats = rad.soft_batch_forward(devs, sps, ws)
    refs = [oracle.features(p, s) for p, s in maps]
    for f, (ref, _) in zip(feats, refs):
        assert_features(f, ref)
    grads = [torch.empty(d.shape, dtype=torch.float64, device="cuda") for d in devs]
    gouts = [tuple(w * (1 + 0.1 * i) for w in W6) for i in range(len(devs))]
    rad.soft_batch_backward(devs, sps, gouts, feats, grads, ws)
    for g, go, (ref, om) in zip(grads, gouts, refs):
        got = g.cpu().numpy()
        if ref["n_vertices"] == 0:
            assert not got.any()
            continue
        gr = oracle.soft_grad_planes(om, go[0], go[1], go[2:], [ref[k] for k in rad.ARGMAX_KEYS])
        scale = np.abs(gr).max()
        assert np.all(np.abs(got - gr) <= 1e-9 * np.abs(gr) + 1e-12 * scale)
    # the single-map calls agree with the batch
    ws1 = rad.Workspace()
    for d, s, f in zip(devs, sps, feats):
        f1 = rad.soft_features(d, s, ws1)
        for k in rad.ARGMAX_KEYS + ("Maximum3DDiameter", "Maximum2DDiameterSlice", "Maximum2DDiameterColumn",
                                    "Maximum2DDiameterRow", "n_vertices", "n_triangles"):
            assert f1[k] == f[k], k


def test_soft_batch_rejects_bad_arguments():
    ws = rad.Workspace()
    p = torch.from_numpy(synth.soft_160(13, n=20)[0]).cuda()
    f = rad.soft_features(p, (1.0, 1.0, 1.0), ws)
    g = torch.empty(p.shape, dtype=torch.float64, device="cuda")
    bad = dict(f)
    bad["argmax_row"] = (0, f["n_vertices"])  # outside the mesh
    with pytest.raises(rad.RadError):
        rad.soft_batch_backward([p], [(1.0, 1.0, 1.0)], [W6], [bad], [g], ws)
    with pytest.raises(ValueError):
        rad.soft_batch_forward([], [], ws)


def test_autograd_planes_and_batch():
    """The six-feature autograd functions (one map, and a batch of maps)
    against the oracle's forward values and analytic gradients."""
    from paper_2510_02894_gb300.soft import SIX, soft_batch_features, soft_shape_features6
    w = torch.tensor([0.3, -0.4, 1.1, 0.9, -0.6, 0.5], dtype=torch.float64, device="cuda")
    maps = [synth.soft_160(20, n=28), synth.soft_160(21, n=36)]
    # one map
    prob, sp = maps[0]
    t = torch.from_numpy(prob).cuda().requires_grad_(True)
    f6 = soft_shape_features6(t, sp)
    (f6 * w).sum().backward()
    ref, om = oracle.features(prob, sp)
    assert [f6[k].item() for k in range(6)][2:] == [ref[k] for k in SIX[2:]]
    gr = oracle.soft_grad_planes(om, 0.3, -0.4, (1.1, 0.9, -0.6, 0.5), [ref[k] for k in rad.ARGMAX_KEYS])
    assert np.allclose(t.grad.double().cpu().numpy(), gr, rtol=1e-6, atol=1e-9 * np.abs(gr).max())
    # a batch of two
    ts = [torch.from_numpy(p).cuda().requires_grad_(True) for p, _ in maps]
    fb = soft_batch_features(ts, [s for _, s in maps])
    (fb * w).sum().backward()
    for tk, (p, s), row in zip(ts, maps, fb):
        ref, om = oracle.features(p, s)
        assert [row[k].item() for k in range(2, 6)] == [ref[k] for k in SIX[2:]]
        gr = oracle.soft_grad_planes(om, 0.3, -0.4, (1.1, 0.9, -0.6, 0.5), [ref[k] for k in rad.ARGMAX_KEYS])
        assert np.allclose(tk.grad.double().cpu().numpy(), gr, rtol=1e-6, atol=1e-9 * np.abs(gr).max())
