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
