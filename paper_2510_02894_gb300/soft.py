"""torch.autograd.Function over the soft-map forward and adjoint kernels.

features = soft_shape_features(prob, spacing) returns the float64 tensor
(SurfaceArea, MeshVolume, Maximum3DDiameter) of the iso-0.5 mesh of a CUDA
float32 probability map; backward calls the hand-written adjoint
(rad_soft_backward), which recomputes the mesh instead of storing it.  Only
the diameter's argmax pair (two ints) is kept between the passes.
"""
import torch

from . import rad


class SoftShapeFeatures(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prob, spacing, ws):
        (area, vol, diam), argmax = rad.soft_forward(prob, spacing, ws)
        ctx.save_for_backward(prob)
        ctx.spacing = tuple(float(s) for s in spacing)
        ctx.argmax = argmax
        ctx.ws = ws
        return torch.tensor([area, vol, diam], dtype=torch.float64, device=prob.device)

    @staticmethod
    def backward(ctx, gout):
        (prob,) = ctx.saved_tensors
        g = [float(v) for v in gout.detach().to(torch.float64).cpu().tolist()]
        grad = torch.empty(prob.shape, dtype=torch.float64, device=prob.device)
        rad.soft_backward(prob, ctx.spacing, g, ctx.argmax, grad, ctx.ws)
        return grad.to(prob.dtype), None, None


def soft_shape_features(prob, spacing, ws=None):
    """(SurfaceArea, MeshVolume, Maximum3DDiameter) with gradients to prob."""
    return SoftShapeFeatures.apply(prob, spacing, ws if ws is not None else rad.Workspace())


SIX = ("SurfaceArea", "MeshVolume", "Maximum3DDiameter", "Maximum2DDiameterSlice", "Maximum2DDiameterColumn",
       "Maximum2DDiameterRow")


class SoftShapeFeatures6(torch.autograd.Function):
    """(A, V, D3, DSlice, DColumn, DRow) of one map; backward through
    rad_soft_backward_planes (each argmax pair, planar ones with their plane,
    held fixed)."""

    @staticmethod
    def forward(ctx, prob, spacing, ws):
        f = rad.soft_features(prob, spacing, ws)
        ctx.save_for_backward(prob)
        ctx.spacing = tuple(float(s) for s in spacing)
        ctx.feats = f
        ctx.ws = ws
        return torch.tensor([f[k] for k in SIX], dtype=torch.float64, device=prob.device)

    @staticmethod
    def backward(ctx, gout):
        (prob,) = ctx.saved_tensors
        g = [float(v) for v in gout.detach().to(torch.float64).cpu().tolist()]
        grad = torch.empty(prob.shape, dtype=torch.float64, device=prob.device)
        rad.soft_backward_planes(prob, ctx.spacing, g, ctx.feats, grad, ctx.ws)
        return grad.to(prob.dtype), None, None


def soft_shape_features6(prob, spacing, ws=None):
    """(A, V, D3, DSlice, DColumn, DRow) with gradients to prob."""
    return SoftShapeFeatures6.apply(prob, spacing, ws if ws is not None else rad.Workspace())


class SoftBatchFeatures(torch.autograd.Function):
    """The six features of several maps in one set of launches, forward and
    backward (rad_soft_batch_forward / rad_soft_batch_backward); returns an
    (n, 6) float64 tensor."""

    @staticmethod
    def forward(ctx, spacings, ws, *probs):
        feats = rad.soft_batch_forward(list(probs), spacings, ws)
        ctx.save_for_backward(*probs)
        ctx.spacings = [tuple(float(v) for v in s) for s in spacings]
        ctx.feats = feats
        ctx.ws = ws
        return torch.tensor([[f[k] for k in SIX] for f in feats], dtype=torch.float64, device=probs[0].device)

    @staticmethod
    def backward(ctx, gout):
        probs = ctx.saved_tensors
        g = gout.detach().to(torch.float64).cpu().tolist()
        grads = [torch.empty(p.shape, dtype=torch.float64, device=p.device) for p in probs]
        rad.soft_batch_backward(list(probs), ctx.spacings, g, ctx.feats, grads, ctx.ws)
        return (None, None) + tuple(gr.to(p.dtype) for gr, p in zip(grads, probs))


def soft_batch_features(probs, spacings, ws=None):
    """(n, 6) features of n maps with gradients to each map."""
    return SoftBatchFeatures.apply(list(spacings), ws if ws is not None else rad.Workspace(), *probs)
