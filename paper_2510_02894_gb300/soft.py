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
