"""The projector as a differentiable PyTorch operation.

``TomoProject.apply(cube, geom, pointing, nu, nv, mask, n_frames)`` returns
``P x`` (Eq. lo, stacked over images as in Eq. srt), including the smoothly
time-varying model in which each image sees the linear interpolation of its
two neighbouring frames (Section 3.3.3, a parameterised temporal evolution).
Its backward pass is the transpose kernel: ``grad_x = P^T grad_y`` with the
same segments, mask, gains and time weights, so gradients of any loss built
on the projection flow to every frame.  The pointing is not differentiated.
"""

import torch

from . import tomo


class TomoProject(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cube, geom, pointing, nu, nv, mask=None, n_frames=1,
                ctx=None):
        fctx.geom, fctx.pointing = geom, pointing
        fctx.n_frames, fctx.tctx = n_frames, ctx
        fctx.cube_shape, fctx.cube_dtype = cube.shape, cube.dtype
        fctx.save_for_backward(mask if mask is not None else cube.new_empty(0))
        fctx.has_mask = mask is not None
        return tomo.tomo_project(cube.contiguous(), geom, pointing, nu, nv,
                                 mask=mask, n_frames=n_frames, ctx=ctx)

    @staticmethod
    def backward(fctx, grad_y):
        (mask,) = fctx.saved_tensors
        grad = None
        if fctx.needs_input_grad[0]:
            g = tomo.tomo_backproject(
                grad_y.contiguous().float(), fctx.geom, fctx.pointing,
                mask=mask if fctx.has_mask else None,
                n_frames=fctx.n_frames, ctx=fctx.tctx)
            grad = g.reshape(fctx.cube_shape).to(fctx.cube_dtype)
        return grad, None, None, None, None, None, None, None


def project(cube, geom, pointing, nu, nv, mask=None, n_frames=1, ctx=None):
    """Differentiable ``P x``."""
    return TomoProject.apply(cube, geom, pointing, nu, nv, mask, n_frames, ctx)
