"""The projector as a differentiable PyTorch operation.

``TomoProject.apply(cube, geom, pointing, nu, nv, mask, n_frames, ctx,
map_mask)`` returns ``P x`` (Eq. lo, stacked over images as in Eq. srt), or
``P K x`` with a map mask (K zeroes the excluded voxels), including the smoothly
time-varying model in which each image sees the linear interpolation of its
two neighbouring frames (Section 3.3.3, a parameterised temporal evolution).
Its backward pass is the transpose kernel: ``grad_x = P^T grad_y`` with the
same segments, mask, gains and time weights (``K P^T grad_y`` with a map
mask), so gradients of any loss built on the projection flow to every frame.  The pointing is not differentiated.
"""

import torch

from . import tomo


class TomoProject(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cube, geom, pointing, nu, nv, mask=None, n_frames=1,
                ctx=None, map_mask=None, kind="emission", limb_u=0.0):
        fctx.geom, fctx.pointing = geom, pointing
        fctx.kind, fctx.limb_u = kind, limb_u
        fctx.n_frames, fctx.tctx = n_frames, ctx
        fctx.cube_shape, fctx.cube_dtype = cube.shape, cube.dtype
        empty = cube.new_empty(0)
        fctx.save_for_backward(mask if mask is not None else empty,
                               map_mask if map_mask is not None else empty)
        fctx.has_mask = mask is not None
        fctx.has_map_mask = map_mask is not None
        return tomo.tomo_project(cube.contiguous(), geom, pointing, nu, nv,
                                 mask=mask, n_frames=n_frames, ctx=ctx,
                                 map_mask=map_mask, kind=kind, limb_u=limb_u)

    @staticmethod
    def backward(fctx, grad_y):
        mask, map_mask = fctx.saved_tensors
        grad = None
        if fctx.needs_input_grad[0]:
            g = tomo.tomo_backproject(
                grad_y.contiguous().float(), fctx.geom, fctx.pointing,
                mask=mask if fctx.has_mask else None,
                n_frames=fctx.n_frames, ctx=fctx.tctx,
                map_mask=map_mask if fctx.has_map_mask else None,
                kind=fctx.kind, limb_u=fctx.limb_u)
            grad = g.reshape(fctx.cube_shape).to(fctx.cube_dtype)
        return (grad, None, None, None, None, None, None, None, None, None,
                None)


def project(cube, geom, pointing, nu, nv, mask=None, n_frames=1, ctx=None,
            map_mask=None, kind="emission", limb_u=0.0):
    """Differentiable ``P x`` (``P K x`` with a map mask; the Thomson
    operator of white-light images with ``kind`` "pB" or "B")."""
    return TomoProject.apply(cube, geom, pointing, nu, nv, mask, n_frames, ctx,
                             map_mask, kind, limb_u)
