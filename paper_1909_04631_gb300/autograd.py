"""torch.autograd wrappers of the differentiable S-BKI form.

Forward and backward both run in libsbki's CUDA kernels (sbki_insert_training,
sbki_heldout_loglik, sbki_grad_add_alpha, sbki_backward); these classes only
move tensors across the C ABI.  l and sigma0 are 0-dim float tensors; xyz is
a float32 [p,3] CUDA tensor of world coordinates and labels an int [p] tensor
with classes 0..K.  Each forward builds a map of the given parameters (the
support of Eq. (kernel) depends on l), which is kept for the backward pass.
"""
from __future__ import annotations

import torch

from . import sbki as _sb


def _params_with(params: _sb.Params, l: torch.Tensor, sigma0: torch.Tensor) -> _sb.Params:
    p = _sb.Params.from_buffer_copy(params)
    p.length_scale = float(l)
    p.sigma0 = float(sigma0)
    return p


def _xyzl(xyz: torch.Tensor, labels: torch.Tensor) -> torch.Tensor:
    return torch.cat([xyz.detach().float().reshape(-1, 3), labels.reshape(-1, 1).float()], 1).contiguous()


class SBKIFunction(torch.autograd.Function):
    """(keys, alpha) = S-BKI(xyz, labels; l, sigma0): alpha (with prior) at every
    voxel of the blocks the training set reaches, in the map's pool order
    (blocks in allocation order, x fastest inside a block).  keys is not
    differentiable; alpha is differentiable in xyz, l and sigma0.  Both stay on
    the device: forward and backward make no host copy of alpha or its
    gradient."""

    @staticmethod
    def forward(ctx, xyz, labels, l, sigma0, params):
        m = _sb.Map(_params_with(params, l, sigma0))
        xyzl = _xyzl(xyz, labels)
        m.insert_training(xyzl[:, :3], xyzl[:, 3].to(torch.int32))
        kt, at = m.export_blocks(device=xyz.device)
        ctx.m, ctx.xyzl = m, xyzl
        ctx.keys = kt
        ctx.shapes = (l.shape, sigma0.shape)
        ctx.mark_non_differentiable(kt)
        return kt, at

    @staticmethod
    def backward(ctx, _gkeys, galpha):
        m = ctx.m
        m.grad_clear()
        m.grad_add_alpha(ctx.keys, galpha.detach().float().contiguous())
        gl, gs, gx = m.backward(ctx.xyzl, grad_xyz=ctx.needs_input_grad[0])
        dev = ctx.xyzl.device
        lshape, sshape = ctx.shapes
        return (gx, None, torch.full(lshape, gl, dtype=torch.float32, device=dev),
                torch.full(sshape, gs, dtype=torch.float32, device=dev), None)


class HeldoutLogLik(torch.autograd.Function):
    """LL = sum_h log(alpha^{y_h} / sum_k alpha^k) at the voxels of held-out
    points, with alpha from the training set (xyz, labels; l, sigma0)."""

    @staticmethod
    def forward(ctx, xyz, labels, l, sigma0, held_xyz, held_labels, params):
        m = _sb.Map(_params_with(params, l, sigma0))
        xyzl = _xyzl(xyz, labels)
        m.insert_training(xyzl[:, :3], xyzl[:, 3].to(torch.int32))
        m.grad_clear()
        ll = m.heldout_loglik(held_xyz.detach().float().contiguous(), held_labels.to(torch.int32).contiguous(),
                              grad=True)
        ctx.m, ctx.xyzl = m, xyzl
        ctx.shapes = (l.shape, sigma0.shape)
        return torch.tensor(ll, dtype=torch.float64, device=xyz.device)

    @staticmethod
    def backward(ctx, g):
        gl, gs, gx = ctx.m.backward(ctx.xyzl, grad_xyz=ctx.needs_input_grad[0])
        dev = ctx.xyzl.device
        s = float(g)
        lshape, sshape = ctx.shapes
        return ((gx * s) if gx is not None else None, None,
                torch.full(lshape, gl * s, dtype=torch.float32, device=dev),
                torch.full(sshape, gs * s, dtype=torch.float32, device=dev), None, None, None)


def sbki_alpha(xyz, labels, l, sigma0, params):
    return SBKIFunction.apply(xyz, labels, l, sigma0, params)


def heldout_loglik(xyz, labels, l, sigma0, held_xyz, held_labels, params):
    return HeldoutLogLik.apply(xyz, labels, l, sigma0, held_xyz, held_labels, params)
