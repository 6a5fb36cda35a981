"""P and P^T as a differentiable PyTorch operation.

`project(geom, f)` maps a volume (nz, ny, nx) or a batch (B, nz, ny, nx) to its projections
with the library's Siddon projector; its backward pass is the library's exact adjoint
(cbct_backproject), so gradients of any loss on the projections flow back to the volume —
for ½‖P f − y‖² the gradient is P^T (P f − y) (Eq. (A1) makes P^T the exact adjoint).
Both passes run in the CUDA library; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import Geometry, backproject_batch, project_batch


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, geom):
        ctx.geom = geom
        batched = f.dim() == 4
        fb = f if batched else f.unsqueeze(0)
        out = project_batch(geom, fb.contiguous())
        return out if batched else out[0]

    @staticmethod
    def backward(ctx, grad_out):
        geom = ctx.geom
        batched = grad_out.dim() == 4
        gb = grad_out if batched else grad_out.unsqueeze(0)
        grad_f = backproject_batch(geom, gb.contiguous().to(torch.float32))
        return (grad_f if batched else grad_f[0]), None


def project(geom: Geometry, f: torch.Tensor) -> torch.Tensor:
    """Differentiable P f; f is (nz, ny, nx) or (B, nz, ny, nx), float32 on the GPU."""
    return _Project.apply(f, geom)
