"""torch.autograd.Function around the batched real 2x2 SVD.

Forward: the CUDA forward kernel with back-scaling (Fig. 1), so the singular
values are those of A itself.  Backward: the hand-written adjoint kernel
(svd2_bwd_d / svd2_bwd_s) with the near-equal singular value safeguard.
The singular vectors of the method are fixed by its pivoting and sign choices
(Eq. 29), which are locally constant, so the map A -> (U, S, V) is smooth
wherever those choices and s1 != s2 hold, and the adjoint is its derivative.
"""
from __future__ import annotations

import torch

from . import svd2 as S


class Svd2Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A: torch.Tensor, rel_delta: float | None = None):
        r = S.svd2(A.contiguous(), backscale=True)
        Sg = torch.stack([r.smax, r.smin])
        ctx.save_for_backward(r.U, r.V, r.smax, r.smin)
        ctx.rel_delta = rel_delta
        return r.U, Sg, r.V

    @staticmethod
    def backward(ctx, gU, gS, gV):
        U, V, s1, s2 = ctx.saved_tensors
        g1 = gS[0].contiguous() if gS is not None else None
        g2 = gS[1].contiguous() if gS is not None else None
        gA = S.svd2_bwd(U, V, s1, s2, None if gU is None else gU.contiguous(),
                        None if gV is None else gV.contiguous(), g1, g2, ctx.rel_delta)
        return gA, None


def svd2(A: torch.Tensor, rel_delta: float | None = None):
    """Differentiable batched SVD of real 2x2 matrices in the split layout:
    A (4, n) float64/float32 on a CUDA device -> (U (4, n), S (2, n), V (4, n))
    with A = U diag(S) V^T per matrix."""
    if A.dim() != 2 or A.shape[0] != 4:
        raise ValueError("A must have shape (4, n) (real matrices)")
    return Svd2Fn.apply(A, rel_delta)
