"""torch.autograd.Function around the batched 2x2 SVD (real and complex).

Forward: the CUDA forward kernel with back-scaling (Fig. 1), so the singular
values are those of A itself.  Backward: the hand-written adjoint kernels
(svd2_bwd_{d,s,z,c}) with the near-equal singular value safeguard; for
complex data, with the phase-gauge terms (exact for gauge-invariant losses).
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
    """Differentiable batched SVD of 2x2 matrices in the split layout: A (4, n)
    real or (8, n) complex (real and imaginary rows), float64/float32 on a CUDA
    device -> (U, S (2, n), V) with A = U diag(S) V^* per matrix.  For complex
    data the gradient rows are dL/dRe and dL/dIm; a loss of U and V should be
    invariant under the phase gauge U, V -> U D, V D for its gradient to be
    defined."""
    if A.dim() != 2 or A.shape[0] not in (4, 8):
        raise ValueError("A must have shape (4, n) or (8, n)")
    return Svd2Fn.apply(A, rel_delta)
