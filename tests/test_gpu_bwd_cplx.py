"""The complex adjoint kernels (svd2_bwd_z / svd2_bwd_c) and the complex path
of the autograd Function:

- bit for bit against the oracle's complex adjoint on the same forward
  outputs (FP64 and FP32; NULL upstream gradients count as zero);
- central differences of the GPU forward through the autograd Function on a
  loss invariant under the phase gauge, in all 8 real directions, on
  matrices whose pivot choices stay fixed (tolerance conditioned on
  min(relative gap, s2/s1));
- torch.autograd.gradcheck of that loss on well-separated matrices.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import autograd as AG
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.helpers import bits_equal

pytestmark = pytest.mark.gpu


def _dev(x, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)


@pytest.mark.parametrize("dt,tdt", [(np.float64, torch.float64), (np.float32, torch.float32)])
def test_bwd_cplx_matches_oracle_bitwise(dt, tdt):
    n = 2**16 + 5
    A = inputs.normal_batch(n, 8, 201, dt)
    A[:, :8] = 0.0
    A[0, 1] = A[6, 1] = 1.0          # diag(1, 1): equal singular values
    A[0, 2] = 2.0                   # rank one
    rng = np.random.default_rng(202)
    gU, gV = rng.standard_normal((2, 8, n)).astype(dt)
    gS = rng.standard_normal((2, n)).astype(dt)
    r = S.svd2(_dev(A, tdt), backscale=True)
    dl = S.default_rel_delta(tdt)
    gA = S.svd2_bwd(r.U, r.V, r.smax, r.smin, _dev(gU, tdt), _dev(gV, tdt), _dev(gS[0], tdt),
                    _dev(gS[1], tdt), dl)
    torch.cuda.synchronize()
    o = oracle.bwd(r.U.cpu().numpy(), r.V.cpu().numpy(), r.smax.cpu().numpy(),
                   r.smin.cpu().numpy(), gU, gV, gS[0], gS[1], dl)
    assert bits_equal(gA.cpu().numpy(), o)
    gA0 = S.svd2_bwd(r.U, r.V, r.smax, r.smin, None, None, _dev(gS[0], tdt), None, dl)
    z = np.zeros_like(gU)
    o0 = oracle.bwd(r.U.cpu().numpy(), r.V.cpu().numpy(), r.smax.cpu().numpy(),
                    r.smin.cpu().numpy(), z, z, gS[0], np.zeros_like(gS[1]), dl)
    assert bits_equal(gA0.cpu().numpy(), o0)


def test_bwd_complex128_across_the_exponent_range():
    """Upstream gradients from subnormal to 2^300, with zeros, on matrices
    scaled by 2^-300, 1 or 2^300: the complex FP64 adjoint's products run on
    the integer pipe, and a matrix with a product outside its domain is read
    again and done with the hardware multiply.  Bit for bit against the
    oracle's complex adjoint (every value finite)."""
    n = 4099
    rng = np.random.default_rng(211)
    A = inputs.normal_batch(n, 8, 212, np.float64) * np.ldexp(1.0, rng.choice([-300, 0, 300],
                                                                             size=n))
    A = np.ascontiguousarray(A)

    def grad(*shape):
        x = rng.standard_normal(shape) * np.ldexp(1.0, rng.choice([-1070, -1040, -600, 0, 300],
                                                                  size=shape))
        x[rng.random(shape) < 0.05] = 0.0
        return x

    gU, gV, gS = grad(8, n), grad(8, n), grad(2, n)
    r = S.svd2(_dev(A), backscale=True)
    dl = S.default_rel_delta(torch.float64)
    gA = S.svd2_bwd(r.U, r.V, r.smax, r.smin, _dev(gU), _dev(gV), _dev(gS[0]), _dev(gS[1]), dl)
    torch.cuda.synchronize()
    with np.errstate(all="ignore"):
        o = oracle.bwd(r.U.cpu().numpy(), r.V.cpu().numpy(), r.smax.cpu().numpy(),
                       r.smin.cpu().numpy(), gU, gV, gS[0], gS[1], dl)
    assert np.isfinite(o).all()
    assert bits_equal(gA.cpu().numpy(), o)


def _loss(U, Sg, V, W):
    """Gauge-invariant loss (torch, split rows): weights on |U|^2, |V|^2, the
    singular values, and Re sum conj(W) o (u_i v_i^*) for both pairs."""
    W2, W3, w, W4r, W4i, W5r, W5i = W
    Ur, Ui, Vr, Vi = U[0::2], U[1::2], V[0::2], V[1::2]
    L = (W2 * (Ur**2 + Ui**2)).sum(0) + (W3 * (Vr**2 + Vi**2)).sum(0) + (w * Sg).sum(0)
    for cols, Wr, Wi in (([0, 1], W4r, W4i), ([2, 3], W5r, W5i)):
        ur, ui, vr, vi = Ur[cols], Ui[cols], Vr[cols], Vi[cols]
        # u_a conj(v_b) for a, b in {0, 1}: (ur + i ui)(vr - i vi)
        for a in range(2):
            for b in range(2):
                pr = ur[a] * vr[b] + ui[a] * vi[b]
                pi = ui[a] * vr[b] - ur[a] * vi[b]
                L = L + Wr[a, b] * pr + Wi[a, b] * pi       # Re(conj(W) p)
    return L


def _weights(n, seed):
    rng = np.random.default_rng(seed)
    d = lambda *s: _dev(rng.standard_normal(s))  # noqa: E731
    return (d(4, n), d(4, n), d(2, n), d(2, 2, n), d(2, 2, n), d(2, 2, n), d(2, 2, n))


def test_autograd_complex_vs_central_differences():
    n = 8192
    A = inputs.normal_batch(n, 8, 211)
    W = _weights(n, 212)
    Ad = _dev(A).requires_grad_(True)
    U, Sg, V = AG.svd2(Ad)
    _loss(U, Sg, V, W).sum().backward()
    grad = Ad.grad.cpu().numpy()
    s = Sg.detach().cpu().numpy()
    piv0 = oracle.svd2(A)["piv"]
    h = 1e-6
    same = np.ones(n, bool)
    fd = np.empty_like(A)
    with torch.no_grad():
        for e in range(8):
            Lpm = []
            for sg in (1, -1):
                Ap = A.copy()
                Ap[e] += sg * h
                same &= oracle.svd2(Ap)["piv"] == piv0
                Up, Sp, Vp = AG.svd2(_dev(Ap))
                Lpm.append(_loss(Up, Sp, Vp, W).cpu().numpy())
            fd[e] = (Lpm[0] - Lpm[1]) / (2 * h)
    gap = (s[0] - s[1]) / s[0]
    c = np.minimum(gap, s[1] / s[0])
    keep = same & (gap > 1e-3)
    err = np.abs(fd - grad).max(axis=0) / (np.abs(grad).max(axis=0) + 1)
    tol = 1e-7 + 1e-10 / c**2
    assert keep.mean() > 0.9
    assert np.all(err[keep] <= tol[keep]), float((err[keep] / tol[keep]).max())


def test_gradcheck_complex_small():
    A = inputs.normal_batch(512, 8, 221)
    r = oracle.svd2(A, backscale=True)
    keep = ((r["smax"] - r["smin"]) >= 0.05 * r["smax"]) & (r["smin"] >= 0.05 * r["smax"])
    for e in range(8):
        for sg in (1, -1):
            Ap = A.copy()
            Ap[e] += sg * 1e-5
            keep &= oracle.svd2(Ap)["piv"] == r["piv"]
    A = np.ascontiguousarray(A[:, keep][:, :8])
    assert A.shape[1] == 8
    W = _weights(8, 222)
    Ad = _dev(A).requires_grad_(True)
    f = lambda a: _loss(*AG.svd2(a), W)  # noqa: E731
    assert torch.autograd.gradcheck(f, (Ad,), eps=1e-6, atol=1e-6, rtol=1e-5)
