"""The adjoint kernels (svd2_bwd_d / svd2_bwd_s) and the autograd Function.

- bit for bit against the oracle's adjoint on the same forward outputs;
- central finite differences (h = 1e-6) of the GPU forward, on matrices with
  relative singular-value gap >= 1e-3 whose pivot choices (from the oracle) do
  not change at A +- h E_ij;
- the binary128 reference gradient (the method and the adjoint in binary128)
  for every gap class: error <= 16 eps / gap relative to the gradient's
  natural size N = max(|ref|, (|gU| + |gV|) / (s1 - s2)) -- the rotation term
  is (a + b) / (2 (s1 - s2)) with a, b of size |gU| + |gV| and errors of
  eps / gap of that size (the singular vectors' own condition number), even
  where a + b cancels; measured constant on the oracle <= 3.5;
- FP32 gradients against FP64 ones on the same inputs where both pick the same
  pivots: <= 16 eps32 / gap relative to N for gap >= 1e-2 (measured <= 3);
- the gradient workload at full size (n = 2^22), sampled.
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

EPS64 = 2.0**-52
EPS32 = 2.0**-23


def _dev(x, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)


def _edge_and_batch(n, dt):
    g = inputs.grad_batch(n, seed=81)
    A = g["A"]
    extra = np.array([[0.0, 0.0, 0.0, 0.0], [1.0, 0.0, 0.0, 1.0], [2.0, 0.0, 0.0, 2.0],
                      [0.6, 0.8, -0.8, 0.6], [3.0, 0.0, 0.0, 1e-300 if dt == np.float64 else 0.0]]).T
    A = np.concatenate([A, extra], axis=1).astype(dt)
    m = A.shape[1]
    rng = np.random.default_rng(82)
    gU, gV = rng.standard_normal((2, 4, m)).astype(dt)
    gS = rng.standard_normal((2, m)).astype(dt)
    return np.ascontiguousarray(A), gU, gV, gS


@pytest.mark.parametrize("dt,tdt", [(np.float64, torch.float64), (np.float32, torch.float32)])
def test_bwd_matches_oracle_adjoint_bitwise(dt, tdt):
    A, gU, gV, gS = _edge_and_batch(2**17 + 3, dt)
    r = S.svd2(_dev(A, tdt), backscale=True)
    dl = S.default_rel_delta(tdt)
    gA = S.svd2_bwd(r.U, r.V, r.smax, r.smin, _dev(gU, tdt), _dev(gV, tdt), _dev(gS[0], tdt),
                    _dev(gS[1], tdt), dl)
    torch.cuda.synchronize()
    o = oracle.bwd(r.U.cpu().numpy(), r.V.cpu().numpy(), r.smax.cpu().numpy(),
                   r.smin.cpu().numpy(), gU, gV, gS[0], gS[1], dl)
    assert bits_equal(gA.cpu().numpy(), o)


@pytest.mark.parametrize("rows", [4, 8])
@pytest.mark.parametrize("dt,tdt", [(np.float64, torch.float64), (np.float32, torch.float32)])
def test_bwd_equal_singular_values_without_safeguard(rows, dt, tdt):
    """rel_delta = 0 with s1 = s2: the rotation term takes the safeguard's
    value at zero gap (0), not 0/0; gA is finite and equal to the oracle's."""
    rng = np.random.default_rng(91)
    n = 4099
    U, V = rng.standard_normal((2, rows, n)).astype(dt)
    s = (np.abs(rng.standard_normal(n)) + 0.5).astype(dt)
    gU, gV = rng.standard_normal((2, rows, n)).astype(dt)
    g1, g2 = rng.standard_normal((2, n)).astype(dt)
    gA = S.svd2_bwd(_dev(U, tdt), _dev(V, tdt), _dev(s, tdt), _dev(s, tdt), _dev(gU, tdt),
                    _dev(gV, tdt), _dev(g1, tdt), _dev(g2, tdt), 0.0)
    torch.cuda.synchronize()
    g = gA.cpu().numpy()
    assert np.all(np.isfinite(g))
    assert bits_equal(g, oracle.bwd(U, V, s, s, gU, gV, g1, g2, 0.0))


def test_bwd_null_gradients_are_zero():
    A, gU, gV, gS = _edge_and_batch(1000, np.float64)
    r = S.svd2(_dev(A), backscale=True)
    gA = S.svd2_bwd(r.U, r.V, r.smax, r.smin, None, None, _dev(gS[0]), None)
    z = np.zeros_like(gU)
    o = oracle.bwd(r.U.cpu().numpy(), r.V.cpu().numpy(), r.smax.cpu().numpy(),
                   r.smin.cpu().numpy(), z, z, gS[0], np.zeros_like(gS[1]),
                   S.default_rel_delta(torch.float64))
    assert bits_equal(gA.cpu().numpy(), o)


def test_bwd_fp32_vector_and_scalar_paths():
    """The FP32 adjoint takes two matrices per thread when every array is
    8-byte aligned and one otherwise (arrays 4 bytes off): both give the
    oracle's bits, with and without NULL upstream gradients, on an odd n (the
    tail of the two-per-thread path)."""
    A, gU, gV, gS = _edge_and_batch(2**16 + 1, np.float32)
    n = A.shape[1]
    r = S.svd2(_dev(A, torch.float32), backscale=True)
    dl = S.default_rel_delta(torch.float32)
    Uh, Vh = r.U.cpu().numpy(), r.V.cpu().numpy()
    s1h, s2h = r.smax.cpu().numpy(), r.smin.cpu().numpy()

    def off(x):   # a copy whose data start 4 bytes past an 8-byte boundary
        x = np.ascontiguousarray(x)
        buf = torch.zeros(x.shape[:-1] + (x.shape[-1] + 1,), dtype=torch.float32, device="cuda")
        buf[..., 1:] = torch.from_numpy(x).cuda()
        return buf[..., 1:]

    z4, z1 = np.zeros_like(gU), np.zeros_like(gS[0])
    for with_grads in (True, False):
        o = oracle.bwd(Uh, Vh, s1h, s2h, gU if with_grads else z4, gV, gS[0],
                       gS[1] if with_grads else z1, dl)
        for mk in (lambda x: _dev(x, torch.float32), off):
            gA = S.svd2_bwd(mk(Uh), mk(Vh), mk(s1h), mk(s2h), mk(gU) if with_grads else None,
                            mk(gV), mk(gS[0]), mk(gS[1]) if with_grads else None, dl)
            torch.cuda.synchronize()
            assert bits_equal(gA.cpu().numpy(), o), (with_grads, n)


def _natural(ref, gU, gV, s1, s2):
    return np.maximum(np.abs(ref).max(axis=0),
                      (np.abs(gU).max(axis=0) + np.abs(gV).max(axis=0)) / (s1 - s2))


def _loss(U, Sg, V, gU, gS, gV):
    return (gU * U).sum(0) + (gV * V).sum(0) + (gS * Sg).sum(0)


def test_autograd_vs_finite_differences():
    g = inputs.grad_batch(8192, seed=83)
    keep = ~g["small_gap"]
    A = np.ascontiguousarray(g["A"][:, keep])
    gU, gV, gS = (_dev(np.ascontiguousarray(x[:, keep])) for x in (g["gU"], g["gV"], g["gS"]))
    Ad = _dev(A).requires_grad_(True)
    U, Sg, V = AG.svd2(Ad)
    _loss(U, Sg, V, gU, gS, gV).sum().backward()
    grad = Ad.grad.cpu().numpy()
    h = 1e-6
    piv0 = oracle.svd2(A)["piv"]
    same = np.ones(A.shape[1], bool)
    fd = np.empty_like(A)
    with torch.no_grad():
        for e in range(4):
            Lpm = []
            for sgn in (1, -1):
                Ap = A.copy()
                Ap[e] += sgn * h
                same &= oracle.svd2(Ap)["piv"] == piv0
                Up, Sp, Vp = AG.svd2(_dev(Ap))
                Lpm.append(_loss(Up, Sp, Vp, gU, gS, gV).cpu().numpy())
            fd[e] = (Lpm[0] - Lpm[1]) / (2 * h)
    s = Sg.detach().cpu().numpy()
    gap = (s[0] - s[1]) / s[0]
    err = np.abs(fd - grad).max(axis=0) / (np.abs(grad).max(axis=0) + 1)
    tol = 1e-7 + 1e-10 / gap**2
    assert same.mean() > 0.95
    assert np.all(err[same] <= tol[same]), float((err[same] / tol[same]).max())


def test_autograd_vs_binary128_reference_all_gaps():
    g = inputs.grad_batch(2**17, seed=84)
    A, gU, gV, gS = g["A"], g["gU"], g["gV"], g["gS"]
    dl = S.default_rel_delta(torch.float64)
    Ad = _dev(A).requires_grad_(True)
    U, Sg, V = AG.svd2(Ad, dl)
    _loss(U, Sg, V, _dev(gU), _dev(gS), _dev(gV)).sum().backward()
    hi, lo = oracle.refgrad(A, gU, gV, gS[0], gS[1], dl)
    s = Sg.detach().cpu().numpy()
    gap = (s[0] - s[1]) / s[0]
    err = np.abs((Ad.grad.cpu().numpy() - hi) - lo).max(axis=0) / _natural(hi, gU, gV, s[0], s[1])
    assert np.all(err <= 16 * EPS64 / gap), float((err * gap / EPS64).max())
    assert g["small_gap"].sum() > 10000


def test_fp32_gradient_against_fp64():
    g = inputs.grad_batch(2**17, seed=85)
    A32 = g["A"].astype(np.float32)
    gU, gV, gS = (x.astype(np.float32) for x in (g["gU"], g["gV"], g["gS"]))
    grads = {}
    same_piv = oracle.svd2(A32)["piv"] == oracle.svd2(A32.astype(np.float64))["piv"]
    for tdt in (torch.float32, torch.float64):
        Ad = _dev(A32, tdt).requires_grad_(True)
        U, Sg, V = AG.svd2(Ad, S.default_rel_delta(torch.float32))
        _loss(U, Sg, V, _dev(gU, tdt), _dev(gS, tdt), _dev(gV, tdt)).sum().backward()
        grads[tdt] = Ad.grad.double().cpu().numpy()
        if tdt == torch.float64:
            s = Sg.detach().cpu().numpy()
    gap = (s[0] - s[1]) / s[0]
    m = (gap >= 1e-2) & same_piv
    err = np.abs(grads[torch.float32] - grads[torch.float64]).max(axis=0) / \
        _natural(grads[torch.float64], gU, gV, s[0], s[1])
    assert m.mean() > 0.5
    assert np.all(err[m] <= 16 * EPS32 / gap[m]), float((err[m] * gap[m] / EPS32).max())


def test_gradcheck_small():
    """torch.autograd.gradcheck on matrices whose gap is >= 1e-2 and whose pivot
    choices do not change under any +-1e-5 perturbation of one entry."""
    g = inputs.grad_batch(256, seed=86)
    A = g["A"]
    r = oracle.svd2(A, backscale=True)
    keep = (r["smax"] - r["smin"]) >= 1e-2 * r["smax"]
    for e in range(4):
        for sgn in (1, -1):
            Ap = A.copy()
            Ap[e] += sgn * 1e-5
            keep &= oracle.svd2(Ap)["piv"] == r["piv"]
    Ad = _dev(A[:, keep][:, :16]).requires_grad_(True)
    assert Ad.shape[1] == 16
    assert torch.autograd.gradcheck(lambda a: AG.svd2(a), (Ad,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_full_size_gradient_workload_sampled():
    """n = 2^22, forward + backward on the GPU; 2^14 sampled matrices against the
    oracle's adjoint (bit for bit) and the binary128 reference gradient."""
    g = inputs.grad_batch(2**22)
    A, gU, gV, gS = g["A"], g["gU"], g["gV"], g["gS"]
    dl = S.default_rel_delta(torch.float64)
    Ad = _dev(A).requires_grad_(True)
    U, Sg, V = AG.svd2(Ad, dl)
    _loss(U, Sg, V, _dev(gU), _dev(gS), _dev(gV)).sum().backward()
    idx = np.sort(np.random.default_rng(3).choice(A.shape[1], 2**14, replace=False))
    it = torch.from_numpy(idx).cuda()
    grad = Ad.grad.index_select(1, it).cpu().numpy()
    Us = U.detach().index_select(1, it).cpu().numpy()
    Vs = V.detach().index_select(1, it).cpu().numpy()
    Ss = Sg.detach().index_select(1, it).cpu().numpy()
    o = oracle.bwd(Us, Vs, Ss[0], Ss[1], gU[:, idx], gV[:, idx], gS[0, idx], gS[1, idx], dl)
    assert bits_equal(grad, o)
    hi, lo = oracle.refgrad(np.ascontiguousarray(A[:, idx]), np.ascontiguousarray(gU[:, idx]),
                            np.ascontiguousarray(gV[:, idx]), gS[0, idx], gS[1, idx], dl)
    gap = (Ss[0] - Ss[1]) / Ss[0]
    err = np.abs((grad - hi) - lo).max(axis=0) / _natural(hi, gU[:, idx], gV[:, idx], Ss[0], Ss[1])
    assert np.all(err <= 16 * EPS64 / gap), float((err * gap / EPS64).max())


def test_bwd_fp64_across_the_exponent_range():
    """Upstream gradients from subnormal to 2^300, with zeros, on matrices
    scaled by 2^-300, 1 or 2^300: in FP64 the adjoint's products run on the
    integer pipe, whose domain is normal operands with a normal product, and a
    matrix with a product outside it is read again and done with the hardware
    multiply.  Bit for bit against the oracle's adjoint (every value finite)."""
    n = 4099
    g = inputs.grad_batch(n, seed=91)
    rng = np.random.default_rng(92)
    A = np.ascontiguousarray(g["A"] * np.ldexp(1.0, rng.choice([-300, 0, 300], size=n)))

    def grad(*shape):
        x = rng.standard_normal(shape) * np.ldexp(1.0, rng.choice([-1070, -1040, -600, 0, 300],
                                                                  size=shape))
        x[rng.random(shape) < 0.05] = 0.0
        return x

    gU, gV, gS = grad(4, n), grad(4, n), grad(2, n)
    r = S.svd2(_dev(A), backscale=True)
    dl = S.default_rel_delta(torch.float64)
    gA = S.svd2_bwd(r.U, r.V, r.smax, r.smin, _dev(gU), _dev(gV), _dev(gS[0]), _dev(gS[1]), dl)
    torch.cuda.synchronize()
    with np.errstate(all="ignore"):
        o = oracle.bwd(r.U.cpu().numpy(), r.V.cpu().numpy(), r.smax.cpu().numpy(),
                       r.smin.cpu().numpy(), gU, gV, gS[0], gS[1], dl)
    assert np.isfinite(o).all()
    assert bits_equal(gA.cpu().numpy(), o)
