"""Pins of the oracle's complex adjoint (the derivative of A = U Sigma V^*):

- on real data it is the real adjoint (the complex formulas reduce to it);
- central differences of the oracle's forward method on a loss that is
  invariant under the phase gauge U, V -> U D, V D (|U|^2 and |V|^2 weights,
  singular values, the rank-one terms u_i v_i^*), in all 8 real directions of
  each matrix, on matrices whose pivot choices stay fixed and whose singular
  values are apart;
- a planted sign error in the gauge term, or a conjugation error on one
  element, fails the differences.
"""
import numpy as np
import pytest

import oracle
from paper_2005_07403_gb300 import inputs

EPS = 2.0**-52


def _cplx(X):
    """Split rows (8, n) -> complex (4, n) in the record order x11, x21, x12, x22."""
    return X[0::2] + 1j * X[1::2]


def _split(Z):
    out = np.empty((8, Z.shape[1]))
    out[0::2], out[1::2] = Z.real, Z.imag
    return out


def _loss_and_grads(U8, V8, s1, s2, W):
    """Gauge-invariant loss per matrix and its upstream gradients (dL/dRe + i dL/dIm)."""
    U, V = _cplx(U8), _cplx(V8)
    W2, W3, w1, w2, W4, W5 = W
    u1, u2 = U[[0, 1]], U[[2, 3]]          # columns of U: (x11, x21), (x12, x22)
    v1, v2 = V[[0, 1]], V[[2, 3]]
    L = (W2 * np.abs(U) ** 2).sum(0) + (W3 * np.abs(V) ** 2).sum(0) + w1 * s1 + w2 * s2
    # Re sum_ij conj(W4_ij) u1_i conj(v1_j), W4 as (2, 2, n) [i, j]
    L = L + np.real(np.einsum("ijn,in,jn->n", np.conj(W4), u1, np.conj(v1)))
    L = L + np.real(np.einsum("ijn,in,jn->n", np.conj(W5), u2, np.conj(v2)))
    gU = 2 * W2 * U
    gV = 2 * W3 * V
    gU[[0, 1]] += np.einsum("ijn,jn->in", W4, v1)
    gV[[0, 1]] += np.einsum("ijn,in->jn", np.conj(W4), u1)
    gU[[2, 3]] += np.einsum("ijn,jn->in", W5, v2)
    gV[[2, 3]] += np.einsum("ijn,in->jn", np.conj(W5), u2)
    return L, _split(gU), _split(gV), w1, w2


def _weights(n, seed):
    rng = np.random.default_rng(seed)
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    return (rng.standard_normal((4, n)), rng.standard_normal((4, n)), rng.standard_normal(n),
            rng.standard_normal(n), c(2, 2, n), c(2, 2, n))


def _forward(A):
    r = oracle.svd2(A, backscale=True)
    return r["U"], r["V"], r["smax"], r["smin"], r["piv"]


def test_real_data_gives_the_real_adjoint():
    rng = np.random.default_rng(1)
    n = 4096
    A = inputs.normal_batch(n, 4, 2)
    r = oracle.svd2(A, backscale=True)
    gU, gV, gS = rng.standard_normal((4, n)), rng.standard_normal((4, n)), rng.standard_normal((2, n))
    dl = 64 * EPS
    real = oracle.bwd(r["U"], r["V"], r["smax"], r["smin"], gU, gV, gS[0], gS[1], dl)
    z = lambda X: _split(X.astype(complex))
    cplx = oracle.bwd(z(r["U"]), z(r["V"]), r["smax"], r["smin"], z(gU), z(gV), gS[0], gS[1], dl)
    assert np.array_equal(cplx[0::2], real)
    assert np.array_equal(cplx[1::2], np.zeros_like(real))


def _fd_check(bwd, n=3000, h=1e-6, seed=3):
    A = inputs.normal_batch(n, 8, seed)
    U, V, s1, s2, piv = _forward(A)
    gap = (s1 - s2) / s1
    W = _weights(n, seed + 1)
    L0, gU, gV, g1, g2 = _loss_and_grads(U, V, s1, s2, W)
    gA = bwd(U, V, s1, s2, gU, gV, g1, g2, 64 * EPS)
    same = np.ones(n, bool)
    fd = np.empty_like(A)
    for e in range(8):
        Lpm = []
        for sg in (1, -1):
            Ap = A.copy()
            Ap[e] += sg * h
            Up, Vp, s1p, s2p, pivp = _forward(Ap)
            same &= pivp == piv
            Lpm.append(_loss_and_grads(Up, Vp, s1p, s2p, W)[0])
        fd[e] = (Lpm[0] - Lpm[1]) / (2 * h)
    keep = same & (gap > 1e-3)
    err = np.abs(fd - gA).max(axis=0) / (np.abs(gA).max(axis=0) + 1)
    # the truncation error of the central difference grows like h^2 / c^2 with
    # c = min(relative gap, s2/s1): the singular vectors turn like 1/gap, and the
    # phase of the second pair (the gauge term) like 1/s2
    c = np.minimum(gap, s2 / s1)
    tol = 1e-7 + 1e-10 / c**2
    return keep, err, tol


def test_central_differences_of_gauge_invariant_loss():
    keep, err, tol = _fd_check(oracle.bwd)
    assert keep.mean() > 0.9
    assert np.all(err[keep] <= tol[keep]), float((err[keep] / tol[keep]).max())


@pytest.mark.parametrize("mutation", ["gauge sign", "conjugated element"])
def test_planted_mistakes_fail_the_differences(mutation):
    """The oracle's result with one plausible mistake: the gauge terms t_i
    negated (the result corrected by -2 U diag(i t) V^*), or one element of gU
    conjugated on its way into J (the result of the correct formula on that
    input)."""
    def bad(U, V, s1, s2, gU, gV, g1, g2, dl):
        good = oracle.bwd(U, V, s1, s2, gU, gV, g1, g2, dl)
        if mutation == "gauge sign":
            # t_i -> -t_i: add -2 U diag(i t) V^* to the result
            Uc, Vc, gUc, gVc = _cplx(U), _cplx(V), _cplx(gU), _cplx(gV)
            t = []
            for i, cols in enumerate(([0, 1], [2, 3])):
                Jii = np.sum(np.conj(Uc[cols]) * gUc[cols], 0)
                Kii = np.sum(np.conj(Vc[cols]) * gVc[cols], 0)
                t.append(0.5 * (Jii.imag - Kii.imag) / (s1 if i == 0 else s2))
            Z = _cplx(good)
            for i, cols in enumerate(([0, 1], [2, 3])):
                ui = Uc[cols]                      # column i of U
                vi = Vc[cols]
                outer = np.einsum("an,bn->abn", ui, np.conj(vi))   # u_i v_i^*
                delta = -2j * t[i] * outer        # -2 U (i t_i e_i e_i^T) V^*
                Z[0] += delta[0, 0]; Z[1] += delta[1, 0]; Z[2] += delta[0, 1]; Z[3] += delta[1, 1]
            return _split(Z)
        gU2 = gU.copy()
        gU2[1] = -gU2[1]          # the element x11 of gU conjugated
        return oracle.bwd(U, V, s1, s2, gU2, gV, g1, g2, dl)
    keep, err, tol = _fd_check(bad, n=600)
    assert not np.all(err[keep] <= tol[keep])
