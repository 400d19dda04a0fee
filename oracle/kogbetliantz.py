"""Oracle of one parallel step of the Kogbetliantz method (Sec. 1).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the bench's CPU
baseline; it shares no code with the CUDA path.

Sec. 1: the iteration matrix G of order m = 2n is processed in parallel
steps.  A step takes n disjoint pivot pairs (p_k, q_k) -- together a
permutation of 0 .. m-1 -- assembles A^[k] column by column from the
elements of G at (p_k, p_k), (q_k, p_k), (p_k, q_k), (q_k, q_k), computes
A^[k] = U^[k] Sigma^[k] (V^[k])^*, and updates G from the left by
(U^[k])^* (rows p_k, q_k) and from the right by V^[k] (columns p_k, q_k),
annihilating the off-diagonal pivot positions.  The rows p_k, q_k and the
columns p_j, q_j of G meet in a 2x2 block, so the updated matrix is, block by
block,

    G'[{p_k, q_k}, {p_j, q_j}] = (U^[k])^* G[{p_k, q_k}, {p_j, q_j}] V^[j],

and for j = k the block is Sigma^[k] (the off-diagonal pivot positions
become exact zeros).  The 2x2 SVDs are the C oracle's method (Sec. 2) with
the back-scaling of Fig. 1, so Sigma^[k] holds the true singular values.
"""
from __future__ import annotations

import numpy as np

from . import svd2 as _svd2


def _split(blocks):
    """(n, 2, 2) pivot blocks -> split layout of Sec. 3 (record order of Sec. 8)."""
    els = [blocks[:, 0, 0], blocks[:, 1, 0], blocks[:, 0, 1], blocks[:, 1, 1]]
    if np.iscomplexobj(blocks):
        rows = [p for e in els for p in (e.real, e.imag)]
    else:
        rows = els
    return np.ascontiguousarray(np.stack(rows))


def _unsplit(X, complex_dtype):
    """Split layout (4 or 8, n) -> (n, 2, 2) matrices [[x11, x12], [x21, x22]],
    every bit kept (complex values written through a real view)."""
    pos = [(0, 0), (1, 0), (0, 1), (1, 1)]          # x11, x21, x12, x22
    n = X.shape[1]
    if X.shape[0] == 8:
        R = np.empty((n, 2, 2, 2), dtype=X.dtype)   # last axis: (Re, Im)
        for e, (i, j) in enumerate(pos):
            R[:, i, j, 0] = X[2 * e]
            R[:, i, j, 1] = X[2 * e + 1]
        return R.view(complex_dtype)[..., 0]
    out = np.empty((n, 2, 2), dtype=X.dtype)
    for e, (i, j) in enumerate(pos):
        out[:, i, j] = X[e]
    return out


def pivot_svds(G, pairs):
    """The batch of Sec. 1 for one step: (U (n,2,2), V (n,2,2), smax, smin)
    of the pivot blocks A^[k] of G (the method, back-scaled)."""
    P = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    p, q = P[:, 0], P[:, 1]
    blocks = np.empty((len(P), 2, 2), dtype=G.dtype)
    blocks[:, 0, 0], blocks[:, 1, 0] = G[p, p], G[q, p]
    blocks[:, 0, 1], blocks[:, 1, 1] = G[p, q], G[q, q]
    with np.errstate(all="ignore"):
        r = _svd2(_split(blocks), backscale=True)
    cdt = G.dtype if np.iscomplexobj(G) else None
    return _unsplit(r["U"], cdt), _unsplit(r["V"], cdt), r["smax"], r["smin"]


def kog_step(G, pairs):
    """One parallel step (Sec. 1) on a copy of G (m x m, real or complex);
    returns the updated matrix."""
    G = np.asarray(G)
    m = G.shape[0]
    P = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    assert G.shape == (m, m) and m % 2 == 0 and len(P) == m // 2
    assert np.array_equal(np.sort(P.ravel()), np.arange(m)), "pairs must be a permutation"
    U, V, smax, smin = pivot_svds(G, P)
    Uh = np.conj(np.swapaxes(U, 1, 2))
    # B[k, a, j, b] = G[P[k, a], P[j, b]]
    B = G[P[:, :, None, None], P[None, None, :, :]]
    out = np.einsum("kxa,kajb,jby->kxjy", Uh, B, V)
    n = len(P)
    idx = np.arange(n)
    out[idx, :, idx, :] = 0
    out[idx, 0, idx, 0] = smax
    out[idx, 1, idx, 1] = smin
    Gp = np.empty_like(G)
    Gp[P[:, :, None, None], P[None, None, :, :]] = out
    return Gp


def embedded_unitaries(m, pairs, U, V):
    """The m x m unitaries of one step: U^[k] placed at rows/columns p_k, q_k."""
    P = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    Uf = np.zeros((m, m), dtype=U.dtype)
    Vf = np.zeros((m, m), dtype=V.dtype)
    for k, (p, q) in enumerate(P):
        Uf[np.ix_([p, q], [p, q])] = U[k]
        Vf[np.ix_([p, q], [p, q])] = V[k]
    return Uf, Vf


def off_norm(G):
    """Frobenius norm of the off-diagonal part."""
    return float(np.linalg.norm(G - np.diag(np.diag(G))))
