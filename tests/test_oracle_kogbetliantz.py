"""Pins of the Kogbetliantz-step oracle (Sec. 1) against facts the paper and
the mathematics fix, not against its own formula:

- for m = 2 the step returns diag(sigma_max, sigma_min) of the method;
- on small matrices the blockwise result equals U_full^* G V_full with the
  unitaries embedded at the pivot rows and columns (computed as a product of
  full matrices), for arbitrary pivot pairs -- a transposed or conjugated
  factor, or swapped p/q, fails this;
- the off-diagonal pivot positions are exactly zero afterwards;
- the step is a unitary two-sided transformation: the singular values and the
  Frobenius norm of G are preserved;
- a sweep of round-robin steps drives the off-diagonal norm to zero (the
  method's purpose), and the final diagonal holds the singular values.
"""
import numpy as np
import pytest

import oracle
from oracle import kogbetliantz as K
from paper_2005_07403_gb300 import inputs

EPS = 2.0**-52


def _rand(m, cplx, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, m))
    if cplx:
        G = G + 1j * rng.standard_normal((m, m))
    return G


@pytest.mark.parametrize("cplx", [False, True])
def test_order_two_gives_sigma(cplx):
    G = _rand(2, cplx, 1)
    Gp = K.kog_step(G, [0, 1])
    U, V, smax, smin = K.pivot_svds(G, [0, 1])
    assert Gp[0, 1] == 0 and Gp[1, 0] == 0
    assert Gp[0, 0] == smax[0] and Gp[1, 1] == smin[0]
    sv = np.linalg.svd(G, compute_uv=False)
    assert np.allclose([smax[0], smin[0]], sv, rtol=8 * EPS, atol=0)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m", [4, 6, 10])
def test_blockwise_equals_full_product(m, cplx):
    rng = np.random.default_rng(10 + m)
    G = _rand(m, cplx, 20 + m)
    pairs = rng.permutation(m).astype(np.int32)
    Gp = K.kog_step(G, pairs)
    U, V, smax, smin = K.pivot_svds(G, pairs)
    Uf, Vf = K.embedded_unitaries(m, pairs, U, V)
    F = Uf.conj().T @ G @ Vf
    P = pairs.reshape(-1, 2)
    # pivot blocks: the product is Sigma up to rounding, the step stores Sigma exactly
    for k, (p, q) in enumerate(P):
        assert Gp[p, q] == 0 and Gp[q, p] == 0
        F[p, q] = F[q, p] = 0
    scale = np.abs(Uf).T @ np.abs(G) @ np.abs(Vf)
    assert np.all(np.abs(Gp - F) <= 32 * EPS * scale + 1e-300)


@pytest.mark.parametrize("cplx", [False, True])
def test_step_is_unitary(cplx):
    m = 64
    G = _rand(m, cplx, 31)
    pairs = np.random.default_rng(32).permutation(m).astype(np.int32)
    Gp = K.kog_step(G, pairs)
    s0 = np.linalg.svd(G, compute_uv=False)
    s1 = np.linalg.svd(Gp, compute_uv=False)
    assert np.allclose(s1, s0, rtol=0, atol=64 * EPS * s0[0])
    assert abs(np.linalg.norm(Gp) - np.linalg.norm(G)) <= 64 * EPS * np.linalg.norm(G)


def test_round_robin_ordering_meets_every_pair_once():
    m = 12
    seen = set()
    for step in range(m - 1):
        P = inputs.round_robin_pairs(m, step).reshape(-1, 2)
        assert np.array_equal(np.sort(P.ravel()), np.arange(m))
        seen |= {tuple(sorted(x)) for x in P.tolist()}
    assert len(seen) == m * (m - 1) // 2


@pytest.mark.parametrize("cplx", [False, True])
def test_sweeps_diagonalize(cplx):
    m = 16
    G = _rand(m, cplx, 41)
    s0 = np.linalg.svd(G, compute_uv=False)
    off0 = K.off_norm(G)
    for sweep in range(8):
        for step in range(m - 1):
            G = K.kog_step(G, inputs.round_robin_pairs(m, step))
    assert K.off_norm(G) < 1e-12 * off0
    d = np.sort(np.abs(np.diag(G)))[::-1]
    assert np.allclose(d, s0, rtol=0, atol=1e-12 * s0[0])
