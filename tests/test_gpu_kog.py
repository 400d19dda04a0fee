"""One parallel Kogbetliantz step on the GPU (svd2_kog_step_*) against the
step oracle (Sec. 1):

- the pivot blocks hold the oracle's Sigma bit for bit, with exact zeros at
  the off-diagonal pivot positions;
- every other entry equals the oracle's U^* G V within 32 eps (|U|^T |G| |V|)
  -- the two sides sum the same products in different orders;
- the result does not depend on the layout (row-major or column-major);
- skipped pairs (an index out of range, or p = q) are counted and leave their
  rows and columns untouched;
- round-robin sweeps on the GPU diagonalize G to its singular values.
"""
import numpy as np
import pytest
import torch

from oracle import kogbetliantz as K
from paper_2005_07403_gb300 import inputs
from tests.helpers import bits_equal

pytestmark = pytest.mark.gpu

DT = {("d", False): (np.float64, torch.float64), ("d", True): (np.complex128, torch.complex128),
      ("s", False): (np.float32, torch.float32), ("s", True): (np.complex64, torch.complex64)}


def _rand(m, cplx, prec, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, m))
    if cplx:
        G = G + 1j * rng.standard_normal((m, m))
    return G.astype(DT[(prec, cplx)][0])


def _gpu(G, pairs, layout):
    """Run one step on a copy of G in the given layout; returns the numpy result."""
    from paper_2005_07403_gb300 import svd2 as S
    if layout == "row":
        Gt = torch.from_numpy(np.ascontiguousarray(G)).cuda()
    else:   # column-major storage of the same matrix
        Gt = torch.from_numpy(np.ascontiguousarray(G.T)).cuda().T
    P = torch.from_numpy(np.asarray(pairs, dtype=np.int32)).cuda()
    ws = S.kog_workspace(Gt)
    S.kog_step(Gt, P, workspace=ws)
    torch.cuda.synchronize()
    return Gt.cpu().numpy(), S.kog_skipped(ws)


def _check(G, pairs, Gp, prec):
    eps = 2.0**-52 if prec == "d" else 2.0**-23
    O = K.kog_step(G, pairs)
    U, V, smax, smin = K.pivot_svds(G, pairs)
    P = np.asarray(pairs).reshape(-1, 2)
    for k, (p, q) in enumerate(P):
        assert bits_equal(np.array([Gp[p, p], Gp[q, q]]), np.array([O[p, p], O[q, q]]).astype(Gp.dtype))
        assert Gp[p, q] == 0 and Gp[q, p] == 0
    Uf, Vf = K.embedded_unitaries(G.shape[0], pairs, U, V)
    bound = 32 * eps * (np.abs(Uf).T @ np.abs(G) @ np.abs(Vf)) + np.finfo(Gp.real.dtype).tiny
    assert np.all(np.abs(Gp - O) <= bound), float((np.abs(Gp - O) / bound).max())


@pytest.mark.parametrize("prec", ["d", "s"])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m", [2, 4, 10, 64, 258])
def test_step_matches_oracle_both_layouts(m, cplx, prec):
    G = _rand(m, cplx, prec, 500 + m)
    pairs = np.random.default_rng(600 + m).permutation(m).astype(np.int32)
    out = {}
    for layout in ("row", "col"):
        Gp, skipped = _gpu(G, pairs, layout)
        assert skipped == 0
        _check(G, pairs, Gp, prec)
        out[layout] = Gp
    assert bits_equal(out["row"], out["col"])


@pytest.mark.parametrize("cplx", [False, True])
def test_adjacent_pairs_large(cplx):
    """m = 2050 with the pairs (2i, 2i+1), the coalesced case."""
    m = 2050
    G = _rand(m, cplx, "d", 700)
    pairs = np.arange(m, dtype=np.int32)
    Gp, _ = _gpu(G, pairs, "col")
    _check(G, pairs, Gp, "d")


def test_invalid_pairs_are_skipped():
    m = 8
    G = _rand(m, False, "d", 800)
    pairs = np.array([0, 1, 2, 9, 4, 5, 6, 6], dtype=np.int32)   # (2, 9) out of range, (6, 6)
    Gp, skipped = _gpu(G, pairs, "row")
    assert skipped == 2
    bad = np.array([2, 3, 6, 7])   # indices of skipped pairs, or of none
    sub = np.array([0, 1, 4, 5])   # the valid pairs (0, 1), (4, 5)
    # every block in a row or a column of a skipped pair is untouched ...
    assert np.array_equal(Gp[bad, :], G[bad, :])
    assert np.array_equal(Gp[:, bad], G[:, bad])
    # ... and the blocks among valid pairs are the step on that submatrix
    O = K.kog_step(G[np.ix_(sub, sub)], [0, 1, 2, 3])
    assert np.allclose(Gp[np.ix_(sub, sub)], O, rtol=0, atol=64 * 2.0**-52 * np.abs(G).max())


@pytest.mark.parametrize("cplx", [False, True])
def test_gpu_sweeps_diagonalize(cplx):
    from paper_2005_07403_gb300 import svd2 as S
    m = 64
    G = _rand(m, cplx, "d", 900)
    s0 = np.linalg.svd(G, compute_uv=False)
    Gt = torch.from_numpy(np.ascontiguousarray(G)).cuda()
    ws = S.kog_workspace(Gt)
    pairs = [torch.from_numpy(inputs.round_robin_pairs(m, st)).cuda() for st in range(m - 1)]
    off0 = K.off_norm(G)
    Go = G.copy()
    for sweep in range(16):       # the oracle needs 12 sweeps at m = 64 to reach 1e-12
        for st, P in enumerate(pairs):
            S.kog_step(Gt, P, workspace=ws)
            if sweep < 4:
                Go = K.kog_step(Go, inputs.round_robin_pairs(m, st))
        if sweep == 3:            # same trajectory as the oracle while far from convergence
            ratio = K.off_norm(Gt.cpu().numpy()) / K.off_norm(Go)
            assert 0.99 < ratio < 1.01, ratio
    Gf = Gt.cpu().numpy()
    assert K.off_norm(Gf) < 1e-12 * off0
    d = np.sort(np.abs(np.diag(Gf)))[::-1]
    assert np.allclose(d, s0, rtol=0, atol=1e-12 * s0[0])


@pytest.mark.parametrize("cplx", [False, True])
def test_entries_across_the_exponent_range(cplx):
    """Entries of G from subnormal to 2^1000, with exact zeros: in complex
    double the update's leading products run on the integer pipe, whose domain
    is normal operands with a normal product. Blocks with a zero, a subnormal or
    an underflowing product are read again and done with the hardware
    multiply. Checked against the oracle in both layouts, and the two layouts
    give the same bits."""
    m = 66
    rng = np.random.default_rng(1000 + cplx)
    scale = np.ldexp(1.0, rng.choice([-1070, -1040, -1000, 0, 600, 1000], size=(m, m)))
    G = rng.standard_normal((m, m)) * scale
    if cplx:
        G = G + 1j * rng.standard_normal((m, m)) * np.ldexp(1.0, rng.choice([-1060, 0, 900],
                                                                            size=(m, m)))
    G[rng.random((m, m)) < 0.05] = 0
    pairs = rng.permutation(m).astype(np.int32)
    out = {}
    with np.errstate(all="ignore"):
        for layout in ("row", "col"):
            Gp, skipped = _gpu(G, pairs, layout)
            assert skipped == 0
            _check(G, pairs, Gp, "d")
            out[layout] = Gp
    assert bits_equal(out["row"], out["col"])
