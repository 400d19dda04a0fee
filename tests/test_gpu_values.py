"""Singular-values-only forms (svd2_values_*) and the interleaved (n, 2, 2)
layout (svd2_batch_interleaved_*), bit for bit against the oracle.

- values only: sigma' and s equal the oracle's (and the full form's) for all
  four forms, ordinary and edge matrices, with and without back-scaling;
- interleaved: U, V, sigma' and s of a (n, 2, 2) real or complex batch equal
  the oracle's on the same matrices re-laid in the split layout; the
  values-only variant of the interleaved call likewise.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.helpers import bits_equal
from tests.test_gpu_fwd import sprinkled

pytestmark = pytest.mark.gpu

INT32_MIN = np.iinfo(np.int32).min


def _batch(rows, dtype, n, seed):
    if dtype == np.float32:
        return sprinkled(n, rows, np.float32, seed)
    A = inputs.normal_batch(n, rows, seed, np.float64)
    E = inputs.edge_real(np.float64)
    if rows == 4:
        A[:, :E.shape[1]] = E
    else:
        A[0::2, :E.shape[1]] = E
        A[1::2, :E.shape[1]] = np.roll(E, 3, axis=1)
    return np.ascontiguousarray(A)


@pytest.mark.parametrize("rows,dtype", [(4, np.float64), (8, np.float64),
                                        (4, np.float32), (8, np.float32)])
@pytest.mark.parametrize("backscale", [False, True])
def test_values_only_matches_oracle(rows, dtype, backscale):
    A = _batch(rows, dtype, 2**17 + 7, 101 + rows)
    r = S.svd2_values(torch.from_numpy(A).cuda(), backscale=backscale)
    torch.cuda.synchronize()
    with np.errstate(all="ignore"):
        o = oracle.svd2(A, backscale=backscale)
    assert bits_equal(r.smax.cpu().numpy(), o["smax"])
    assert bits_equal(r.smin.cpu().numpy(), o["smin"])
    s = r.s.cpu().numpy()
    assert np.array_equal(s, o["s"])
    assert not np.isin(s, [INT32_MIN, INT32_MIN + 1]).any()


def _to_interleaved(A):
    """Split layout (4 or 8, n) -> (n, 2, 2) real or complex, row-major entries,
    every bit kept (complex values are written through a real view, so signed
    zeros survive)."""
    rows, n = A.shape
    pos = [(0, 0), (1, 0), (0, 1), (1, 1)]         # a11, a21, a12, a22
    if rows == 4:
        M = np.empty((n, 2, 2), dtype=A.dtype)
        for e, (i, j) in enumerate(pos):
            M[:, i, j] = A[e]
        return M
    R = np.empty((n, 2, 2, 2), dtype=A.dtype)      # last axis: (Re, Im)
    for e, (i, j) in enumerate(pos):
        R[:, i, j, 0] = A[2 * e]
        R[:, i, j, 1] = A[2 * e + 1]
    cdt = np.complex128 if A.dtype == np.float64 else np.complex64
    return R.view(cdt)[..., 0]


def _to_split(M):
    """(n, 2, 2) -> split layout in the record order of Sec. 8."""
    els = [M[:, 0, 0], M[:, 1, 0], M[:, 0, 1], M[:, 1, 1]]
    if np.iscomplexobj(M):
        return np.ascontiguousarray(np.stack([p for e in els for p in (e.real, e.imag)]))
    return np.ascontiguousarray(np.stack(els))


@pytest.mark.parametrize("rows,dtype", [(4, np.float64), (8, np.float64),
                                        (4, np.float32), (8, np.float32)])
def test_interleaved_layout_matches_oracle(rows, dtype):
    A = _batch(rows, dtype, 2**16 + 5, 111 + rows)
    M = _to_interleaved(A)
    assert bits_equal(_to_split(M), A)
    for bs in (False, True):
        r = S.svd2_interleaved(torch.from_numpy(M).cuda(), backscale=bs)
        torch.cuda.synchronize()
        with np.errstate(all="ignore"):
            o = oracle.svd2(A, backscale=bs)
        assert bits_equal(_to_split(r.U.cpu().numpy()), o["U"]), f"U bs={bs}"
        assert bits_equal(_to_split(r.V.cpu().numpy()), o["V"]), f"V bs={bs}"
        assert bits_equal(r.smax.cpu().numpy(), o["smax"])
        assert bits_equal(r.smin.cpu().numpy(), o["smin"])
        assert np.array_equal(r.s.cpu().numpy(), o["s"])
        v = S.svd2_interleaved(torch.from_numpy(M).cuda(), values_only=True, backscale=bs)
        torch.cuda.synchronize()
        assert v.U is None and v.V is None
        assert bits_equal(v.smin.cpu().numpy(), o["smin"])
        assert np.array_equal(v.s.cpu().numpy(), o["s"])


def test_interleaved_reconstructs_torch_matrices():
    """A = U diag(2^-s sigma') V^H on a complex128 (n, 2, 2) torch batch."""
    g = torch.Generator().manual_seed(121)
    M = torch.randn((4096, 2, 2), dtype=torch.complex128, generator=g)
    r = S.svd2_interleaved(M.cuda(), backscale=True)
    U, V = r.U.cpu(), r.V.cpu()
    Sg = torch.diag_embed(torch.stack([r.smax.cpu(), r.smin.cpu()], 1)).to(M.dtype)
    R = U @ Sg @ V.conj().transpose(1, 2)
    err = (R - M).abs().amax(dim=(1, 2)) / M.abs().amax(dim=(1, 2))
    assert float(err.max()) < 8 * 2.0**-52


@pytest.mark.parametrize("rows,dtype", [(4, np.float32), (4, np.float64), (8, np.float32)])
def test_interleaved_unaligned_records_take_the_element_path(rows, dtype):
    """Records whose base is off a 16-byte boundary (one real element, or one
    complex64 element, past it): the kernel reads and writes the interleaved
    layout element by element at its stride (no record vectors); outputs as
    the oracle's."""
    n = 2**15 + 3
    A = _batch(rows, dtype, n, 131 + rows)
    M = np.ascontiguousarray(_to_interleaved(A))
    tdt = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
    off = 2 if rows == 8 else 1                       # scalars before the first record
    flat = torch.zeros(M.size * (2 if rows == 8 else 1) + off, dtype=tdt, device="cuda")
    src = torch.from_numpy(M).cuda()
    flat[off:] = (torch.view_as_real(src) if rows == 8 else src).reshape(-1)
    if rows == 8:
        Mu = torch.view_as_complex(flat[off:].view(n, 2, 2, 2))
    else:
        Mu = flat[off:].view(n, 2, 2)
    assert Mu.data_ptr() % 16 != 0
    r = S.svd2_interleaved(Mu)
    torch.cuda.synchronize()
    with np.errstate(all="ignore"):
        o = oracle.svd2(A)
    assert bits_equal(_to_split(r.U.cpu().numpy()), o["U"])
    assert bits_equal(_to_split(r.V.cpu().numpy()), o["V"])
    assert bits_equal(r.smax.cpu().numpy(), o["smax"])
    assert bits_equal(r.smin.cpu().numpy(), o["smin"])
    assert np.array_equal(r.s.cpu().numpy(), o["s"])
