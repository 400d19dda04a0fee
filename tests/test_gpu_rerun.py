"""FP32 form with FP64 re-run against the oracle's re-run form (same flag
decision in float, same double method, same rounding to float), bit for bit;
the re-run count against the oracle's; and the stated error of the form
against the double oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.helpers import bits_equal
from tests.test_gpu_fwd import assert_same, sprinkled

pytestmark = pytest.mark.gpu


def run(A, tau, backscale=False):
    Ad = torch.from_numpy(A).cuda()
    r = S.svd2_rerun(Ad, tau_log2=tau, backscale=backscale)
    torch.cuda.synchronize()
    g = {k: getattr(r, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}
    return g, S.rerun_count(r.workspace)


@pytest.mark.parametrize("tau", [-8, -4, -20])
def test_rerun_real_matches_oracle(tau):
    A32, _ = inputs.real_fp32_illcond(2**17 + 11)
    g, cnt = run(A32, tau)
    o = oracle.svd2_rerun(A32, tau)
    assert_same(g, o, f"s_rerun tau={tau}")
    assert cnt == o["count"] > 0


def test_rerun_complex_matches_oracle():
    A = inputs.normal_batch(2**16 + 7, 8, 61, np.float32)
    g, cnt = run(A, -6)
    o = oracle.svd2_rerun(A, -6)
    assert_same(g, o, "c_rerun")
    assert cnt == o["count"] > 0


def test_rerun_complex_illcond_matches_oracle():
    A, _ = inputs.complex_fp32_illcond(2**16 + 13, seed=64)
    g, cnt = run(A, -8)
    o = oracle.svd2_rerun(A, -8)
    assert_same(g, o, "c_rerun ill-conditioned")
    assert cnt == o["count"] > 2**16 // 20


def test_rerun_edge_and_backscale():
    A = np.ascontiguousarray(np.concatenate([inputs.edge_real(np.float32),
                                             inputs.random_bits_f32(4096, 4, 62)], axis=1))
    for bs in (False, True):
        g, cnt = run(A, -8, backscale=bs)
        with np.errstate(all="ignore"):
            o = oracle.svd2_rerun(A, -8, backscale=bs)
        assert_same(g, o, f"rerun edge bs={bs}")
        assert cnt == o["count"]


def test_rerun_nothing_flagged_equals_plain_fp32():
    A = inputs.normal_batch(10000, 4, 63, np.float32)
    g, cnt = run(A, -100)
    r = S.svd2(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    assert cnt == 0
    assert bits_equal(g["U"], r.U.cpu().numpy()) and bits_equal(g["smin"], r.smin.cpu().numpy())


def test_rerun_stated_error_full_size_sampled():
    """FP32 vs FP64 workload at n = 2^26: every sampled matrix's sigma'_max within
    8 u of the double method, sigma'_min within 64 u for kept matrices
    (u = 2^-24; measured on the oracle: <= 6.3 u and <= 47 u at tau = 2^-8)
    and within 1 u + the double method's own error for re-run ones."""
    A32, ill = inputs.real_fp32_illcond(2**26)
    Ad = torch.from_numpy(A32).cuda()
    r = S.svd2_rerun(Ad)
    torch.cuda.synchronize()
    cnt = S.rerun_count(r.workspace)
    idx = np.sort(np.random.default_rng(5).choice(A32.shape[1], 1 << 16, replace=False))
    it = torch.from_numpy(idx).cuda()
    sx = r.smax.index_select(0, it).cpu().numpy().astype(np.float64)
    sn = r.smin.index_select(0, it).cpu().numpy().astype(np.float64)
    s = r.s.index_select(0, it).cpu().numpy()
    Asub = np.ascontiguousarray(A32[:, idx].astype(np.float64))
    o64 = oracle.svd2(Asub, backscale=True)
    u = 2.0**-24
    bx = np.ldexp(sx, -s)
    bn = np.ldexp(sn, -s)
    ex = np.abs(bx - o64["smax"]) / o64["smax"]
    assert ex.max() <= 8 * u
    keep = sn >= 2.0**-8 * sx
    en = np.abs(bn - o64["smin"]) / np.where(o64["smin"] > 0, o64["smin"], 1)
    assert en[keep].max() <= 64 * u
    assert en[~keep].max() <= 1.001 * u
    frac = cnt / A32.shape[1]
    assert 0.09 < frac < 0.12, frac


@pytest.mark.parametrize("rows", [4, 8])
def test_rerun_fixup_pass_scattered_edges(rows):
    """Edge matrices among ordinary ones: those the fast single-precision pass
    flags are finished by the fix-up pass (general single-precision method,
    then the re-run test and the double re-run); results, s and the re-run
    count equal the oracle's."""
    A = sprinkled(2**17 + 9, rows, np.float32, 81 + rows, every=499)
    for bs in (False, True):
        g, cnt = run(A, -8, backscale=bs)
        with np.errstate(all="ignore"):
            o = oracle.svd2_rerun(A, -8, backscale=bs)
        assert_same(g, o, f"rerun fixup rows={rows} bs={bs}")
        assert cnt == o["count"]
        assert not np.isin(g["s"], [np.iinfo(np.int32).min, np.iinfo(np.int32).min + 1]).any()


def _shape_sweep_input(rows, n):
    if rows == 4:
        return inputs.real_fp32_illcond(n, seed=71)[0]
    return inputs.complex_fp32_illcond(n, seed=72)[0]


@pytest.mark.parametrize("rows", [4, 8])
def test_rerun_every_matrix_marked(rows):
    """tau = 2^0: every matrix with sigma'_min < sigma'_max is re-run (the
    index list holds the whole batch); bits and count as the oracle's, in the
    default launch shape of the batch pass and two others."""
    n = 2**15 + 17
    A = inputs.normal_batch(n, rows, 73 + rows, np.float32)
    o = oracle.svd2_rerun(A, 0)
    assert o["count"] > n - 16
    kind = "s" if rows == 4 else "c"
    old = S.get_launch(kind)
    try:
        for shape in (old, (64, 4, 2, 0), (512, 1, 1, 4)):
            S.set_launch(kind, *shape)
            g, cnt = run(A, 0)
            assert_same(g, o, f"{kind} all marked {shape}")
            assert cnt == o["count"]
    finally:
        S.set_launch(kind, *old)


@pytest.mark.parametrize("rows", [4, 8])
def test_rerun_misaligned_rows_and_guard_bands(rows):
    """Rows that start 4 bytes off a 16-byte boundary take one matrix per
    thread; canaries around every output array stay untouched by all four
    kernels (the batch pass, the compaction, the scattered re-run stores and
    the fix-up pass)."""
    n, pad = 30011, 64
    A = _shape_sweep_input(rows, n + 1)
    Ad = torch.from_numpy(A).cuda()[:, 1:]
    o = oracle.svd2_rerun(np.ascontiguousarray(A[:, 1:]), -8)
    canary = float.fromhex("0x1.dead0p+7")
    bufs = [torch.full((rows, n + 1 + pad), canary, dtype=torch.float32, device="cuda")
            for _ in range(2)]
    sb = [torch.full((n + 1 + pad,), canary, dtype=torch.float32, device="cuda") for _ in range(2)]
    si = torch.full((n + 1 + pad,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    out = S.Svd2Result(U=bufs[0][:, 1:n + 1], V=bufs[1][:, 1:n + 1], smax=sb[0][1:n + 1],
                       smin=sb[1][1:n + 1], s=si[1:n + 1])
    r = S.svd2_rerun(Ad, tau_log2=-8, out=out)
    torch.cuda.synchronize()
    g = {k: getattr(r, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}
    assert_same(g, o, f"rows={rows} misaligned")
    assert S.rerun_count(r.workspace) == o["count"]
    for b in bufs:
        assert torch.all(b[:, 0] == canary) and torch.all(b[:, n + 1:] == canary)
    for b in sb:
        assert b[0] == canary and torch.all(b[n + 1:] == canary)
    assert si[0] == 0x5A5A5A5A and torch.all(si[n + 1:] == 0x5A5A5A5A)
