"""Real FP32 form with the FP64 tangent step (svd2_batch_s_tan64) against the
oracle's form of the same definition: bit for bit (U, V, sigma', s) and the
count of matrices that took the step, on the ill-conditioned FP32 workload
with a ragged tail, on every launch shape, on edge matrices handed to the
fix-up pass, through the host-buffer entry point, and on a sample of the
full-size batch (n = 2^26) in the launch configuration the bench times."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.test_gpu_fwd import assert_same, sprinkled

pytestmark = pytest.mark.gpu


def run(A, tau, backscale=False):
    Ad = torch.from_numpy(A).cuda()
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    r = S.svd2_tan64(Ad, tau_log2=tau, backscale=backscale, count=cnt)
    torch.cuda.synchronize()
    g = {k: getattr(r, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}
    return g, int(cnt.item())


@pytest.mark.parametrize("tau", [-4, -8, -1, 0, -30])
def test_tan64_matches_oracle(tau):
    A32, _ = inputs.real_fp32_illcond(2**18 + 37, seed=3301)
    g, cnt = run(A32, tau)
    o = oracle.svd2_tan64(A32, tau)
    assert_same(g, o, f"s_tan64 tau={tau}")
    assert cnt == o["count"] > 0


@pytest.mark.parametrize("mpt,unroll", [(1, 1), (1, 2), (2, 1), (2, 2), (4, 1), (4, 2)])
def test_tan64_every_launch_shape(mpt, unroll):
    A32, _ = inputs.real_fp32_illcond(2**16 + 5, seed=3302)
    o = oracle.svd2_tan64(A32, -4)
    old = S.get_launch("s_tan64")
    try:
        S.set_launch("s_tan64", 256, mpt, unroll, 0)
        g, cnt = run(A32, -4)
        S.set_launch("s_tan64", 1024, mpt, unroll, 4)
        g2, cnt2 = run(A32, -4)
    finally:
        S.set_launch("s_tan64", *old)
    assert_same(g2, o, f"s_tan64 block 1024 mpt={mpt} unroll={unroll}")
    assert cnt2 == o["count"]
    assert_same(g, o, f"s_tan64 mpt={mpt} unroll={unroll}")
    assert cnt == o["count"]


@pytest.mark.parametrize("backscale", [False, True])
def test_tan64_edges_and_fixup(backscale):
    """Edge matrices (zeros, subnormals, the top of the exponent range, ties)
    scattered among ill-conditioned ones, plus the paper's random-bit class:
    what the fast kernel flags is finished by the fix-up pass with the general
    arithmetic, the tangent step included."""
    A = sprinkled(2**17 + 9, 4, np.float32, 3303, every=211)
    ill, _ = inputs.real_fp32_illcond(2**17 + 9, seed=3304)
    A[:, 1::2] = ill[:, 1::2]
    A = np.ascontiguousarray(np.concatenate([A, inputs.edge_real(np.float32),
                                             inputs.random_bits_f32(4096, 4, 3305)], axis=1))
    g, cnt = run(A, -4, backscale=backscale)
    with np.errstate(all="ignore"):
        o = oracle.svd2_tan64(A, -4, backscale=backscale)
    assert_same(g, o, f"s_tan64 edges bs={backscale}")
    assert cnt == o["count"]
    assert not np.isin(g["s"], [np.iinfo(np.int32).min]).any()


def test_tan64_misaligned_arrays_and_no_count():
    """Arrays off the 16-byte boundary take the one-matrix-per-thread path;
    count = NULL is accepted."""
    A32, _ = inputs.real_fp32_illcond(5001, seed=3306)
    base = torch.from_numpy(np.ascontiguousarray(np.pad(A32, ((0, 0), (1, 0))))).cuda()
    Ad = base[:, 1:]
    r = S.svd2_tan64(Ad, tau_log2=-4)
    torch.cuda.synchronize()
    g = {k: getattr(r, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}
    assert_same(g, oracle.svd2_tan64(A32, -4), "s_tan64 misaligned")


def test_tan64_argument_errors():
    L = S.lib()
    A = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    out = S.empty_result(4, 8, torch.float32, A.device)
    pa = S.ptr_array([A[i].data_ptr() for i in range(4)])
    pu = S.ptr_array([out.U[i].data_ptr() for i in range(4)])
    pv = S.ptr_array([out.V[i].data_ptr() for i in range(4)])
    args = (pa, pu, pv, out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr())
    assert L.svd2_batch_s_tan64(8, *args, 1, 0, None, None) == S.EINVAL       # tau > 0
    assert L.svd2_batch_s_tan64(8, *args, -101, 0, None, None) == S.EINVAL    # tau < -100
    assert L.svd2_batch_s_tan64(8, *args, -4, 2, None, None) == S.EINVAL      # unknown flag
    assert L.svd2_batch_s_tan64(-1, *args, -4, 0, None, None) == S.EINVAL
    assert L.svd2_batch_s_tan64(0, *args, -4, 0, None, None) == S.OK
    assert L.svd2_batch_s_tan64(8, None, pu, pv, *args[3:], -4, 0, None, None) == S.EINVAL


def test_tan64_host_buffers_match_device():
    """svd2_batch_host op 4 (the form at the default threshold) on pinned host
    arrays gives the device results."""
    A32, _ = inputs.real_fp32_illcond(2**16 + 3, seed=3307)
    g, _ = run(A32, S.TAN64_TAU_LOG2)
    Ah = torch.from_numpy(A32).pin_memory()
    out = S.svd2_host(Ah, tan64=True)
    torch.cuda.synchronize()
    h = {k: getattr(out, k).numpy() for k in ("U", "V", "smax", "smin", "s")}
    assert_same(h, g, "tan64 host")
    # pageable host arrays take the staged copy pipeline
    out2 = S.svd2_host(torch.from_numpy(A32.copy()), tan64=True, chunk=4096,
                       out=S.empty_host_result(4, A32.shape[1], torch.float32, pin=False))
    torch.cuda.synchronize()
    h2 = {k: getattr(out2, k).numpy() for k in ("U", "V", "smax", "smin", "s")}
    assert_same(h2, g, "tan64 host pageable")


def test_tan64_full_size_sampled():
    """The bench's workload and launch configuration, n = 2^26 at the default
    threshold: sampled matrices equal the oracle's form bit for bit, the count
    is the whole batch's, and sigma' against the double method stay within the
    form's stated bounds (8 units of 2^-24 for sigma'_max and for sigma'_min
    of the matrices that took the step; the oracle measures <= 6.2 and <= 5.2)."""
    A32, _ = inputs.real_fp32_illcond(2**26)
    Ad = torch.from_numpy(A32).cuda()
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    r = S.svd2_tan64(Ad, count=cnt)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(9).choice(A32.shape[1], 1 << 17, replace=False))
    it = torch.from_numpy(idx).cuda()
    g = {"U": r.U.index_select(1, it).cpu().numpy(), "V": r.V.index_select(1, it).cpu().numpy(),
         "smax": r.smax.index_select(0, it).cpu().numpy(),
         "smin": r.smin.index_select(0, it).cpu().numpy(),
         "s": r.s.index_select(0, it).cpu().numpy()}
    Asub = np.ascontiguousarray(A32[:, idx])
    o = oracle.svd2_tan64(Asub, S.TAN64_TAU_LOG2)
    assert_same(g, o, "tan64 full size sampled")
    frac = int(cnt.item()) / A32.shape[1]
    assert abs(frac - o["count"] / len(idx)) < 0.01, frac
    o64 = oracle.svd2(Asub.astype(np.float64), backscale=True)
    u = 2.0**-24
    bx = np.ldexp(g["smax"].astype(np.float64), -g["s"])
    bn = np.ldexp(g["smin"].astype(np.float64), -g["s"])
    assert (np.abs(bx - o64["smax"]) / o64["smax"]).max() <= 8 * u
    w = o["wide"].astype(bool) & (o64["smin"] > 0)
    assert (np.abs(bn - o64["smin"])[w] / o64["smin"][w]).max() <= 8 * u


def test_tan64_autotuner_keeps_results():
    """The tuner times the tangent-step kernel under its own launch shape (op
    4), leaves the plain FP32 shape alone, and the tuned kernel still matches
    the oracle bit for bit."""
    from paper_2005_07403_gb300 import tune
    A32, _ = inputs.real_fp32_illcond(50001, seed=3308)
    Ad = torch.from_numpy(A32).cuda()
    saved, saved_s = S.get_launch("s_tan64"), S.get_launch("s")
    try:
        t = tune.tune(Ad, reps=1, use_cache=False, form="tan64")
        assert S.get_launch("s_tan64") == (t["block"], t["mpt"], t["unroll"], t["waves"])
        assert S.get_launch("s") == saved_s
        g, cnt = run(A32, -3)
        o = oracle.svd2_tan64(A32, -3)
        assert_same(g, o, "tan64 tuned")
        assert cnt == o["count"]
    finally:
        S.set_launch("s_tan64", *saved)
