"""Batches past 2^31 matrices: every index of the split layout is 64-bit in
the kernels, the grid-stride loops run past the 32-bit range, and the re-run
form splits such a batch into launches.  A real FP32 batch of just over 2^31
matrices (n = 2^31 + 2^16 + 7; N(0,1) entries drawn on the GPU; 120 GB of
inputs and outputs, plus 8 GB of re-run workspace) with ill-conditioned and
edge matrices planted at the start, across index 2^31 and at the end; sampled outputs of the plain FP32
form, the FP64 tangent-step form and the FP64 re-run form against the oracle,
bit for bit.  Skipped on a device with less free memory than it needs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.test_gpu_fwd import assert_same

pytestmark = pytest.mark.gpu

N = 2**31 + 2**16 + 7
NEED = 140 * 2**30


def _planted():
    ill, _ = inputs.real_fp32_illcond(3 * 4096, seed=4401)
    edge = inputs.edge_real(np.float32)
    bits = inputs.random_bits_f32(1024, 4, 4402)
    return np.ascontiguousarray(np.concatenate([ill, edge, bits], axis=1))


def _sample_index(planted_at, m):
    rng = np.random.default_rng(4403)
    idx = [rng.choice(N, 1 << 14, replace=False)]
    for p in planted_at:
        idx.append(np.arange(p, p + m))
    idx.append(np.arange(N - 64, N))
    idx.append(np.arange(2**31 - 64, 2**31 + 64))
    return np.unique(np.concatenate(idx))


def _take(r, it):
    return {k: getattr(r, k).index_select(-1, it).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}


def test_forms_past_2_31_matrices():
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < NEED:
        pytest.skip(f"needs {NEED >> 30} GiB of free device memory, {free >> 30} GiB free")
    P = _planted()
    m = P.shape[1]
    planted_at = [0, 2**31 - m // 2, N - m]
    A = inputs.normal_batch_device(N, 4, 4404, dtype=torch.float32)
    Pd = torch.from_numpy(P).cuda()
    for p in planted_at:
        A[:, p:p + m] = Pd
    idx = _sample_index(planted_at, m)
    it = torch.from_numpy(idx).cuda()
    Asub = np.ascontiguousarray(A.index_select(1, it).cpu().numpy())
    out = S.empty_result(4, N, torch.float32, A.device)
    with np.errstate(all="ignore"):
        S.svd2(A, out=out)
        torch.cuda.synchronize()
        assert_same(_take(out, it), oracle.svd2(Asub), "plain FP32, n = 2^31 + 2^16 + 7")
        S.svd2_tan64(A, tau_log2=S.TAN64_TAU_LOG2, out=out)
        torch.cuda.synchronize()
        assert_same(_take(out, it), oracle.svd2_tan64(Asub, S.TAN64_TAU_LOG2),
                    "FP64 tangent step, n = 2^31 + 2^16 + 7")
        r = S.svd2_rerun(A, tau_log2=S.RERUN_TAU_LOG2, out=out)
        torch.cuda.synchronize()
        o = oracle.svd2_rerun(Asub, S.RERUN_TAU_LOG2)
        assert_same(_take(out, it), o, "FP64 re-run, n = 2^31 + 2^16 + 7")
        assert S.rerun_count(r.workspace) >= o["count"] > 0
