"""The allocation-free entry point svd2_batch_s_rerun_noalloc, called through
the C ABI, against svd2_batch_s_rerun with a caller-provided workspace.

The allocation-free variant serves callers that cannot allocate device memory
(their memory belongs to another allocator, or they must not call cudaMalloc
while running); it keeps its scratch in a fixed device array shared by all
calls.  Two calls in a row on different inputs check that the shared scratch
starts each call clean.  This file runs last (pytest collects it last), so a
failure here leaves every other test already run; it also passes on its own
in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.helpers import bits_equal

pytestmark = pytest.mark.gpu


def _noalloc(Ad, out, tau):
    L = S.lib()
    rc = L.svd2_batch_s_rerun_noalloc(
        Ad.shape[1], S.ptr_array([Ad[i].data_ptr() for i in range(4)]),
        S.ptr_array([out.U[i].data_ptr() for i in range(4)]),
        S.ptr_array([out.V[i].data_ptr() for i in range(4)]),
        out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr(), tau, 0,
        S.current_stream_handle(Ad.device))
    return rc


@pytest.mark.parametrize("n", [S.NOALLOC_MAX_N, 100003])
def test_noalloc_matches_workspace_entry_point_on_two_calls(n):
    for seed, tau in ((1, -8), (2, -5)):
        A32, _ = inputs.real_fp32_illcond(n, seed=seed)
        Ad = torch.from_numpy(A32).cuda()
        out = S.empty_result(4, n, torch.float32, Ad.device)
        assert _noalloc(Ad, out, tau) == S.OK
        ref = S.svd2_rerun(Ad, tau_log2=tau)
        torch.cuda.synchronize()
        assert S.rerun_count(ref.workspace) > 0
        for k in ("U", "V", "smax", "smin", "s"):
            a = getattr(out, k).cpu().numpy()
            b = getattr(ref, k).cpu().numpy()
            assert bits_equal(a, b) if a.dtype != np.int32 else np.array_equal(a, b), (n, seed, k)


def test_noalloc_rejects_batches_above_its_capacity():
    L = S.lib()
    null4 = S.ptr_array([0, 0, 0, 0])
    assert L.svd2_batch_s_rerun_noalloc(S.NOALLOC_MAX_N + 1, null4, null4, null4, None, None,
                                        None, -8, 0, None) == S.ETOOBIG
    assert L.svd2_batch_s_rerun_noalloc(-1, null4, null4, null4, None, None, None, -8, 0,
                                        None) == S.EINVAL
