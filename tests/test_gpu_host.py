"""svd2_batch_host: batches in host memory through the chunked copy/compute
pipeline, against the oracle bit for bit (every form, many chunks with a
ragged last one, pinned and pageable host memory, back-to-back calls)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.test_gpu_fwd import assert_same

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rows,dt", [(4, np.float64), (8, np.float64), (4, np.float32),
                                     (8, np.float32)])
@pytest.mark.parametrize("pin", [True, False])
def test_host_pipeline_matches_oracle(rows, dt, pin):
    n = 5 * 4096 + 123
    A = inputs.normal_batch(n, rows, 7 + rows, dt)
    At = torch.from_numpy(A)
    if pin:
        At = At.pin_memory()
    out = S.empty_host_result(rows, n, At.dtype, pin=pin)
    S.svd2_host(At, out=out, chunk=4096)
    torch.cuda.synchronize()
    g = {k: getattr(out, k).numpy() for k in ("U", "V", "smax", "smin", "s")}
    assert_same(g, oracle.svd2(A), f"host {rows} {dt} pin={pin}")


def test_host_pipeline_back_to_back_calls():
    outs, As = [], []
    for i in range(3):
        A = inputs.complex_scaled(3 * 4096 + 17 * i, seed=100 + i)
        As.append(A)
        outs.append(S.svd2_host(torch.from_numpy(A).pin_memory(), chunk=4096))
    torch.cuda.synchronize()
    for A, out in zip(As, outs):
        g = {k: getattr(out, k).numpy() for k in ("U", "V", "smax", "smin", "s")}
        assert_same(g, oracle.svd2(A), "back-to-back")
