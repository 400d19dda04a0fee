"""svd2_batch_host: batches in host memory against the oracle bit for bit --
pinned arrays are read and written by the kernel directly, pageable ones (or
a mix) go through the chunked copy/compute pipeline (every form, many chunks
with a ragged last one, back-to-back calls, edge matrices that take the
fix-up pass of the FP32 forms)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.test_gpu_fwd import assert_same, sprinkled

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


@pytest.mark.parametrize("rows", [4, 8])
def test_host_mixed_pinned_and_pageable(rows):
    """Pinned inputs with pageable outputs: not every array is page-locked, so
    the staged pipeline runs."""
    n = 3 * 4096 + 5
    A = sprinkled(n, rows, np.float32, 41 + rows)
    out = S.empty_host_result(rows, n, torch.float32, pin=False)
    S.svd2_host(torch.from_numpy(A).pin_memory(), out=out, chunk=4096)
    torch.cuda.synchronize()
    g = {k: getattr(out, k).numpy() for k in ("U", "V", "smax", "smin", "s")}
    assert_same(g, oracle.svd2(A), "mixed")


@pytest.mark.parametrize("rows", [4, 8])
def test_host_direct_with_fixup_pass(rows):
    """All arrays pinned (the direct path) with edge matrices scattered in: the
    FP32 fix-up pass also reads and writes host memory."""
    n = 2**16 + 3
    A = sprinkled(n, rows, np.float32, 51 + rows, every=101)
    out = S.empty_host_result(rows, n, torch.float32, pin=True)
    S.svd2_host(torch.from_numpy(A).pin_memory(), out=out)
    torch.cuda.synchronize()
    g = {k: getattr(out, k).numpy() for k in ("U", "V", "smax", "smin", "s")}
    with np.errstate(all="ignore"):
        assert_same(g, oracle.svd2(A), "direct + fix-up")
