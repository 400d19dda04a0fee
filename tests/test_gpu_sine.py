"""The sine-based assembly of U (Eq. 31, flag SVD2_SINE) on the GPU against the
oracle's Eq. 31 assembly, bit for bit, for the four forms: ordinary and edge
matrices (the fix-up pass assembles by Eq. 31 too), back-scaling, every
matrices-per-thread shape, host buffers; and the entry points that do not
assemble U by Eq. 31 reject the flag."""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.test_gpu_fwd import assert_same, sprinkled

pytestmark = pytest.mark.gpu

FORMS = [(4, np.float64), (8, np.float64), (4, np.float32), (8, np.float32)]


def gpu(A, **kw):
    r = S.svd2(torch.from_numpy(A).cuda(), **kw)
    torch.cuda.synchronize()
    return {k: getattr(r, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}


@pytest.mark.parametrize("rows,dt", FORMS)
@pytest.mark.parametrize("backscale", [False, True])
def test_sine_matches_oracle(rows, dt, backscale):
    A = sprinkled(2**16 + 13, rows, dt, 700 + rows, every=97)
    g = gpu(A, sine=True, backscale=backscale)
    with np.errstate(all="ignore"):
        o = oracle.svd2(A, sine=True, backscale=backscale)
    assert_same(g, o, f"sine rows={rows} {dt.__name__} bs={backscale}")


@pytest.mark.parametrize("rows,dt", FORMS)
@pytest.mark.parametrize("mpt", [1, 2, 4])
def test_sine_every_shape(rows, dt, mpt):
    kind = S._kind(rows, torch.float64 if dt == np.float64 else torch.float32)
    A = inputs.normal_batch(20011, rows, 710, dt)
    o = oracle.svd2(A, sine=True)
    old = S.get_launch(kind)
    try:
        S.set_launch(kind, 256, mpt, 2, 0)     # the Eq. 31 kernels run one load group
        g = gpu(A, sine=True)
    finally:
        S.set_launch(kind, *old)
    assert_same(g, o, f"sine {kind} mpt={mpt}")


def test_sine_host_buffers():
    A = inputs.normal_batch(30001, 8, 720)
    Ah = torch.from_numpy(A).pin_memory()
    out = S.empty_host_result(8, A.shape[1], torch.float64)
    rc = S.lib().svd2_batch_host(
        S.OPS["z"], A.shape[1], S.ptr_array(S._host_rows(Ah, "A")),
        S.ptr_array(S._host_rows(out.U, "U")), S.ptr_array(S._host_rows(out.V, "V")),
        out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr(), S.SINE, 0,
        S.current_stream_handle())
    assert rc == S.OK
    torch.cuda.synchronize()
    h = {k: getattr(out, k).numpy() for k in ("U", "V", "smax", "smin", "s")}
    assert_same(h, oracle.svd2(A, sine=True), "sine host")


def test_sine_rejected_elsewhere():
    L = S.lib()
    A = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    out = S.empty_result(4, 8, torch.float32, A.device)
    pa = S.ptr_array([A[i].data_ptr() for i in range(4)])
    pu = S.ptr_array([out.U[i].data_ptr() for i in range(4)])
    pv = S.ptr_array([out.V[i].data_ptr() for i in range(4)])
    sx, sn, s = out.smax.data_ptr(), out.smin.data_ptr(), out.s.data_ptr()
    assert L.svd2_values_s(8, pa, sx, sn, s, S.SINE, None) == S.EINVAL
    assert L.svd2_batch_s_tan64(8, pa, pu, pv, sx, sn, s, -3, S.SINE, None, None) == S.EINVAL
    M = torch.zeros((8, 2, 2), dtype=torch.float32, device="cuda")
    U = torch.empty_like(M)
    V = torch.empty_like(M)
    assert L.svd2_batch_interleaved_s(8, M.data_ptr(), U.data_ptr(), V.data_ptr(), sx, sn, s,
                                      S.SINE, None) == S.EINVAL
