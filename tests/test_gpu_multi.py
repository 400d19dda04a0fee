"""The multi-batch launch (svd2_multi_*: one block per tile by default, or a
persistent grid), its CUDA graph, and the autotuners, against the oracle
batch by batch (bit for bit)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.test_gpu_fwd import assert_same, sprinkled

pytestmark = pytest.mark.gpu


def _batches(count, seed, lo=0, hi=3000):
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi, count)
    lens[: 3] = [0, 1, 2]
    kinds = rng.random(count) < 0.5
    out = []
    for i, (n, c) in enumerate(zip(lens, kinds)):
        rows = 8 if c else 4
        A = inputs.normal_batch(int(n), rows, seed * 1000 + i)
        if i % 7 == 3 and not c and n > 0:
            A = inputs.real_mixed(int(n), seed=seed * 1000 + i)
        if i % 7 == 5 and c and n > 0:      # complex edge matrices for the fix-up pass
            A = sprinkled(int(n), 8, np.float64, seed * 1000 + i, every=13)
        out.append(A)
    return out


def _check_all(mb, hosts, what):
    torch.cuda.synchronize()
    for i, (A, o) in enumerate(zip(hosts, mb.outputs)):
        g = {k: getattr(o, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}
        assert_same(g, oracle.svd2(A), f"{what} batch {i}")


@pytest.mark.parametrize("shape", [(256, 1, 1), (64, 2, 2), (512, 1, 2), (128, 2, 1),
                                   (1024, 1, 1), (128, 4, 1), (256, 4, 2)])
def test_multi_matches_oracle_per_batch(shape):
    hosts = _batches(40, 3)
    mb = S.MultiBatch([torch.from_numpy(A).cuda() for A in hosts], *shape)
    mb.run()
    _check_all(mb, hosts, str(shape))


@pytest.mark.parametrize("grid", [1, 7, 304, 100000])
def test_multi_explicit_grids_match(grid):
    """A persistent grid (one block, a few, one resident wave) and a grid with
    more blocks than tiles give the same results as one block per tile."""
    hosts = _batches(30, 5, hi=6000)
    mb = S.MultiBatch([torch.from_numpy(A).cuda() for A in hosts], 256, 1, 1)
    mb.run(grid=grid)
    _check_all(mb, hosts, f"grid {grid}")


def test_multi_graph_replay_follows_data():
    hosts = _batches(25, 4)
    dev = [torch.from_numpy(A).cuda() for A in hosts]
    mb = S.MultiBatch(dev, 128, 1, 2)
    g = mb.graph()
    g.launch()
    _check_all(mb, hosts, "graph 1")
    new = [inputs.normal_batch(A.shape[1], A.shape[0], 77 + i) for i, A in enumerate(hosts)]
    for d, A in zip(dev, new):
        d.copy_(torch.from_numpy(A))
    g.launch()
    g.launch()
    _check_all(mb, new, "graph 2")
    g.close()


def test_multi_shape_mismatch_is_rejected():
    """A launch whose tile size (block x mpt x unroll) differs from the plan's
    would process nothing: run and graph creation return SVD2_EINVAL and leave
    the outputs untouched."""
    hosts = _batches(5, 5, lo=100, hi=500)
    mb = S.MultiBatch([torch.from_numpy(A).cuda() for A in hosts], 256, 1, 1)
    for o in mb.outputs:
        o.smax.fill_(7.0)
    L = S.lib()
    assert L.svd2_multi_run(mb.plan.data_ptr(), 128, 1, 1, 0, S.current_stream_handle()) == S.EINVAL
    assert L.svd2_multi_run(mb.plan.data_ptr(), 256, 2, 1, 0, S.current_stream_handle()) == S.EINVAL
    h = ctypes.c_void_p()
    assert L.svd2_multi_graph_create(mb.plan.data_ptr(), 128, 1, 1, 0, ctypes.byref(h)) == S.EINVAL
    torch.cuda.synchronize()
    assert all(bool(torch.all(o.smax == 7.0)) for o in mb.outputs)
    # the plan's own shape still runs
    assert L.svd2_multi_run(mb.plan.data_ptr(), 256, 1, 1, 0, S.current_stream_handle()) == S.OK
    _check_all(mb, hosts, "after rejected shapes")


def test_multi_autotune_picks_a_valid_shape():
    hosts = _batches(30, 6, hi=20000)
    mb = S.MultiBatch([torch.from_numpy(A).cuda() for A in hosts])
    best = mb.autotune(reps=2)
    assert best["block"] in (64, 128, 256, 512, 1024) and best["mpt"] in (1, 2, 4)
    assert best["ms"] > 0
    mb.run()
    _check_all(mb, hosts, "tuned")


@pytest.mark.parametrize("kind,rows,dt", [("d", 4, np.float64), ("z", 8, np.float64),
                                          ("s", 4, np.float32), ("c", 8, np.float32)])
def test_autotune_fwd_keeps_results(kind, rows, dt):
    from paper_2005_07403_gb300 import tune
    A = inputs.normal_batch(50001, rows, 9, dt)
    Ad = torch.from_numpy(A).cuda()
    saved = S.get_launch(kind)
    try:
        best = S.autotune_fwd(Ad, reps=1)
        assert S.get_launch(kind) == (best["block"], best["mpt"], best["unroll"], best["waves"])
        r = S.svd2(Ad)
        torch.cuda.synchronize()
        g = {k: getattr(r, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}
        assert_same(g, oracle.svd2(A), f"tuned {kind}")
        t = tune.tune(Ad, reps=1, use_cache=False)
        assert t["cached"] is False
        t2 = tune.tune(Ad)
        assert t2["cached"] is True and t2["block"] == t["block"]
    finally:
        S.set_launch(kind, *saved)


def test_multi_full_workload_sampled():
    """The Kogbetliantz batching workload at full size: 2048 batches, lengths
    log-uniform in [16, 2^20], real FP64 / complex128 at random, N(0,1) entries
    drawn on the device; one graph replay; 2^15 sampled matrices against the
    oracle."""
    lens, cplx = inputs.kog_batches()
    dev = [inputs.normal_batch_device(int(n), 8 if c else 4, 5000 + i)
           for i, (n, c) in enumerate(zip(lens, cplx))]
    mb = S.MultiBatch(dev, 256, 1, 1)
    g = mb.graph()
    g.launch()
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    picks = rng.choice(len(dev), 64, replace=False)
    for bi in picks:
        n = dev[bi].shape[1]
        idx = np.sort(rng.choice(n, min(n, 512), replace=False))
        it = torch.from_numpy(idx).cuda()
        A = dev[bi].index_select(1, it).cpu().numpy()
        o = mb.outputs[bi]
        gg = {k: getattr(o, k).index_select(-1, it).cpu().numpy()
              for k in ("U", "V", "smax", "smin", "s")}
        assert_same(gg, oracle.svd2(np.ascontiguousarray(A)), f"batch {bi}")
    g.close()
