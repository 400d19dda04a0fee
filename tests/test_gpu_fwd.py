"""Parity of the CUDA forward kernels with the CPU oracle, element by element.

Every step of both sides is a correctly rounded IEEE operation in the paper's
order, so the kernels must reproduce the oracle bit for bit (signed zeros
included): this is stricter than the stated bar (s exact, sigma within 4 ulp,
backward error <= 8 eps ||A||_F), which the oracle itself meets (see the oracle
pins).  Inputs come from the seeded generators; sizes span many blocks and a
ragged tail; the full-size workloads are checked on sampled matrices.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2005_07403_gb300 import inputs
from paper_2005_07403_gb300 import svd2 as S
from tests.helpers import bits_equal

pytestmark = pytest.mark.gpu


def gpu_svd2(A, backscale=False, row_offset=0):
    """Run the kernel on numpy batch A; row_offset > 0 places every array at an
    element offset (misaligned for vector loads)."""
    rows, n = A.shape
    dt = torch.float64 if A.dtype == np.float64 else torch.float32
    if row_offset:
        buf = torch.empty((rows, n + row_offset), dtype=dt, device="cuda")
        buf[:, row_offset:] = torch.from_numpy(A).cuda()
        Ad = buf[:, row_offset:]
        out = S.Svd2Result(
            U=torch.empty((rows, n + row_offset), dtype=dt, device="cuda")[:, row_offset:],
            V=torch.empty((rows, n + row_offset), dtype=dt, device="cuda")[:, row_offset:],
            smax=torch.empty(n + row_offset, dtype=dt, device="cuda")[row_offset:],
            smin=torch.empty(n + row_offset, dtype=dt, device="cuda")[row_offset:],
            s=torch.empty(n + row_offset, dtype=torch.int32, device="cuda")[row_offset:])
    else:
        Ad = torch.from_numpy(A).cuda()
        out = None
    r = S.svd2(Ad, backscale=backscale, out=out)
    torch.cuda.synchronize()
    return {k: getattr(r, k).cpu().numpy() for k in ("U", "V", "smax", "smin", "s")}


def assert_same(g, o, what=""):
    for k in ("U", "V", "smax", "smin"):
        if not bits_equal(g[k], o[k]):
            bad = np.nonzero((g[k] != o[k]) & ~(np.isnan(g[k]) & np.isnan(o[k])))
            raise AssertionError(f"{what}: {k} differs at {bad[-1][:8]} ({len(bad[-1])} values)")
    assert np.array_equal(g["s"], o["s"]), what


def check(A, what, backscale=False, **kw):
    g = gpu_svd2(A, backscale=backscale, **kw)
    with np.errstate(all="ignore"):
        o = oracle.svd2(A, backscale=backscale)
    assert_same(g, o, what)


# ------------------------------------------------------------------ FP64

def test_real_mixed_workload():
    """The real FP64 workload: n = 65536 mixed classes (zero, diagonal,
    upper-triangular, rank-1, 2^e-scaled entries among N(0,1) matrices)."""
    check(inputs.real_mixed(65536), "real_mixed")


def test_real_ragged_tail_and_random_bits():
    check(inputs.real_mixed(65536 + 37, seed=7), "real_mixed+37")
    check(inputs.random_bits(2**16 + 3, 4, 11), "rbits")


def test_real_edge_cases():
    check(inputs.edge_real(), "edge")
    check(np.ascontiguousarray(np.repeat(inputs.edge_real(), 33, axis=1)), "edge x33")


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 31, 33, 255, 257])
def test_small_n(n):
    check(inputs.normal_batch(n, 4, 100 + n), f"d n={n}")
    check(inputs.normal_batch(n, 8, 200 + n), f"z n={n}")
    check(inputs.normal_batch(n, 4, 300 + n, np.float32), f"s n={n}")
    check(inputs.normal_batch(n, 8, 400 + n, np.float32), f"c n={n}")


def test_complex_workload_small():
    check(inputs.complex_scaled(2**16 + 5), "complex_scaled")
    check(inputs.random_bits(2**15 + 1, 8, 12), "crbits")
    check(inputs.normal_batch(2**15, 8, 13), "cnormal")


def test_complex_with_real_values():
    Ar = inputs.edge_real()
    Ac = np.zeros((8, Ar.shape[1]))
    Ac[0::2] = Ar
    check(Ac, "complex edge")


# ------------------------------------------------------------------ FP32

def test_fp32_real_and_complex():
    check(inputs.normal_batch(2**16 + 3, 4, 21, np.float32), "s normal")
    check(inputs.random_bits_f32(2**16, 4, 22), "s rbits")
    check(inputs.edge_real(np.float32), "s edge")
    A32, _ = inputs.real_fp32_illcond(2**16)
    check(A32, "s illcond")
    check(inputs.normal_batch(2**15 + 1, 8, 23, np.float32), "c normal")
    check(inputs.random_bits_f32(2**15, 8, 24), "c rbits")
    Z32, _ = inputs.complex_fp32_illcond(2**15 + 7, seed=25)
    check(Z32, "c illcond")
    check(Z32.astype(np.float64), "z illcond widened")


# ----------------------------------------------------------- options/shapes

def test_backscale_flag():
    """Fig. 1: Sigma = 2^-s Sigma' correctly rounded (overflow to inf allowed) and s = 0."""
    check(inputs.random_bits(2**14, 4, 31), "d backscale", backscale=True)
    check(inputs.random_bits(2**14, 8, 32), "z backscale", backscale=True)
    check(inputs.random_bits_f32(2**14, 4, 33), "s backscale", backscale=True)
    check(inputs.edge_real(), "edge backscale", backscale=True)


LAUNCHES = [(32, 1, 1, 0), (64, 2, 2, 1), (128, 4, 1, 2), (512, 4, 2, 0), (256, 1, 2, 1),
            (96, 2, 1, 3)]


@pytest.mark.parametrize("shape", LAUNCHES)
def test_launch_shapes_do_not_change_results(shape):
    A = {"d": inputs.real_mixed(40000 + 3, seed=5), "z": inputs.complex_scaled(20000 + 1),
         "s": inputs.normal_batch(40000 + 2, 4, 6, np.float32),
         "c": inputs.normal_batch(20000 + 3, 8, 7, np.float32)}
    saved = {k: S.get_launch(k) for k in A}
    try:
        for k, a in A.items():
            S.set_launch(k, *shape)
            check(a, f"{k} {shape}")
    finally:
        for k, v in saved.items():
            S.set_launch(k, *v)


def test_misaligned_arrays_take_the_scalar_path():
    check(inputs.real_mixed(10001), "d offset", row_offset=1)
    check(inputs.normal_batch(5003, 8, 41, np.float32), "c offset", row_offset=3)


def test_output_guard_bands_untouched():
    """Canaries after every output array (in place of a memory checker)."""
    n, pad = 10007, 64
    A = torch.from_numpy(inputs.normal_batch(n, 8, 51)).cuda()
    canary = float.fromhex("0x1.dead0p+7")
    bufs = [torch.full((8, n + pad), canary, dtype=torch.float64, device="cuda") for _ in range(2)]
    sb = [torch.full((n + pad,), canary, dtype=torch.float64, device="cuda") for _ in range(2)]
    si = torch.full((n + pad,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    out = S.Svd2Result(U=bufs[0][:, :n], V=bufs[1][:, :n], smax=sb[0][:n], smin=sb[1][:n], s=si[:n])
    S.svd2(A, out=out)
    torch.cuda.synchronize()
    for b in bufs:
        assert torch.all(b[:, n:] == canary)
    for b in sb:
        assert torch.all(b[n:] == canary)
    assert torch.all(si[n:] == 0x5A5A5A5A)


def test_zero_length_is_noop():
    A = torch.empty((4, 0), dtype=torch.float64, device="cuda")
    r = S.svd2(A)
    assert r.U.shape == (4, 0)


# ------------------------------------------------------ full-size, sampled

def sprinkled(n, rows, dtype, seed, every=997):
    """N(0,1) batch with an edge matrix (zeros, subnormals, the top of the
    exponent range, pivot ties) at every `every`-th position from 3: the
    matrices the fast arithmetic of the batch kernels hands to the fix-up pass,
    scattered over blocks, vector lanes and the ragged tail."""
    A = inputs.normal_batch(n, rows, seed, dtype)
    E = inputs.edge_real(dtype)
    m = E.shape[1]
    idx = np.arange(3, n, every)
    k = np.arange(len(idx))
    if rows == 4:
        A[:, idx] = E[:, k % m]
    else:   # complex: real parts from one edge case, imaginary parts from another
        A[0::2, idx] = E[:, k % m]
        A[1::2, idx] = E[:, (k + 5) % m]
    return np.ascontiguousarray(A)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("rows", [4, 8])
@pytest.mark.parametrize("backscale", [False, True])
def test_fixup_pass_scattered_edges(dtype, rows, backscale):
    """The batch kernels finish ordinary matrices on branch-free fast forms and
    leave the rest (s = INT32_MIN) to a second pass with the general
    arithmetic: the combined result must equal the oracle bit for bit, and no
    sentinel may remain."""
    A = sprinkled(2**18 + 5, rows, dtype, 71 + rows)
    g = gpu_svd2(A, backscale=backscale)
    with np.errstate(all="ignore"):
        o = oracle.svd2(A, backscale=backscale)
    assert_same(g, o, f"fixup rows={rows} bs={backscale}")
    assert not np.isin(g["s"], [np.iinfo(np.int32).min, np.iinfo(np.int32).min + 1]).any()


def spread_cases(seed, spreads):
    """Real FP32 matrices whose nonzero entries span a given number of binades:
    the largest entry near 2^E (E = max(0, d - 120), so every entry stays
    normal), others 2^(E-d) times a random significand, placed in every
    position, with random signs; plus nearly and exactly singular ones
    (a22 = a21 a12 / a11 up to a few ulps) whose r''22 (Eq. 7) cancels."""
    rng = np.random.default_rng(seed)
    cols = []
    for d in spreads:
        first = len(cols)
        for pos in range(4):
            for _ in range(24):
                sig = rng.uniform(1.0, 2.0, 4) * rng.choice([-1.0, 1.0], 4)
                e = -rng.integers(0, d + 1, 4)
                e[pos] = -d
                e[rng.integers(0, 4)] = 0
                cols.append(np.ldexp(sig, e))
        for _ in range(24):
            a11, a21, a12 = np.ldexp(rng.uniform(1, 2, 3), [0, -d // 2, -(d - d // 2)])
            for k in range(-2, 3):
                a22 = np.float32(a21 * a12 / a11)
                a22 = np.nextafter(a22, np.float32(np.inf)) if k > 0 else a22
                cols.append([a11, a21, a12, a22 * (1 + k * 2.0**-23)])
        E = max(0, d - 120)
        cols[first:] = [np.ldexp(np.asarray(c, dtype=np.float64), E) for c in cols[first:]]
    return np.ascontiguousarray(np.array(cols, dtype=np.float64).T.astype(np.float32))


def test_fp32_spread_boundary_of_the_fast_path():
    """The real FP32 kernels run the method at the scale h - 64 when every
    nonzero entry is within 64 binades of the largest (and none is subnormal),
    and hand the rest to the fix-up pass.  Matrices with spreads around that
    boundary, and around the range where a shifted exponent would wrap, must
    all match the oracle bit for bit."""
    A = spread_cases(91, list(range(58, 71)) + list(range(180, 196)))
    for bs in (False, True):
        check(A, f"spread boundary bs={bs}", backscale=bs)


def spread_cases_complex(seed, spreads):
    """Complex FP32 matrices (8 split rows) whose nonzero parts span a given
    number of binades, the largest part in every position; nearly rank-one
    complex matrices u v^T + a few-ulp perturbation whose imaginary parts are
    2^-k times the real ones (k up to 60: the cancellation of Eq. 7 and the
    phase of r'_12 then leave tiny parts in r'_12, r''_22 and r'_22); and
    real-valued ones (zero imaginary parts)."""
    rng = np.random.default_rng(seed)
    cols = []
    for d in spreads:
        for pos in range(8):
            for _ in range(12):
                sig = rng.uniform(1.0, 2.0, 8) * rng.choice([-1.0, 1.0], 8)
                e = -rng.integers(0, d + 1, 8)
                e[pos] = -d
                e[rng.integers(0, 8)] = 0
                cols.append(np.ldexp(sig, e))
    for k in list(range(0, 61, 4)) + [62, 63, 64, 65]:
        for _ in range(48):
            u = rng.standard_normal(2) + 1j * np.ldexp(rng.standard_normal(2), -k)
            v = rng.standard_normal(2) + 1j * np.ldexp(rng.standard_normal(2), -k)
            M = np.outer(u, v)
            M = M * (1 + 2.0**-23 * rng.integers(-3, 4, (2, 2)))
            if rng.random() < 0.25:
                M = M.real + 0j
            # record order: a11, a21, a12, a22, each (Re, Im)
            z = [M[0, 0], M[1, 0], M[0, 1], M[1, 1]]
            cols.append(np.array([x for w in z for x in (w.real, w.imag)]))
    A = np.array(cols, dtype=np.float64).T
    return np.ascontiguousarray(A.astype(np.float32))


def test_complex_fp32_spread_boundary_of_the_fast_path():
    """The complex FP32 kernels run the method at the scale h - 64 when every
    nonzero part is within 64 binades of the largest, and flag for the fix-up
    pass any matrix whose Eq. 7 cancellation (or the phase of r'_12) leaves a
    part of r'_12, r''_22, r'_22 below 2^-100 at that scale: spreads around the
    boundary and such cancellations must all match the oracle bit for bit."""
    A = spread_cases_complex(92, list(range(58, 71)) + [100, 150, 200, 240])
    for bs in (False, True):
        check(A, f"complex spread boundary bs={bs}", backscale=bs)


def _sampled_check(A, what, nsample=1 << 15, seed=0):
    g = S.svd2(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(seed).choice(A.shape[1], nsample, replace=False))
    idx_t = torch.from_numpy(idx).cuda()
    gs = {k: getattr(g, k).index_select(-1, idx_t).cpu().numpy()
          for k in ("U", "V", "smax", "smin", "s")}
    o = oracle.svd2(np.ascontiguousarray(A[:, idx]))
    assert_same(gs, o, what)


def test_full_size_complex_workload_sampled():
    """The complex128 workload at its full size n = 2^24, in the launch shape
    the benchmark uses, on 2^15 sampled matrices."""
    _sampled_check(inputs.complex_scaled(2**24), "complex 2^24")


def test_full_size_fp32_workload_sampled():
    A32, _ = inputs.real_fp32_illcond(2**26)
    _sampled_check(A32, "fp32 2^26")


def test_full_size_fp64_workload_sampled():
    """The FP32-vs-FP64 batch at n = 2^26 through the FP64 form (the exact
    widening of the FP32 values), on 2^15 sampled matrices."""
    A32, _ = inputs.real_fp32_illcond(2**26)
    _sampled_check(A32.astype(np.float64), "fp64 2^26")


def test_full_size_complex64_workload_sampled():
    Z32, _ = inputs.complex_fp32_illcond(2**25)
    _sampled_check(Z32, "complex64 2^25")
