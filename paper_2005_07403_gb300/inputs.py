"""Seeded synthetic batches of 2x2 matrices in the split layout of Sec. 3.

This module only draws and places input numbers; it contains none of the SVD
method's arithmetic, so both the CPU oracle's tests and the CUDA library's tests
and benchmark can use it.  Every generator is deterministic in its seed (numpy
PCG64, identical on x86-64 and AArch64).

Real batches have shape (4, n): rows a11, a21, a12, a22.  Complex batches have
shape (8, n): Re a11, Im a11, Re a21, Im a21, Re a12, Im a12, Re a22, Im a22
(the record order of Sec. 8).

The paper's own data (Sec. 8) were 2^36 random-bit finite doubles read from
/dev/urandom; that file is not available, so these seeded workloads stand in
for it, and ``random_bits`` reproduces its distribution.
"""
from __future__ import annotations

import numpy as np

SEED_CFG1 = 2005074031
SEED_CFG2 = 2005074032
SEED_CFG3 = 2005074033
SEED_CFG4 = 2005074034
SEED_CFG5 = 2005074035

REAL_ROWS = 4
CPLX_ROWS = 8


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rot(theta):
    c, s = np.cos(theta), np.sin(theta)
    return c, s


def _from_rotations(theta1, sig1, sig2, theta2):
    """A = R(theta1) diag(sig1, sig2) R(theta2)^T as (4, m) rows a11, a21, a12, a22."""
    c1, s1 = _rot(theta1)
    c2, s2 = _rot(theta2)
    # R(t) = [[c, -s], [s, c]]
    a11 = c1 * sig1 * c2 + (-s1) * sig2 * (-s2)
    a12 = c1 * sig1 * s2 + (-s1) * sig2 * c2
    a21 = s1 * sig1 * c2 + c1 * sig2 * (-s2)
    a22 = s1 * sig1 * s2 + c1 * sig2 * c2
    return np.stack([a11, a21, a12, a22])


def real_mixed(n: int = 65536, seed: int = SEED_CFG1) -> np.ndarray:
    """Real FP64 batch: 7/8 i.i.d. N(0,1) entries; the other 1/8 split evenly
    (class j mod 5) among zero, diagonal, upper-triangular, rank-1 (outer product
    of two N(0,1) vectors) and N(0,1) entries scaled by 2^e, e uniform in
    [-1000, 1000] drawn per entry.  Classes are placed by a seeded permutation.
    Also returns nothing else: the class of each column is ``real_mixed_classes``.
    """
    return _real_mixed(n, seed)[0]


def real_mixed_classes(n: int = 65536, seed: int = SEED_CFG1) -> np.ndarray:
    """Class code per column of ``real_mixed``: -1 = N(0,1), 0 = zero, 1 = diagonal,
    2 = upper-triangular, 3 = rank-1, 4 = scaled by 2^e."""
    return _real_mixed(n, seed)[1]


def _real_mixed(n, seed):
    rng = _rng(seed)
    A = rng.standard_normal((4, n))
    nspec = n // 8
    cls = np.full(n, -1, np.int8)
    pos = rng.permutation(n)[:nspec]
    kinds = np.arange(nspec) % 5
    cls[pos] = kinds
    # zero
    z = pos[kinds == 0]
    A[:, z] = 0.0
    # diagonal: off-diagonal +0
    d = pos[kinds == 1]
    A[1, d] = 0.0
    A[2, d] = 0.0
    # upper-triangular: a21 = +0
    u = pos[kinds == 2]
    A[1, u] = 0.0
    # rank-1 u v^T
    r = pos[kinds == 3]
    uu = rng.standard_normal((2, r.size))
    vv = rng.standard_normal((2, r.size))
    A[0, r] = uu[0] * vv[0]
    A[1, r] = uu[1] * vv[0]
    A[2, r] = uu[0] * vv[1]
    A[3, r] = uu[1] * vv[1]
    # scaled per entry by 2^e, e in [-1000, 1000]
    sc = pos[kinds == 4]
    e = rng.integers(-1000, 1001, size=(4, sc.size))
    A[:, sc] = np.ldexp(A[:, sc], e)
    return np.ascontiguousarray(A), cls


def complex_scaled(n: int = 2**24, seed: int = SEED_CFG2) -> np.ndarray:
    """Complex128 batch: real and imaginary parts uniform in [-1, 1] times 2^e, e
    uniform integer in [-500, 500] per matrix; 1% of the matrices are
    rank-deficient outer products u v^T of random complex vectors (parts uniform
    in [-1, 1]) times 2^e."""
    rng = _rng(seed)
    A = rng.uniform(-1.0, 1.0, size=(8, n))
    e = rng.integers(-500, 501, size=n)
    nr = n // 100
    r = rng.permutation(n)[:nr]
    u = rng.uniform(-1.0, 1.0, size=(4, nr))   # Re u1, Im u1, Re u2, Im u2
    v = rng.uniform(-1.0, 1.0, size=(4, nr))
    ur = (u[0], u[2])
    ui = (u[1], u[3])
    vr = (v[0], v[2])
    vi = (v[1], v[3])
    # element (i, j) = u_i * v_j ; record slot 2*(2*j+i)
    for j in range(2):
        for i in range(2):
            slot = 2 * (2 * j + i)
            A[slot, r] = ur[i] * vr[j] - ui[i] * vi[j]
            A[slot + 1, r] = ur[i] * vi[j] + ui[i] * vr[j]
    A = np.ldexp(A, e[None, :])
    return np.ascontiguousarray(A)


def real_fp32_illcond(n: int = 2**26, seed: int = SEED_CFG3):
    """Real batch for the FP32 vs FP64 comparison: 90% i.i.d. N(0,1) entries and
    10% ill-conditioned R(t1) diag(1, 10^-u) R(t2)^T with t uniform in [0, 2pi)
    and u uniform in [2, 12].  Generated in FP64 and rounded to FP32; the FP64
    form runs on the exact widening of these FP32 values.  Returns
    (A32 of shape (4, n), is_illcond bool mask)."""
    rng = _rng(seed)
    A = rng.standard_normal((4, n), dtype=np.float64)
    ni = n // 10
    idx = rng.permutation(n)[:ni]
    t1 = rng.uniform(0.0, 2 * np.pi, ni)
    t2 = rng.uniform(0.0, 2 * np.pi, ni)
    u = rng.uniform(2.0, 12.0, ni)
    A[:, idx] = _from_rotations(t1, np.ones(ni), 10.0 ** (-u), t2)
    mask = np.zeros(n, bool)
    mask[idx] = True
    return np.ascontiguousarray(A.astype(np.float32)), mask


def complex_fp32_illcond(n: int = 2**25, seed: int = SEED_CFG3 + 100):
    """Complex batch for the complex FP32 form with re-run: 90% i.i.d. N(0,1)
    parts and 10% ill-conditioned D1 R(t1) diag(1, 10^-u) R(t2)^T D2 with
    D1 = diag(e^(i a1), e^(i a2)), D2 = diag(e^(i b1), e^(i b2)), the phases
    uniform in [0, 2pi) and t, u drawn as in ``real_fp32_illcond`` (the phase
    factors are unitary: the singular values are 1 and 10^-u).  Generated in
    FP64 and rounded to FP32.  Returns (A32 of shape (8, n), is_illcond mask)."""
    rng = _rng(seed)
    A = rng.standard_normal((8, n), dtype=np.float64)
    ni = n // 10
    idx = rng.permutation(n)[:ni]
    t1 = rng.uniform(0.0, 2 * np.pi, ni)
    t2 = rng.uniform(0.0, 2 * np.pi, ni)
    u = rng.uniform(2.0, 12.0, ni)
    ph = rng.uniform(0.0, 2 * np.pi, (4, ni))          # a1, a2, b1, b2
    M = _from_rotations(t1, np.ones(ni), 10.0 ** (-u), t2)   # m11, m21, m12, m22
    # entry (i, j) of D1 M D2 is e^(i (a_i + b_j)) m_ij
    for e, (ai, bj) in enumerate(((0, 2), (1, 2), (0, 3), (1, 3))):
        phase = ph[ai] + ph[bj]
        A[2 * e, idx] = M[e] * np.cos(phase)
        A[2 * e + 1, idx] = M[e] * np.sin(phase)
    mask = np.zeros(n, bool)
    mask[idx] = True
    return np.ascontiguousarray(A.astype(np.float32)), mask


def kog_batches(seed: int = SEED_CFG4, count: int = 2048, lo_log2: float = 4.0,
                hi_log2: float = 20.0):
    """Batch shapes of a sequence of Kogbetliantz steps: ``count`` batches with
    lengths n_i = round(2^U(lo, hi)) (log-uniform in [16, 2^20] by default) and
    kinds Bernoulli(1/2) real FP64 / complex128.  Returns (lengths int64 array,
    is_complex bool array)."""
    rng = _rng(seed)
    lengths = np.rint(np.exp2(rng.uniform(lo_log2, hi_log2, count))).astype(np.int64)
    cplx = rng.random(count) < 0.5
    return lengths, cplx


def normal_batch(n: int, rows: int, seed: int, dtype=np.float64) -> np.ndarray:
    """i.i.d. N(0,1) entries (real and imaginary parts alike), shape (rows, n)."""
    return np.ascontiguousarray(_rng(seed).standard_normal((rows, n)).astype(dtype))


def grad_batch(n: int = 2**22, seed: int = SEED_CFG5):
    """Inputs for the differentiation check: A = R(t1) diag(s1, s2) R(t2)^T with
    s1 uniform in [0.5, 2] and relative gap g = (s1 - s2)/s1 log-uniform in
    [1e-3, 1] for 90% and in [1e-12, 1e-6] for 10% of the matrices, plus
    i.i.d. N(0,1) upstream gradients.  Returns dict(A, gU, gV, gS (2, n),
    small_gap mask)."""
    rng = _rng(seed)
    t1 = rng.uniform(0.0, 2 * np.pi, n)
    t2 = rng.uniform(0.0, 2 * np.pi, n)
    s1 = rng.uniform(0.5, 2.0, n)
    small = np.zeros(n, bool)
    small[rng.permutation(n)[: n // 10]] = True
    lg = np.where(small, rng.uniform(np.log(1e-12), np.log(1e-6), n),
                  rng.uniform(np.log(1e-3), np.log(1.0), n))
    g = np.exp(lg)
    s2 = s1 * (1.0 - g)
    A = np.ascontiguousarray(_from_rotations(t1, s1, s2, t2))
    gU = rng.standard_normal((4, n))
    gV = rng.standard_normal((4, n))
    gS = rng.standard_normal((2, n))
    return dict(A=A, gU=gU, gV=gV, gS=gS, small_gap=small)


def random_bits(n: int, rows: int = 4, seed: int = 1) -> np.ndarray:
    """Uniform random 64-bit patterns read as doubles, non-finite ones redrawn
    (the test data of Sec. 8)."""
    rng = _rng(seed)
    bits = rng.integers(0, 2**64, size=(rows, n), dtype=np.uint64, endpoint=False)
    A = bits.view(np.float64)
    bad = ~np.isfinite(A)
    while bad.any():
        A[bad] = rng.integers(0, 2**64, size=int(bad.sum()), dtype=np.uint64).view(np.float64)
        bad = ~np.isfinite(A)
    return np.ascontiguousarray(A)


def random_bits_f32(n: int, rows: int = 4, seed: int = 1) -> np.ndarray:
    """Uniform random 32-bit patterns read as floats, non-finite ones redrawn."""
    rng = _rng(seed)
    bits = rng.integers(0, 2**32, size=(rows, n), dtype=np.uint32)
    A = bits.view(np.float32)
    bad = ~np.isfinite(A)
    while bad.any():
        A[bad] = rng.integers(0, 2**32, size=int(bad.sum()), dtype=np.uint32).view(np.float32)
        bad = ~np.isfinite(A)
    return np.ascontiguousarray(A)


def edge_real(dtype=np.float64) -> np.ndarray:
    """Hand-picked real matrices exercising the special cases of Sec. 2: zeros
    of both signs, subnormals, entries at the top of the exponent range (s < 0),
    equal column norms and equal row magnitudes (pivot ties), x = 0, y = 0, and
    the tan(2 phi) bound of Eq. 14.  Shape (4, m), rows a11, a21, a12, a22."""
    fi = np.finfo(dtype)
    tiny = fi.smallest_subnormal
    big = fi.max
    top = np.ldexp(dtype(1), fi.maxexp - 1)       # 2^(MAX_EXP-1): exponent h+2, s = -2
    top1 = np.ldexp(dtype(1), fi.maxexp - 2)      # exponent h+1, s = -1
    eps_small = np.ldexp(dtype(1), -60 if dtype == np.float64 else -30)
    lo = float(np.ldexp(dtype(1), fi.minexp + 24))   # normal, far below 1
    hi = float(np.ldexp(dtype(1), fi.maxexp - 24))   # finite, far above 1
    cases = [
        (0.0, 0.0, 0.0, 0.0),
        (-0.0, -0.0, -0.0, -0.0),
        (0.0, -0.0, -0.0, 0.0),
        (1.0, 0.0, 0.0, 1.0),
        (2.0, 0.0, 0.0, -3.0),
        (-5.0, 0.0, 0.0, 5.0),
        (0.0, 1.0, 1.0, 0.0),
        (1.0, 1.0, 1.0, 1.0),
        (1.0, -1.0, 1.0, 1.0),
        (3.0, 4.0, 0.0, 0.0),
        (0.0, 0.0, 3.0, 4.0),
        (1.0, 0.0, 1.0, 1.0),
        (1.0, 0.0, eps_small, 1.0),          # x > 0, y = 1: tan(2 phi) bound (Eq. 14)
        (tiny, 0.0, 0.0, 0.0),
        (tiny, tiny, tiny, tiny),
        (tiny, -tiny, 2 * tiny, 3 * tiny),
        (big, 0.0, 0.0, big),
        (big, big, big, big),
        (big, -big, big, big),
        (top, tiny, tiny, 1.0),              # s = -2 with subnormal loss
        (top1, 3 * tiny, 0.0, 1.0),          # s = -1
        (top, 1.0, 1.0, top),
        (1.0, 2.0, 2.0, 4.0),                # rank 1
        (lo, hi, lo, hi),
        (np.ldexp(dtype(1), fi.minexp), 0.0, 0.0, tiny),
        (-1.0, -2.0, -3.0, -4.0),
        (1.0, 1.0, -1.0, 1.0),
    ]
    A = np.array(cases, dtype=np.float64).T
    with np.errstate(over="ignore", under="ignore"):
        return np.ascontiguousarray(A.astype(dtype))


def normal_batch_device(n: int, rows: int, seed: int, device="cuda", dtype=None):
    """i.i.d. N(0,1) entries of shape (rows, n), drawn on the GPU by torch's
    seeded Philox generator (for workloads too large to draw on the host, such
    as the 2048-batch Kogbetliantz sequence)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn((rows, n), generator=g, device=device, dtype=dtype or torch.float64)


def round_robin_pairs(m: int, step: int) -> np.ndarray:
    """Pivot pairs (p_0, q_0, p_1, q_1, ...) of step `step` (0 .. m-2) of the
    round-robin tournament ordering of 0 .. m-1 (m even): every index meets
    every other exactly once in m - 1 steps, a cyclic parallel ordering for
    the Kogbetliantz step of Sec. 1 (the paper leaves the ordering open).
    int32 array of m entries, each pair with p < q."""
    others = list(range(1, m))
    r = step % (m - 1)
    players = [0] + others[r:] + others[:r]
    pairs = []
    for i in range(m // 2):
        a, b = players[i], players[m - 1 - i]
        pairs += [min(a, b), max(a, b)]
    return np.array(pairs, dtype=np.int32)
