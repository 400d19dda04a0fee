"""Pins of the CPU oracle to facts the paper and the mathematics fix.

No expected value here comes from the CUDA path.  Each test names the passage
it checks.  The tolerances follow from the error analysis of the method (all
steps are correctly rounded operations, so sigma_max and the normwise sigma_min
carry a few eps) and are written next to each check.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_07403_gb300 import inputs
from tests.helpers import EPS32, EPS64, ZERO_S, bits_equal, hexf, read_rows, rel_err_hilo


def widen(r):
    return {k: (v.astype(np.float64) if v.dtype == np.float32 else v) for k, v in r.items()}


# ----------------------------------------------------------------- constants

def test_sqrt_max_constants():
    """Fig. 10 prints sqrt(DBL_MAX) as 1.34078079299425956E+154: the literal the
    oracle uses must be RN(sqrt(DBL_MAX)); the float bound of Sec. 7 must be
    RN(sqrt(FLT_MAX))."""
    c = oracle.constants()
    assert c["sqrt_dbl_max_literal"] == math.sqrt(np.finfo(np.float64).max)
    assert c["sqrt_dbl_max"] == c["sqrt_dbl_max_literal"]
    assert c["sqrt_dbl_max_literal"] == float.fromhex("0x1.fffffffffffffp+511")
    assert np.float32(c["sqrt_flt_max"]) == np.sqrt(np.finfo(np.float32).max)


# ------------------------------------------------------------ Eq. 2 scaling

def test_scale_exponent_golden():
    """Hand-derived s of Eq. 2 (Sec. 2.1), including the zero matrix, s = -2 and
    -1 at the top of the exponent range, and subnormals (exp2 of Sec. 2.1 is
    exact for them)."""
    for row in read_rows("scale_exponents.txt"):
        dt = np.float64 if row[0] == "f64" else np.float32
        A = np.array([[hexf(t, dt)] for t in row[1:5]], dtype=dt)
        r = oracle.svd2(A)
        assert int(r["s"][0]) == int(row[5]), row


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_scale_exponent_vs_frexp(dt):
    """Eq. 2 recomputed independently with numpy's frexp: s = h - max_ij exp2 a_ij
    with exp2 = frexp exponent - 1 (exact for subnormals), and -2 <= s."""
    if dt == np.float64:
        A = np.concatenate([inputs.random_bits(20000, 4, 3), inputs.real_mixed(8192),
                            inputs.edge_real()], axis=1)
        h, smax_allowed = 1021, 1021 + 1074
    else:
        A = np.concatenate([inputs.random_bits_f32(20000, 4, 3),
                            inputs.edge_real(np.float32)], axis=1)
        h, smax_allowed = 125, 125 + 149
    r = oracle.svd2(np.ascontiguousarray(A.astype(dt)))
    m, e = np.frexp(A.astype(np.float64) if dt == np.float32 else A)
    e = np.where(A != 0, e.astype(np.int64) - 1, np.iinfo(np.int64).min)
    emax = e.max(axis=0)
    expect = np.where(emax == np.iinfo(np.int64).min, ZERO_S, h - emax)
    assert np.array_equal(r["s"].astype(np.int64), expect)
    nz = r["s"] != ZERO_S
    assert r["s"][nz].min() >= -2 and r["s"][nz].max() <= smax_allowed


def test_scale_exponent_complex_vs_frexp():
    """Eq. 2 over both real and imaginary parts (Fig. 3)."""
    A = np.concatenate([inputs.random_bits(20000, 8, 4), inputs.complex_scaled(4096)], axis=1)
    r = oracle.svd2(np.ascontiguousarray(A))
    _, e = np.frexp(A)
    e = np.where(A != 0, e.astype(np.int64) - 1, np.iinfo(np.int64).min)
    emax = e.max(axis=0)
    expect = np.where(emax == np.iinfo(np.int64).min, ZERO_S, 1021 - emax)
    assert np.array_equal(r["s"].astype(np.int64), expect)


# ------------------------------------------------------------- golden cases

def test_hand_cases():
    """SVDs evaluated by hand from Eq. 2 - Eq. 29 (zero matrix and a diagonal
    matrix needing both pivots), compared bit for bit, signed zeros included."""
    for row in read_rows("hand_cases.txt"):
        fields = dict(tok.split("=") for tok in row[1:])
        A = np.array([[hexf(t)] for t in fields["A"].split(",")])
        r = oracle.svd2(A)
        U = np.array([hexf(t) for t in fields["U"].split(",")])
        V = np.array([hexf(t) for t in fields["V"].split(",")])
        assert bits_equal(r["U"][:, 0], U), (row[0], r["U"][:, 0])
        assert bits_equal(r["V"][:, 0], V), (row[0], r["V"][:, 0])
        assert r["smax"][0] == hexf(fields["smax"])
        assert r["smin"][0] == hexf(fields["smin"])
        assert int(r["s"][0]) == int(fields["s"])
        assert int(r["piv"][0]) == int(fields["piv"])


def test_tan2phi_bound_case():
    """Eq. 14 - Eq. 15: for x > 0, y = 1 with x +- y rounding to +-1, the bound
    sqrt(DBL_MAX) makes tan(phi) = -1 exactly, so every entry of U and V has
    magnitude 1/sqrt(2) (U = c [[1,-1],[1,1]] and V = cos(psi) [[1,-1],[1,1]]
    with tan(psi) = RN(-1 - x) = -1)."""
    A = np.array([[1.0], [0.0], [2.0**-60], [1.0]])
    r = oracle.svd2(A)
    inv_sqrt2 = 1.0 / math.sqrt(2.0)
    assert np.all(np.abs(r["U"][:, 0]) == inv_sqrt2), r["U"][:, 0]
    assert np.all(np.abs(r["V"][:, 0]) == inv_sqrt2), r["V"][:, 0]
    # signs: U = c [[1, -1], [1, 1]]  (rows a11, a21, a12, a22)
    assert np.array_equal(np.sign(r["U"][:, 0]), [1, 1, -1, 1])
    assert np.array_equal(np.sign(r["V"][:, 0]), [1, 1, -1, 1])


def test_rank_one_exact_zero():
    """y = 0 case of the proof of Theorem 1: for the exactly rank-1 [[1,2],[2,4]],
    r''_22 = cos(alpha) fma(-1/2, 2^1020, 2^1019) = 0, so sigma_min = 0 exactly and
    sigma_max = 5 within the sigma bound."""
    A = np.array([[1.0], [2.0], [2.0], [4.0]])
    r = oracle.svd2(A, backscale=True)
    assert r["smin"][0] == 0.0
    assert abs(r["smax"][0] - 5.0) <= 4 * EPS64 * 5.0


def test_pivot_ties_strict():
    """Fig. 5 and Fig. 6 swap only on a strict '<': equal column norms or equal
    row magnitudes leave the matrix in place."""
    A = np.array([[1.0, 1.0, 2.0], [1.0, 1.0, -2.0], [1.0, -1.0, 0.0], [1.0, 1.0, 0.0]])
    r = oracle.svd2(A)
    assert list(r["piv"]) == [0, 0, 0]


# ------------------------------------------------- singular values vs truth

def _sigma_checks(A, dt, tol_max=4.0, tol_min=4.0):
    """Scaled singular values Sigma' (Eq. 17) against the binary128 closed form
    scaled by the same 2^s (exact; Sigma' is what the method returns, Sec. 2.3)."""
    eps = EPS64 if dt == np.float64 else EPS32
    r = widen(oracle.svd2(A.astype(dt)))
    sxh, sxl, snh, snl = oracle.truth(A.astype(np.float64), r["s"])
    z = r["s"] == ZERO_S
    ok = ~z
    ex = rel_err_hilo(r["smax"][ok], sxh[ok], sxl[ok])
    en = np.abs((r["smin"][ok] - snh[ok]) - snl[ok]) / sxh[ok]
    assert ex.max() <= tol_max * eps, ex.max() / eps
    assert en.max() <= tol_min * eps, en.max() / eps
    # zero matrices give exact zeros
    assert np.all(r["smax"][z] == 0) and np.all(r["smin"][z] == 0)
    return r


@pytest.mark.parametrize("name", ["normal", "mixed", "rbits", "edge"])
def test_sigma_vs_closed_form_real(name):
    """Singular values against the binary128 closed form of O2:
    sigma'_max within 4 eps relative, sigma'_min within 4 eps * sigma'_max."""
    A = {"normal": lambda: inputs.normal_batch(50000, 4, 21),
         "mixed": lambda: inputs.real_mixed(),
         "rbits": lambda: inputs.random_bits(50000, 4, 22),
         "edge": lambda: inputs.edge_real()}[name]()
    _sigma_checks(A, np.float64)


@pytest.mark.parametrize("name", ["normal", "cfg2", "rbits"])
def test_sigma_vs_closed_form_complex(name):
    A = {"normal": lambda: inputs.normal_batch(30000, 8, 23),
         "cfg2": lambda: inputs.complex_scaled(30000),
         "rbits": lambda: inputs.random_bits(30000, 8, 24)}[name]()
    _sigma_checks(A, np.float64)


def test_sigma_vs_closed_form_float():
    """Single precision (Sec. 1, Sec. 7), against the exact singular values of
    the float input."""
    A = np.concatenate([inputs.normal_batch(50000, 4, 25, np.float32),
                        inputs.edge_real(np.float32)], axis=1)
    _sigma_checks(A, np.float32)
    Ac = inputs.normal_batch(30000, 8, 26, np.float32)
    _sigma_checks(Ac, np.float32)


def test_diagonal_closed_form():
    """x = 0 case of Theorem 1's proof: for diagonal A all tangents vanish, so
    sigma = sorted |a_ii| exactly and U, V are signed permutations."""
    rng = np.random.default_rng(31)
    d = rng.standard_normal((2, 2000)) * np.exp2(rng.integers(-300, 300, (2, 2000)))
    A = np.stack([d[0], np.zeros(2000), np.zeros(2000), d[1]])
    r = oracle.svd2(A, backscale=True)
    assert np.array_equal(r["smax"], np.maximum(np.abs(d[0]), np.abs(d[1])))
    assert np.array_equal(r["smin"], np.minimum(np.abs(d[0]), np.abs(d[1])))
    for X in (r["U"], r["V"]):
        assert np.all(np.isin(np.abs(X), [0.0, 1.0]))
        assert np.all(np.abs(X).sum(axis=0) == 2.0)


def test_rotation_closed_form():
    """A = R(t1) diag(s1, s2) R(t2)^T with well separated s1 > s2: the singular
    vectors are the rotation columns up to sign."""
    rng = np.random.default_rng(32)
    n = 4000
    t1, t2 = rng.uniform(0, 2 * np.pi, (2, n))
    s1 = rng.uniform(1.0, 2.0, n)
    s2 = s1 * rng.uniform(0.0, 0.5, n)
    c1, sn1, c2, sn2 = np.cos(t1), np.sin(t1), np.cos(t2), np.sin(t2)
    A = np.stack([c1 * s1 * c2 + sn1 * s2 * sn2, sn1 * s1 * c2 - c1 * s2 * sn2,
                  c1 * s1 * sn2 - sn1 * s2 * c2, sn1 * s1 * sn2 + c1 * s2 * c2])
    r = oracle.svd2(A, backscale=True)
    # first columns: u1 = +-(c1, s1), v1 = +-(c2, s2)
    for X, c, s in ((r["U"], c1, sn1), (r["V"], c2, sn2)):
        dot = np.abs(X[0] * c + X[1] * s)
        assert np.all(np.abs(dot - 1.0) < 1e-13)
    assert np.all(np.abs(r["smax"] - s1) <= 1e-14 * s1)


# ------------------------------------------------- backward error (Sec. 8)

@pytest.mark.parametrize("name,dt", [("normal", np.float64), ("mixed", np.float64),
                                     ("rbits", np.float64), ("cnormal", np.float64),
                                     ("cfg2", np.float64), ("crbits", np.float64),
                                     ("fnormal", np.float32), ("fcnormal", np.float32),
                                     ("frbits", np.float32)])
def test_backward_error_orthogonality(name, dt):
    """rho (Eq. 33) <= 8 eps, delta (Eq. 34) and eta (Eq. 35) <= 16 eps, in
    binary128, for the scaled-and-returned Sigma', s convention (Sec. 2.3)."""
    A = {"normal": lambda: inputs.normal_batch(50000, 4, 41),
         "mixed": lambda: inputs.real_mixed(),
         "rbits": lambda: inputs.random_bits(50000, 4, 42),
         "cnormal": lambda: inputs.normal_batch(30000, 8, 43),
         "cfg2": lambda: inputs.complex_scaled(30000),
         "crbits": lambda: inputs.random_bits(30000, 8, 44),
         "fnormal": lambda: inputs.normal_batch(50000, 4, 45, np.float32),
         "fcnormal": lambda: inputs.normal_batch(30000, 8, 46, np.float32),
         "frbits": lambda: inputs.random_bits_f32(50000, 4, 47)}[name]()
    eps = EPS64 if dt == np.float64 else EPS32
    r = widen(oracle.svd2(A))
    m = oracle.metrics(A.astype(np.float64), r["U"], r["V"], r["smax"], r["smin"], r["s"])
    assert m["rho"].max() <= 8 * eps, m["rho"].max() / eps
    assert m["delta"].max() <= 16 * eps, m["delta"].max() / eps
    assert m["eta"].max() <= 16 * eps, m["eta"].max() / eps


def test_theorem1_on_random_bits():
    """Theorem 1: for every finite input, infinity > sigma'_max >= sigma'_min >= 0;
    and, as observed in Sec. 8, back-scaling random-bit data overflows for some
    matrices, which is why Sigma' and s are returned."""
    A = inputs.random_bits(100000, 4, 51)
    r = oracle.svd2(A)
    assert np.all(np.isfinite(r["smax"])) and np.all(np.isfinite(r["smin"]))
    assert np.all(r["smax"] >= r["smin"]) and np.all(r["smin"] >= 0)
    for X in (r["U"], r["V"]):
        assert np.all(np.isfinite(X))
    # Back-scaling is unsafe (Sec. 2.3, Sec. 8): all entries DBL_MAX give a finite
    # sigma'_max but sigma_max = 2 DBL_MAX overflows once 2^-s is applied.
    big = np.full((4, 1), np.finfo(np.float64).max)
    r1 = oracle.svd2(big)
    assert np.isfinite(r1["smax"][0]) and int(r1["s"][0]) == -2
    with np.errstate(over="ignore"):
        rb = oracle.svd2(big, backscale=True)
    assert np.isinf(rb["smax"][0])
    Ac = inputs.random_bits(50000, 8, 52)
    rc = oracle.svd2(Ac)
    assert np.all(np.isfinite(rc["smax"])) and np.all(rc["smax"] >= rc["smin"])
    assert np.all(rc["smin"] >= 0)


def test_v_structure_eq29():
    """Eq. 29 fixes V = P_c cos(psi) [[1, tan psi], [-d~ tan psi, d~]] with
    1/sqrt(3) <= cos(psi) <= 1 and -sqrt(2) <= tan(psi) <= 0 (Theorem 1): the
    un-permuted first row of V is (cos psi, cos psi tan psi) and the other row
    has the same magnitudes, swapped."""
    A = inputs.normal_batch(50000, 4, 53)
    r = oracle.svd2(A)
    pc = (r["piv"] & 1).astype(bool)
    V = r["V"]
    v11 = np.where(pc, V[1], V[0])   # (1,1) before P_c
    v12 = np.where(pc, V[3], V[2])
    v21 = np.where(pc, V[0], V[1])
    v22 = np.where(pc, V[2], V[3])
    assert np.all(v11 >= 1 / math.sqrt(3) * (1 - 4 * EPS64)) and np.all(v11 <= 1.0)
    assert np.all(v12 <= 0)
    assert np.all(np.abs(v12) <= math.sqrt(2) * v11 * (1 + 4 * EPS64))
    assert np.array_equal(np.abs(v21), np.abs(v12))
    assert np.array_equal(np.abs(v22), v11)


# ---------------------------------------------------------- complex vs real

def test_complex_with_zero_imaginary_parts_matches_real():
    """With zero imaginary parts every step of the complex path (Eq. 1, Eq. 4,
    Eq. 5, Eq. 8, Eq. 9) reduces to the real one of Eq. 10: hypot(a, 0) = |a|,
    e^{i arg a} = sign a.  Singular values and s agree bit for bit.  U and V
    agree bit for bit where no intermediate is a signed zero: the real path
    applies signs by XOR (Fig. 7) and keeps -0 where the complex fma of Eq. 5
    gives -0 + +0 = +0, so a zero entry may pick the other, equally valid,
    sign convention; those matrices are checked by their backward error."""
    Ar = np.concatenate([inputs.normal_batch(20000, 4, 61), inputs.real_mixed(8192)], axis=1)
    Ac = np.zeros((8, Ar.shape[1]))
    Ac[0::2] = Ar
    rr = oracle.svd2(np.ascontiguousarray(Ar))
    rc = oracle.svd2(Ac)
    assert np.array_equal(rr["smax"], rc["smax"]) and np.array_equal(rr["smin"], rc["smin"])
    assert np.array_equal(rr["s"], rc["s"]) and np.array_equal(rr["piv"], rc["piv"])
    nz = (Ar != 0).all(axis=0)
    assert nz.mean() > 0.8
    assert np.array_equal(rr["U"][:, nz], rc["U"][0::2, nz])
    assert np.array_equal(rr["V"][:, nz], rc["V"][0::2, nz])
    assert np.all(rc["U"][1::2] == 0) and np.all(rc["V"][1::2] == 0)
    m = oracle.metrics(Ac, rc["U"], rc["V"], rc["smax"], rc["smin"], rc["s"])
    assert m["rho"].max() <= 8 * EPS64


def test_complex_phase_invariance():
    """A and e^{i theta} A have the same singular values."""
    A = inputs.normal_batch(20000, 8, 62)
    th = np.random.default_rng(63).uniform(0, 2 * np.pi, A.shape[1])
    c, s = np.cos(th), np.sin(th)
    B = np.empty_like(A)
    B[0::2] = A[0::2] * c - A[1::2] * s
    B[1::2] = A[0::2] * s + A[1::2] * c
    ra = oracle.svd2(A, backscale=True)
    rb = oracle.svd2(B, backscale=True)
    assert np.all(np.abs(ra["smax"] - rb["smax"]) <= 16 * EPS64 * ra["smax"])
    assert np.all(np.abs(ra["smin"] - rb["smin"]) <= 16 * EPS64 * ra["smax"])


# ------------------------------------------------------ brute force (mpmath)

def test_brute_force_small_integers():
    """All 7^4 real matrices with entries in {-3..3}, at three binades (2^0,
    2^600, 2^-540): singular values against a 60-digit mpmath evaluation of the
    closed form, backward error against binary128."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    vals = np.arange(-3, 4, dtype=np.float64)
    grid = np.array(np.meshgrid(vals, vals, vals, vals, indexing="ij")).reshape(4, -1)
    exact = []
    for k in range(grid.shape[1]):
        a11, a21, a12, a22 = (mp.mpf(int(x)) for x in grid[:, k])
        F2 = a11**2 + a21**2 + a12**2 + a22**2
        d = abs(a11 * a22 - a12 * a21)
        smax = (mp.sqrt(F2 + 2 * d) + mp.sqrt(F2 - 2 * d)) / 2
        smin = d / smax if smax > 0 else mp.mpf(0)
        exact.append((smax, smin))
    for k2 in (0, 600, -540):
        A = np.ascontiguousarray(np.ldexp(grid, k2))
        r = oracle.svd2(A, backscale=True)
        for k in range(grid.shape[1]):
            smax, smin = exact[k]
            smax = smax * mp.mpf(2) ** k2
            smin = smin * mp.mpf(2) ** k2
            if smax == 0:
                assert r["smax"][k] == 0 and r["smin"][k] == 0
                continue
            assert abs(mp.mpf(r["smax"][k]) - smax) <= 4 * EPS64 * smax
            assert abs(mp.mpf(r["smin"][k]) - smin) <= 4 * EPS64 * smax
        r2 = oracle.svd2(A)
        m = oracle.metrics(A, r2["U"], r2["V"], r2["smax"], r2["smin"], r2["s"])
        assert m["rho"].max() <= 8 * EPS64
        assert max(m["delta"].max(), m["eta"].max()) <= 16 * EPS64


# ------------------------------------------------ FP32 form with FP64 re-run

def test_rerun_form_consistency():
    """The FP32 form flags exactly the matrices with sigma'_min < 2^tau
    sigma'_max in float; their results are the double method's rounded to
    float, so their singular values are within one float rounding (2^-24
    relative, plus the scale change) of the double method's."""
    A32, ill = inputs.real_fp32_illcond(40000)
    tau = -10
    r32 = oracle.svd2(A32)
    rr = oracle.svd2_rerun(A32, tau)
    flag = r32["smin"] < np.float32(2.0**tau) * r32["smax"]
    assert np.array_equal(rr["flagged"].astype(bool), flag)
    assert rr["count"] == int(flag.sum())
    assert np.array_equal(rr["s"], r32["s"])
    nf = ~flag
    assert np.array_equal(rr["smax"][nf], r32["smax"][nf])
    assert np.array_equal(rr["U"][:, nf], r32["U"][:, nf])
    r64 = oracle.svd2(A32.astype(np.float64), backscale=True)
    back = np.ldexp(rr["smin"][flag].astype(np.float64), -rr["s"][flag])
    rel = np.abs(back - r64["smin"][flag]) / r64["smin"][flag]
    assert rel.max() <= 2.0**-24 * 1.0001
    assert ill[flag].mean() > 0.5      # the ill-conditioned class dominates the re-runs


# --------------------------------------------------------------- the adjoint

def _loss(A, gU, gV, gS):
    r = oracle.svd2(A, backscale=True)
    L = (gU * r["U"]).sum(axis=0) + (gV * r["V"]).sum(axis=0) + gS[0] * r["smax"] + gS[1] * r["smin"]
    return L, r["piv"]


def test_adjoint_vs_finite_differences():
    """Central differences (h = 1e-6) of the oracle's own forward map, on
    matrices whose relative singular-value gap is >= 1e-3 and whose pivot bits
    do not change at A +- h E_ij."""
    g = inputs.grad_batch(3000, seed=71)
    A, gU, gV, gS = g["A"], g["gU"], g["gV"], g["gS"]
    keep = ~g["small_gap"]
    A, gU, gV, gS = (np.ascontiguousarray(x[:, keep]) for x in (A, gU, gV, gS))
    r = oracle.svd2(A, backscale=True)
    gA = oracle.bwd(r["U"], r["V"], r["smax"], r["smin"], gU, gV, gS[0], gS[1], 2.0**-40)
    h = 1e-6
    _, piv0 = _loss(A, gU, gV, gS)
    fd = np.empty_like(A)
    same = np.ones(A.shape[1], bool)
    for e in range(4):
        Ap = A.copy()
        Am = A.copy()
        Ap[e] += h
        Am[e] -= h
        Lp, pp = _loss(Ap, gU, gV, gS)
        Lm, pm = _loss(Am, gU, gV, gS)
        fd[e] = (Lp - Lm) / (2 * h)
        same &= (pp == piv0) & (pm == piv0)
    gap = (r["smax"] - r["smin"]) / r["smax"]
    scale = np.abs(gA).max(axis=0) + 1.0
    err = np.abs(fd - gA).max(axis=0) / scale
    # FD truncation ~ h^2 |L'''| ~ h^2 / gap^2; rounding ~ eps / h
    tol = 1e-7 + 1e-10 / gap**2
    assert same.mean() > 0.95
    assert np.all(err[same] <= tol[same]), (err[same] / tol[same]).max()


def test_adjoint_vs_binary128_reference():
    """The double adjoint evaluated on the double oracle's outputs agrees with
    the binary128 reference gradient (method and adjoint both in binary128) to
    eps times the conditioning 1/gap of the singular vectors."""
    g = inputs.grad_batch(20000, seed=72)
    A, gU, gV, gS = g["A"], g["gU"], g["gV"], g["gS"]
    delta = 2.0**-40
    r = oracle.svd2(A, backscale=True)
    gA = oracle.bwd(r["U"], r["V"], r["smax"], r["smin"], gU, gV, gS[0], gS[1], delta)
    hi, lo = oracle.refgrad(A, gU, gV, gS[0], gS[1], delta)
    gap = (r["smax"] - r["smin"]) / r["smax"]
    big = gap >= 1e-3
    err = np.abs((gA - hi) - lo).max(axis=0) / (np.abs(hi).max(axis=0) + 1)
    assert np.all(err[big] <= 64 * EPS64 / gap[big] ** 2)


def test_adjoint_safeguard():
    """With equal singular values the safeguarded factor is 0 instead of a
    division by zero; for gaps far above delta it equals 1/(s1 - s2)."""
    U = np.array([[1.0], [0.0], [0.0], [1.0]])
    V = U.copy()
    gU = np.array([[0.0], [0.0], [1.0], [0.0]])
    gV = np.zeros((4, 1))
    one = np.array([1.0])
    gA = oracle.bwd(U, V, one, one, gU, gV, np.zeros(1), np.zeros(1), 1e-8)
    assert np.all(np.isfinite(gA))
    # a = J12 - J21 = 1, b = 0, s1 = 2, s2 = 1: m12 = 1/6 - 1/2, m21 = -1/6 - 1/2
    gA = oracle.bwd(U, V, np.array([2.0]), one, gU, gV, np.zeros(1), np.zeros(1), 1e-8)
    assert np.allclose(gA[:, 0], [0.0, -1 / 6 - 0.5, 1 / 6 - 0.5, 0.0], rtol=1e-12, atol=0)


@pytest.mark.parametrize("rows,dt", [(4, np.float64), (4, np.float32), (8, np.float64),
                                     (8, np.float32)])
def test_adjoint_equal_singular_values_without_safeguard(rows, dt):
    """rel_delta = 0 turns the safeguard off, where g / (s1 (g^2 + 0)) reads 0/0
    at s1 = s2 (a multiple of an orthogonal or unitary matrix).  The adjoint
    then takes the value the safeguard has at g = 0 for every rel_delta > 0,
    namely 0 for the rotation term: finite, and bit-identical to rel_delta > 0."""
    rng = np.random.default_rng(7)
    n = 64
    U = rng.standard_normal((rows, n)).astype(dt)
    V = rng.standard_normal((rows, n)).astype(dt)
    s = np.abs(rng.standard_normal(n)).astype(dt) + dt(0.5)
    gU, gV = rng.standard_normal((2, rows, n)).astype(dt)
    g1, g2 = rng.standard_normal((2, n)).astype(dt)
    a0 = oracle.bwd(U, V, s, s, gU, gV, g1, g2, 0.0)
    a1 = oracle.bwd(U, V, s, s, gU, gV, g1, g2, 1e-3)
    assert np.all(np.isfinite(a0))
    assert bits_equal(a0, a1)


# ----------------------------------------------------------- the generators

def test_generators_shapes_and_classes():
    A = inputs.real_mixed(4096)
    cls = inputs.real_mixed_classes(4096)
    assert A.shape == (4, 4096) and (cls >= 0).sum() == 512
    assert np.all(A[:, cls == 0] == 0)
    assert np.all(A[1, cls == 2] == 0)
    B = inputs.complex_scaled(1000)
    assert B.shape == (8, 1000) and np.all(np.isfinite(B))
    C, ill = inputs.real_fp32_illcond(1000)
    assert C.dtype == np.float32 and ill.sum() == 100
    # complex ill-conditioned members: singular values 1 and 10^-u, u in [2, 12]
    Z, zill = inputs.complex_fp32_illcond(2000, seed=7)
    assert Z.shape == (8, 2000) and Z.dtype == np.float32 and zill.sum() == 200
    Zc = Z.astype(np.float64)[0::2] + 1j * Z.astype(np.float64)[1::2]   # a11, a21, a12, a22
    M = np.stack([np.stack([Zc[0], Zc[2]], -1), np.stack([Zc[1], Zc[3]], -1)], -2)
    sv = np.linalg.svd(M[zill], compute_uv=False)
    assert np.abs(sv[:, 0] - 1).max() < 1e-6 and (sv[:, 1] / sv[:, 0]).max() < 0.011
    lens, cplx = inputs.kog_batches()
    assert lens.size == 2048 and lens.min() >= 16 and lens.max() <= 2**20
    assert np.array_equal(inputs.normal_batch(10, 4, 5), inputs.normal_batch(10, 4, 5))


# -------------------------------------- FP32 form with the FP64 tangent step

def _tan64_truth_errors(o, A32, tau):
    """Relative errors, in units of 2^-24, of the FP32-with-FP64-tangent form
    (oracle build ``o``) against the binary128 closed form of the float input
    (sigma_max, sigma_min) and against the pinned double method (sigma_min),
    plus the exact sigma_min / sigma_max and the form's own result."""
    u = 2.0**-24
    r = o.svd2_tan64(A32, tau)
    A64 = A32.astype(np.float64)
    sxh, sxl, snh, snl = o.truth(A64, r["s"])
    with np.errstate(all="ignore"):
        ex = np.abs((r["smax"].astype(np.float64) - sxh) - sxl) / sxh / u
        en = np.abs((r["smin"].astype(np.float64) - snh) - snl) / snh / u
        d = o.svd2(A64, backscale=True)
        back = np.ldexp(r["smin"].astype(np.float64), -r["s"])
        e64 = np.abs(back - d["smin"]) / d["smin"] / u
        ratio = (snh + snl) / (sxh + sxl)
    return r, ex, en, e64, ratio


def test_tan64_form_pins():
    """The FP32 form that evaluates the tangent step of Eq. 6 - Eq. 7 in double
    when |r''_22| < 2^tau r11:
    - matrices that do not take the step are the plain float method bit for bit;
    - the step's trigger brackets sigma_min / sigma_max: every matrix below
      2^(tau-1) takes it, none above 2^tau does (r11 <= sigma_max <= sqrt(2) r11
      and sigma_max sigma_min = r11 r22, so r22 / r11 is within a factor 2);
    - in the real case only the quotient tan(alpha) is rounded before the
      cancellation of Eq. 7, so with it in double sigma_min is as accurate as
      float can hold wherever the double method is: within 8 units of 2^-24 of
      the binary128 closed form up to kappa = 2^24 (the double method's own
      error there is below 2^-29), and within 8 units of the double method at
      every kappa of the batch (up to 10^12)."""
    A32, ill = inputs.real_fp32_illcond(60000, seed=2024)
    tau = -4
    r, ex, en, e64, ratio = _tan64_truth_errors(oracle._default(), A32, tau)
    w = r["wide"].astype(bool)
    assert r["count"] == int(w.sum())
    p = oracle.svd2(A32)
    for k in ("U", "V", "smax", "smin"):
        assert bits_equal(r[k][..., ~w], p[k][..., ~w]), k
    assert np.array_equal(r["s"], p["s"])
    assert np.all(w[ratio < 2.0**(tau - 1) * 0.999])
    assert not np.any(w & (ratio > 2.0**tau * 1.001))
    assert np.nanmax(ex) <= 8
    kappa = 1 / ratio
    sel = w & (kappa <= 2.0**24)
    assert sel.sum() > 1000 and en[sel].max() <= 8
    assert (w & (kappa > 2.0**30)).sum() > 500
    assert e64[w].max() <= 8
    # without the step the same matrices lose sigma_min entirely
    _, _, en0, _, _ = _tan64_truth_errors(oracle._default(), A32, -200)
    assert en0[w & (kappa > 2.0**20)].max() > 1e3


def test_tan64_threshold_zero_and_extremes():
    """tau = 0 runs the step wherever r''_22 < r11, i.e. on every matrix but the
    zero matrix and those with r''_22 = r11; at tau = -200 it never runs and the
    form is the plain float method."""
    A = inputs.normal_batch(4096, 4, 77, np.float32)
    A[:, :16] = 0                                          # zero matrices
    A[1, 16:32] = 0                                        # upper triangular
    A[:, 32:48] = inputs.random_bits_f32(16, 4, seed=78)   # the paper's random-bit class
    r0 = oracle.svd2_tan64(A, -200)
    p = oracle.svd2(A)
    assert r0["count"] == 0
    for k in ("U", "V", "smax", "smin", "s"):
        assert bits_equal(r0[k], p[k]) if k != "s" else np.array_equal(r0[k], p[k])
    r1 = oracle.svd2_tan64(A, 0)
    zero = np.all(A == 0, axis=0)
    assert not r1["wide"][zero].any()
    assert r1["count"] > 0.9 * A.shape[1]


# ------------------------------------------- the sine-based assembly of Eq. 31

@pytest.mark.parametrize("rows,dt", [(4, np.float64), (8, np.float64), (4, np.float32),
                                     (8, np.float32)])
def test_sine_assembly_eq31(rows, dt):
    """U assembled by Eq. 31 from sin = cos tan (Sec. 7) instead of the tangent
    form of Eq. 29: the two are the same matrix in exact arithmetic, V and the
    singular values are unchanged, and the decomposition keeps the accuracy
    the paper measures (Sec. 8): rho <= 8 eps, delta and eta <= 16 eps; the
    rounding of the two forms differs by a few eps per entry."""
    eps = 2.0**-52 if dt == np.float64 else 2.0**-23
    A = inputs.normal_batch(30000, rows, 41, dt)
    if dt == np.float64:
        A = np.concatenate([A, inputs.random_bits(2000, rows, 42)], axis=1)
    t = oracle.svd2(A)
    s = oracle.svd2(A, sine=True)
    for k in ("V", "smax", "smin"):
        assert bits_equal(t[k], s[k]), k
    assert np.array_equal(t["s"], s["s"]) and np.array_equal(t["piv"], s["piv"])
    assert np.abs(t["U"].astype(np.float64) - s["U"].astype(np.float64)).max() <= 3 * eps
    d = lambda x: x.astype(np.float64)
    m = oracle.metrics(d(A), d(s["U"]), d(s["V"]), d(s["smax"]), d(s["smin"]), s["s"])
    assert m["rho"].max() <= 8 * eps
    assert max(m["delta"].max(), m["eta"].max()) <= 16 * eps


def test_sine_assembly_exact_cases():
    """Diagonal and zero matrices: alpha = phi = 0 makes every sine a signed
    zero and every cosine 1, so both assemblies are exact and agree bit for
    bit, signed zeros included; the golden hand cases hold for Eq. 31 too."""
    A = np.array([[2.0, 0.0, 0.0, -3.0], [0.0, 0.0, 0.0, 0.0], [-5.0, 0.0, 0.0, 0.5],
                  [0.0, 0.0, 0.0, 7.0]]).T.copy()
    t = oracle.svd2(A)
    s = oracle.svd2(A, sine=True)
    assert bits_equal(t["U"], s["U"]) and bits_equal(t["V"], s["V"])
    for row in read_rows("hand_cases.txt"):
        fields = dict(tok.split("=") for tok in row[1:])
        A1 = np.array([[hexf(tok)] for tok in fields["A"].split(",")])
        r = oracle.svd2(A1, sine=True)
        U = np.array([hexf(tok) for tok in fields["U"].split(",")])
        assert bits_equal(r["U"][:, 0], U), row[0]
