"""The library's double division and square root (integer/FP32 pipes) against
the GPU's own IEEE instructions, bit for bit, through svd2_arith_check."""
import numpy as np
import pytest
import torch

from paper_2005_07403_gb300 import svd2 as S

pytestmark = pytest.mark.gpu

N = 1 << 24


def _bits(n, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    hi = torch.randint(0, 2**32, (n,), generator=g, device="cuda", dtype=torch.int64)
    lo = torch.randint(0, 2**32, (n,), generator=g, device="cuda", dtype=torch.int64)
    return (hi << 32) | lo


def _with_exponent(bits, lo, hi, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    e = torch.randint(lo, hi, bits.shape, generator=g, device="cuda", dtype=torch.int64)
    frac = bits & ((1 << 52) - 1)
    sign = (bits >> 63) & 1
    return ((sign << 63) | (e << 52) | frac).view(torch.float64)


def _same(a, b):
    a = a.view(torch.int64)
    b = b.view(torch.int64)
    nan = torch.isnan(a.view(torch.float64)) & torch.isnan(b.view(torch.float64))
    return bool(torch.all((a == b) | nan).item())


@pytest.mark.parametrize("cls", ["anybits", "near", "wide", "ulp1"])
def test_division_matches_hardware(cls):
    if cls == "anybits":
        x = _bits(N, 1).view(torch.float64)
        y = _bits(N, 2).view(torch.float64)
    elif cls == "near":            # exponents near each other: the method's use
        x = _with_exponent(_bits(N, 3), 1000, 1046, 4)
        y = _with_exponent(_bits(N, 5), 1000, 1046, 6)
    elif cls == "wide":            # the whole normal range: over/underflowing quotients
        x = _with_exponent(_bits(N, 7), 1, 2047, 8)
        y = _with_exponent(_bits(N, 9), 1, 2047, 10)
    else:                          # quotients within an ulp of 1 and of small integers
        y = _with_exponent(_bits(N, 11), 1023, 1024, 12)
        k = torch.randint(1, 1000, (N,), device="cuda", dtype=torch.float64)
        x = torch.nextafter(y * k, torch.full_like(y, float("inf")))
    lib, hw = S.arith_check("div", x, y)
    torch.cuda.synchronize()
    assert _same(lib, hw), cls


@pytest.mark.parametrize("cls", ["anybits", "normal", "squares"])
def test_sqrt_matches_hardware(cls):
    if cls == "anybits":
        x = _bits(N, 21).view(torch.float64)
    elif cls == "normal":
        x = _with_exponent(_bits(N, 22), 1, 2047, 23).abs()
    else:                          # exact squares and their neighbours
        t = torch.randint(2**25, 2**26, (N // 3,), device="cuda", dtype=torch.int64).double()
        sq = t * t
        x = torch.cat([sq, torch.nextafter(sq, torch.zeros_like(sq)),
                       torch.nextafter(sq, torch.full_like(sq, float("inf")))])
    lib, hw = S.arith_check("sqrt", x)
    torch.cuda.synchronize()
    assert _same(lib, hw), cls


@pytest.mark.parametrize("cls", ["anybits", "float-range", "ties"])
def test_rounding_to_float_matches_hardware(cls):
    """Double -> float on the integer pipe (the FP64 re-run's outputs)."""
    if cls == "anybits":
        x = _bits(N, 31).view(torch.float64)
    else:                          # around the float range: subnormal results, overflow
        x = _with_exponent(_bits(N, 32), 896 - 26, 896 + 258, 33)
        if cls == "ties":          # the 29 dropped bits exactly half an ulp, or +-1 from it
            b = x.view(torch.int64) & ~((1 << 29) - 1)
            g = torch.Generator(device="cuda").manual_seed(34)
            d = torch.randint(-1, 2, b.shape, generator=g, device="cuda", dtype=torch.int64)
            x = (b | ((1 << 28) + d)).view(torch.float64)
    lib, hw = S.arith_check("d2f", x)
    torch.cuda.synchronize()
    assert _same(lib, hw), cls


def test_widening_from_float_matches_hardware():
    """Float -> double on the integer pipe, every class of float pattern."""
    x = (_bits(N, 41) & 0xFFFFFFFF).view(torch.float64)
    lib, hw = S.arith_check("f2d", x)
    torch.cuda.synchronize()
    assert _same(lib, hw)


# ------------------------------------------- single precision, branch-free forms

def _selfcheck(op, begin, count):
    r = S.fp32_selfcheck(op, begin, count)
    assert r["mismatches"] == 0, (op, hex(r["first"]), r)
    return r


def test_fp32_reciprocal_exhaustive():
    """The branch-free reciprocal equals __frcp_rn on every float in
    [2^-125, 2^125] (its stated range)."""
    lo, hi = 0x01000000, 0x7C000000          # 2^-125 .. 2^125
    r = _selfcheck("rcp", lo, hi - lo + 1)
    assert r["checked"] == hi - lo + 1


def test_fp32_sqrt_exhaustive():
    """The branch-free square root equals __fsqrt_rn on every float in
    [1, FLT_MAX] (its stated range)."""
    lo, hi = 0x3F800000, 0x7F7FFFFF
    _selfcheck("sqrt", lo, hi - lo + 1)


def test_fp32_division_significand_pairs():
    """The branch-free division equals __fdiv_rn on 2^36 significand pairs (8
    runs of 1024 consecutive significands of a spread over [1, 2), each against
    every b in [1, 2)), and on 2^32 random operand pairs inside its stated
    domain."""
    for c in range(8):
        _selfcheck("div_sig", c << 43, 1 << 33)
    r = _selfcheck("div_rand", 0, 1 << 32)
    assert r["checked"] > 1 << 28


@pytest.mark.parametrize("cls", ["near", "below", "wide", "exact"])
def test_float_quotient_division_matches_hardware(cls):
    """The double quotient of two floats completed from their float quotient
    (the tangent step of the FP32 form): where it accepts the operands, the
    hardware double division of the widened floats, bit for bit; it accepts
    every pair with normal floats and a normal float quotient."""
    if cls == "near":              # exponents near each other
        x = _with_exponent(_bits(N, 31), 1000, 1046, 32).float().double()
        y = _with_exponent(_bits(N, 33), 1000, 1046, 34).float().double()
    elif cls == "below":           # numerator below the divisor: the method's tan(alpha)
        y = _with_exponent(_bits(N, 35), 1023, 1060, 36).float().double()
        x = (y * torch.rand(N, device="cuda", dtype=torch.float64)).float().double()
    elif cls == "wide":            # the float exponent range
        x = _with_exponent(_bits(N, 37), 1023 - 126, 1023 + 127, 38).float().double()
        y = _with_exponent(_bits(N, 39), 1023 - 126, 1023 + 127, 40).float().double()
    else:                          # exact quotients: small integer multiples
        y = _with_exponent(_bits(N, 41), 1023, 1030, 42).float().double()
        k = torch.randint(1, 4096, (N,), device="cuda", dtype=torch.float64)
        x = (y * k).float().double()
    lib, hw = S.arith_check("div_ff", x, y)
    torch.cuda.synchronize()
    q = (x.float() / y.float()).abs()
    normal = (x != 0) & (q >= 2.0**-126) & torch.isfinite(q)
    flagged = torch.isnan(lib)
    assert not bool(torch.any(flagged & normal)), cls
    ok = flagged | (lib.view(torch.int64) == hw.view(torch.int64))
    assert bool(torch.all(ok)), cls
