// Host check of the integer-pipe IEEE division and square root
// (paper_2005_07403_gb300/csrc/svd2_softfp.cuh), in their general and
// branch-free forms (the latter where they do not flag the operands), against
// the CPU's correctly rounded hardware division and square root, bit for bit.  The header's host
// build replaces the FP32 approximate reciprocals by the nearest float moved
// by up to +-2 units in the last place, wider than the GPU instructions'
// error.  Usage: softfp_host_check <count per class> <seed>; prints the
// number of checked cases and mismatches, exits 1 on any mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>

#include "svd2_softfp.cuh"

using svd2::sfp::dbits;
using svd2::sfp::dval;

static uint64_t sm64(uint64_t &s) {  // SplitMix64
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static long long checked = 0, bad = 0;

// the branch-free forms: where they do not flag the operands, the same bits
static void chk_div_fast(double a, double b, double h) {
  unsigned flag = 0;
  const double r = svd2::sfp::div_fast(a, b, flag);
  ++checked;
  if (!flag && dbits(r) != dbits(h)) {
    if (bad < 10) std::printf("div_fast mismatch a=%a b=%a soft=%a hw=%a\n", a, b, r, h);
    ++bad;
  }
}
static void chk_sqrt_fast(double x, double h) {
  unsigned flag = 0;
  const double r = svd2::sfp::sqrt_fast(x, flag);
  ++checked;
  if (!flag && dbits(r) != dbits(h)) {
    if (bad < 10) std::printf("sqrt_fast mismatch x=%a soft=%a hw=%a\n", x, r, h);
    ++bad;
  }
}
static void chk_div(double a, double b) {
  const double r = svd2::sfp::div_rn(a, b), h = a / b;
  ++checked;
  if (dbits(r) != dbits(h) && !(std::isnan(r) && std::isnan(h))) {
    if (bad < 10) std::printf("div mismatch a=%a b=%a soft=%a hw=%a\n", a, b, r, h);
    ++bad;
  }
  chk_div_fast(a, b, h);
}
static void chk_sqrt(double x) {
  const double r = svd2::sfp::sqrt_rn(x), h = std::sqrt(x);
  ++checked;
  if (dbits(r) != dbits(h) && !(std::isnan(r) && std::isnan(h))) {
    if (bad < 10) std::printf("sqrt mismatch x=%a soft=%a hw=%a\n", x, r, h);
    ++bad;
  }
  chk_sqrt_fast(x, h);
}

static void chk_d2f(double x) {
  const float r = svd2::sfp::d2f(x), h = (float)x;
  ++checked;
  uint32_t br, bh;
  std::memcpy(&br, &r, 4);
  std::memcpy(&bh, &h, 4);
  if (br != bh && !(std::isnan(r) && std::isnan(h))) {
    if (bad < 10) std::printf("d2f mismatch x=%a soft=%a hw=%a\n", x, (double)r, (double)h);
    ++bad;
  }
}
static void chk_f2d(uint32_t b) {
  float f;
  std::memcpy(&f, &b, 4);
  const double r = svd2::sfp::f2d(f), h = (double)f;
  ++checked;
  if (dbits(r) != dbits(h) && !(std::isnan(r) && std::isnan(h))) {
    if (bad < 10) std::printf("f2d mismatch x=%a soft=%a hw=%a\n", (double)f, r, h);
    ++bad;
  }
}

// the integer-pipe multiplication: where it does not flag the operands, the
// CPU's product; it flags no pair of normal operands whose product is normal
// and above the smallest normal (a product rounded up to the smallest normal
// from below it is flagged: its exponent is below the range before rounding)
static long long mul_flagged = 0;
static void chk_mul(double a, double b) {
  unsigned flag = 0;
  const double r = svd2::sfp::mul_fast(a, b, flag), h = a * b;
  ++checked;
  const bool normal_in = (std::fpclassify(a) == FP_NORMAL || a == 0) &&
                         (std::fpclassify(b) == FP_NORMAL || b == 0);
  const bool normal_out = (std::fpclassify(h) == FP_NORMAL && std::fabs(h) > 0x1p-1022) ||
                          (h == 0 && (a == 0 || b == 0));
  if (flag) ++mul_flagged;
  if ((!flag && dbits(r) != dbits(h)) || (flag && normal_in && normal_out)) {
    if (bad < 10) std::printf("mul_fast mismatch a=%a b=%a soft=%a hw=%a flag=%u\n", a, b, r, h, flag);
    ++bad;
  }
}

// the float-quotient division: where it does not flag the operands, the CPU's
// double quotient of the widened floats, given the CPU's float quotient
static long long ff_checked = 0;
static void chk_div_ff(float a, float b) {
  const float q32 = a / b;
  unsigned flag = 0;
  const double r = svd2::sfp::div_ff(a, b, q32, flag), h = (double)a / (double)b;
  ++checked;
  if (!flag) ++ff_checked;
  if (!flag && dbits(r) != dbits(h)) {
    if (bad < 10) std::printf("div_ff mismatch a=%a b=%a soft=%a hw=%a\n", (double)a, (double)b, r, h);
    ++bad;
  }
}
static float fmk(uint32_t sign, uint32_t bexp, uint32_t frac) {
  return svd2::sfp::fval((sign << 31) | ((bexp & 0xffu) << 23) | (frac & 0x7fffffu));
}

// a double with the given biased exponent and mantissa bits
static double mk(uint64_t sign, uint64_t bexp, uint64_t frac) {
  return dval((sign << 63) | ((bexp & 0x7ff) << 52) | (frac & 0xfffffffffffffull));
}

int main(int argc, char **argv) {
  const long long n = argc > 1 ? std::atoll(argv[1]) : 1000000;
  uint64_t s = argc > 2 ? std::strtoull(argv[2], nullptr, 10) : 1;
  const uint64_t specials[] = {0, 1, 2, 3, 0xfffffffffffffull, 0xffffffffffffeull,
                               0x8000000000000ull, 0x7ffffffffffffull, 0x0000000000001ull,
                               0xaaaaaaaaaaaaaull, 0x5555555555555ull, 0xfffff00000000ull,
                               0x00000fffffffful, 0x1000000000000ull};
  // conversion boundaries: FLT_MAX and the tie above it (rounds to infinity),
  // the smallest normal float and the binade below it, zeros, infinities, NaN
  for (int sg = 0; sg < 2; ++sg) {
    for (uint64_t fr : {0xfffffe0000000ull, 0xfffffefffffffull, 0xffffff0000000ull,
                        0xfffffffffffffull, 0ull, 0x0000010000000ull, 0x0000001ull})
      for (uint64_t e : {1150ull, 1151ull, 1152ull, 895ull, 896ull, 897ull, 0ull, 2047ull})
        chk_d2f(mk(sg, e, fr));
    for (uint32_t b : {0u, 1u, 0x7fffffu, 0x800000u, 0x7f7fffffu, 0x7f800000u, 0x7fc00000u,
                       0x7f800001u, 0x3f800000u})
      chk_f2d(b | (sg ? 0x80000000u : 0u));
  }
  // zero numerators over normal divisors, both signs: the fast form's signed zero
  for (int sa = 0; sa < 2; ++sa)
    for (int sb = 0; sb < 2; ++sb)
      for (uint64_t e : {1ull, 1023ull, 2046ull}) chk_div(mk(sa, 0, 0), mk(sb, e, 0x123456789abcull));
  // float quotients: zero numerators, exact quotients, the binade edges
  for (uint32_t fb : {0u, 1u, 0x7fffffu, 0x400000u, 0x555555u})
    for (uint32_t eb : {1u, 64u, 127u, 200u, 254u}) {
      chk_div_ff(0.0f, fmk(0, eb, fb));
      chk_div_ff(-0.0f, fmk(1, eb, fb));
      for (uint32_t fa : {0u, 1u, 0x7fffffu, 0x400000u, fb, fb ^ 1u, fb + 1u})
        for (uint32_t ea : {1u, 100u, 127u, 128u, 254u}) chk_div_ff(fmk(0, ea, fa), fmk(0, eb, fb));
    }
  // products: zeros of both signs, exact powers of two, the ends of the
  // exponent range (results at the normal boundary and the overflow threshold)
  for (int sa = 0; sa < 2; ++sa)
    for (int sb = 0; sb < 2; ++sb)
      for (uint64_t e : {1ull, 1023ull, 2046ull}) {
        chk_mul(mk(sa, 0, 0), mk(sb, e, 0x123456789abcull));
        chk_mul(mk(sa, e, 0xfffffffffffffull), mk(sb, 0, 0));
        chk_mul(mk(sa, e, 0), mk(sb, 1023, 0));
        for (uint64_t f : {0ull, 1ull, 0xfffffffffffffull, 0x8000000000000ull})
          for (uint64_t e2 : {1ull, 2ull, 1022ull, 1023ull, 1024ull, 2045ull, 2046ull})
            chk_mul(mk(sa, e, f), mk(sb, e2, 0xfffffffffffffull ^ f));
      }
  for (long long i = 0; i < n; ++i) {
    {
      // products: random significands with exponents around 1, anywhere in the
      // range (under- and overflowing results flagged), structured mantissas,
      // and halfway cases (a significand times 1 + 2^-k)
      const uint64_t e1 = 1023 + (sm64(s) % 64) - 32, e2 = 1023 + (sm64(s) % 64) - 32;
      chk_mul(mk(sm64(s) & 1, e1, sm64(s)), mk(sm64(s) & 1, e2, sm64(s)));
      chk_mul(mk(sm64(s) & 1, 1 + sm64(s) % 2046, sm64(s)), mk(sm64(s) & 1, 1 + sm64(s) % 2046, sm64(s)));
      chk_mul(mk(0, e1, specials[sm64(s) % 14]), mk(1, e2, specials[sm64(s) % 14]));
      chk_mul(mk(0, e1, sm64(s) << 20), mk(0, e2, (1ull << (sm64(s) % 52))));
      chk_mul(dval(sm64(s)), dval(sm64(s)));
    }
    {
      // float quotients: random significands, exponents near each other and
      // anywhere, numerators below the divisor (the method's use), small
      // integer multiples (exact quotients), runs of ones
      const uint32_t r1 = (uint32_t)sm64(s), r2 = (uint32_t)sm64(s), r3 = (uint32_t)sm64(s);
      const uint32_t eb = 1 + r3 % 254, ea = 1 + (r3 >> 8) % 254;
      chk_div_ff(fmk(r1 >> 31, ea, r1), fmk(r2 >> 31, eb, r2));
      const uint32_t en = eb - 40 + (r3 >> 16) % 41;
      if (en >= 1 && en <= 254) chk_div_ff(fmk(0, en, r1), fmk(0, eb, r2));
      chk_div_ff(fmk(0, eb, r1 | 0x7ff000u), fmk(0, eb, r2 | 0x7ff000u));
      const float b = fmk(0, 100 + r3 % 50, r2), k = (float)(1 + r1 % 4096);
      chk_div_ff(b * k, b);
      chk_div_ff(fmk(0, eb, 0x7fffffu ^ (1u << (r1 % 23))), fmk(0, eb, r2));
    }
    // conversions: any float pattern; doubles around the float range (float
    // subnormal results, overflow), with the 29 dropped bits random, exactly
    // half an ulp (ties), or half an ulp +-1
    chk_f2d((uint32_t)sm64(s));
    chk_d2f(dval(sm64(s)));
    const uint64_t ec = 896 - 26 + sm64(s) % 284, fc = sm64(s);
    const uint64_t drop[] = {fc & 0x1fffffffull, 0x10000000ull, 0x0fffffffull, 0x10000001ull, 0};
    const uint64_t fr = (fc & ~0x1fffffffull) | drop[sm64(s) % 5];
    chk_d2f(mk(sm64(s) & 1, ec, fr));
    // uniform random bit patterns (any class: normal, subnormal, zero, inf, NaN)
    chk_div(dval(sm64(s)), dval(sm64(s)));
    chk_sqrt(dval(sm64(s)));
    // random mantissas, exponents near each other (the method's typical use)
    const uint64_t ea = 1023 + (sm64(s) % 64) - 32, eb = 1023 + (sm64(s) % 64) - 32;
    chk_div(mk(sm64(s) & 1, ea, sm64(s)), mk(sm64(s) & 1, eb, sm64(s)));
    chk_sqrt(mk(0, ea, sm64(s)));
    // structured mantissas (all ones, single bits, runs)
    const uint64_t fa = specials[sm64(s) % 14] ^ ((sm64(s) % 4 == 0) ? (1ull << (sm64(s) % 52)) : 0);
    const uint64_t fb = specials[sm64(s) % 14] ^ ((sm64(s) % 4 == 0) ? (1ull << (sm64(s) % 52)) : 0);
    chk_div(mk(0, ea, fa), mk(0, eb, fb));
    chk_sqrt(mk(0, ea, fa));
    chk_sqrt(mk(0, ea + 1, fb));
    // exponent extremes: results near overflow and underflow, subnormal operands
    const uint64_t e1 = 1 + sm64(s) % 2046, e2 = 1 + sm64(s) % 2046;
    chk_div(mk(0, e1, sm64(s)), mk(1, e2, sm64(s)));
    chk_div(mk(0, 0, sm64(s)), mk(0, e2, sm64(s)));
    chk_sqrt(mk(0, 0, sm64(s)));
    // exact squares and neighbours: sqrt results near a representable value
    const uint64_t t = (sm64(s) >> 38) | (1ull << 25);     // 26-bit integer
    const double sq = (double)t * (double)t;               // exact
    chk_sqrt(sq);
    chk_sqrt(std::nextafter(sq, 0.0));
    chk_sqrt(std::nextafter(sq, 1e300));
    // quotients near integers: a = b * k (+-1 ulp)
    const double bb = mk(0, 1023, sm64(s));
    const double kk = (double)(1 + sm64(s) % 1000);
    const double aa = bb * kk;
    chk_div(aa, bb);
    chk_div(std::nextafter(aa, 0.0), bb);
    chk_div(std::nextafter(aa, 1e300), bb);
    // ratios within an ulp of 1, and b with short mantissas
    chk_div(std::nextafter(bb, 0.0), bb);
    chk_div(mk(0, ea, sm64(s)), mk(0, eb, (sm64(s) % 4096) << 40));
  }
  std::printf("float quotients in domain %lld\n", ff_checked);
  std::printf("checked %lld mismatches %lld\n", checked, bad);
  return bad ? 1 : 0;
}
