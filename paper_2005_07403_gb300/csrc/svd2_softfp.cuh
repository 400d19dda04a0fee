// Correctly rounded (round to nearest, ties to even) IEEE double division and
// square root computed on the integer and FP32 pipes, and the conversions
// between float and double on the integer pipe (end of file).
//
// On GB300 the FP64 pipe retires 2 lanes per clock per SM, and the hardware
// IEEE double division and square root each take about ten of its slots, while
// the integer and FP32 pipes are 32-64x wider.  The 2x2 SVD needs 10 (real) or
// 24 (complex) divisions and 6 or 12 square roots per matrix, so these two
// operations decide its speed.  The routines below return exactly the IEEE
// result (the same bits as __ddiv_rn / __dsqrt_rn) for operands in their fast
// domain -- normal operands and a normal result -- and defer to the hardware
// instruction otherwise (zeros, subnormals, overflow, NaN), which keeps every
// result bit-identical to IEEE arithmetic.
//
// Method (both operations): the 53-bit significand of the result is produced
// as three digits of 24, 18 and 11 bits.  The first digit comes from the FP32
// approximate reciprocal (square root: reciprocal square root) of the top 24
// bits of the operand; each further digit is estimated in FP32 from the exact
// residual, which is kept as a wrapping 64-bit integer (its true value is
// small, so arithmetic modulo 2^64 gives it exactly).  A final exact residual
// fixes the last unit, and its comparison with half a unit rounds to nearest,
// ties to even (a square root is never exactly half way).  Conversions
// between small integers (|x| < 2^22) and FP32 use the 1.5 * 2^23 bias, so the
// only special-function-unit instruction is the approximate reciprocal.
//
// The error bounds that fix the digit sizes are stated inline; the routines
// are tested against the hardware on random, structured and near-tie operands
// on the host (with a perturbed seed) and on the GPU.
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define SFP_FN __host__ __device__ __forceinline__
#else
#define SFP_FN inline
#endif

namespace svd2 {
namespace sfp {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kAbs = 0x7fffffffffffffffull;
constexpr uint64_t kFrac = 0x000fffffffffffffull;
constexpr uint64_t kImpl = 0x0010000000000000ull;

// The bit pattern of x.  On the device it passes through an opaque register
// move: written as a plain reinterpretation, the compiler turns tests on the
// pattern (zero, normal, finite) back into floating-point comparisons, which
// run on the FP64 pipe at 1/64 of the integer rate.
SFP_FN uint64_t dbits(double x) {
#if defined(__CUDA_ARCH__)
  uint64_t u;
  asm("mov.b64 %0, %1;" : "=l"(u) : "d"(x));
  return u;
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}
SFP_FN double dval(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}
SFP_FN uint32_t fbits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
SFP_FN float fval(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}
SFP_FN float fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
SFP_FN float fadd(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}

#if !defined(__CUDA_ARCH__)
// Host stand-ins for the approximate reciprocal instructions, used only to
// test the integer logic on the CPU.  They return the float nearest to the
// exact value moved by up to +-SFP_HOST_PERTURB_ULPS units in the last place
// (a deterministic function of the argument), wider than the hardware's error.
#ifndef SFP_HOST_PERTURB_ULPS
#define SFP_HOST_PERTURB_ULPS 2
#endif
inline float host_perturb(float r, float x) {
  uint32_t h = fbits(x) * 2654435761u;
  int k = (int)((h >> 24) % (2u * SFP_HOST_PERTURB_ULPS + 1u)) - SFP_HOST_PERTURB_ULPS;
  uint32_t b = fbits(r);
  return fval((uint32_t)((int32_t)b + k));
}
#endif

// ~1/x for x in [2^22, 2^24] (an FP32 approximation good to ~2^-22 relative).
SFP_FN float rcp_approx(float x) {
#if defined(__CUDA_ARCH__)
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return host_perturb((float)(1.0 / (double)x), x);
#endif
}
// ~1/sqrt(x) for x in [2^22, 2^24].
SFP_FN float rsqrt_approx(float x) {
#if defined(__CUDA_ARCH__)
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  double s = 1.0;
  {
    // a correctly rounded double square root, then the reciprocal
    double v = (double)x;
    s = 1.0 / __builtin_sqrt(v);
  }
  return host_perturb((float)s, x);
#endif
}

// x as a float, exactly, for |x| < 2^22 (1.5 * 2^23 bias).
SFP_FN float i2f_small(int32_t x) { return fadd(fval(0x4B400000u + (uint32_t)x), -12582912.0f); }
// the nearest integer to y, for |y| < 2^22.
SFP_FN int32_t f2i_small(float y) { return (int32_t)(fbits(fadd(y, 12582912.0f)) - 0x4B400000u); }
// the integer nearest to a float y in about [2^23 - 8, 2^24 + 8], clamped to [2^23, 2^24 - 1].
SFP_FN uint32_t f_to_u24_clamped(float y) {
  const float c = y < 8388608.0f ? 8388608.0f : (y > 16777215.0f ? 16777215.0f : y);
  return (fbits(c) & 0x7FFFFFu) | 0x800000u;
}

// The hardware instructions, for the operands outside the fast domain.
SFP_FN double hw_div(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __ddiv_rn(a, b);
#else
  return a / b;
#endif
}
SFP_FN double hw_sqrt(double a) {
#if defined(__CUDA_ARCH__)
  return __dsqrt_rn(a);
#else
  return __builtin_sqrt(a);
#endif
}

// Wrapping 64-bit product of a signed and an unsigned operand (the true
// values of the residuals below are small; only their low 64 bits are formed).
SFP_FN uint64_t mulw(int64_t a, uint64_t b) { return (uint64_t)a * b; }

// RN(a / b) for a, b normal with the quotient's exponent e0 - 1 or e0 in
// [1, 2045] (e0 = ea - eb + 1023): the significand quotient by three integer
// digits, sign and exponent attached.
SFP_FN double div_core(uint64_t ua, uint64_t ub, uint64_t sgn, int e0) {
  const uint64_t ma = (ua & kFrac) | kImpl, mb = (ub & kFrac) | kImpl;
  const int lt = ma < mb ? 1 : 0;
  const uint64_t A = ma << lt;              // A in [mb, 2 mb): A/mb in [1, 2)
  const int e = e0 - lt;
  // Q = floor(A 2^52 / mb) in [2^52, 2^53), built as q0 2^29 + q1 2^11 + q2.
  const float fb = fval(0x4B000000u | ((uint32_t)(mb >> 29) & 0x7FFFFFu));   // mb >> 29, exact
  const float fa = fval(0x4B000000u | ((uint32_t)(ma >> 29) & 0x7FFFFFu));   // ma >> 29, exact
  const float r = rcp_approx(fb);
  // relative error of r fa / (ma / mb) is at most 2^-23 (fa) + 2^-23 (fb) +
  // 2^-22 (r) + 2^-23 (two roundings) < 2^-20.6
  // digit 0 (24 bits): q0 ~ A 2^23 / mb, within 10.5
  const uint32_t q0 = f_to_u24_clamped(fmul(fmul(fa, r), lt ? 16777216.0f : 8388608.0f));
  int64_t R = (int64_t)((A << 23) - (uint64_t)q0 * mb);                // |R| <= 10.5 mb < 2^56.4
  // digit 1 (18 bits): q1 ~ R 2^18 / mb ~ (R >> 35) 2^53 / mb ~ (R >> 35) r 2^24,
  // |q1| < 2^21.4; error <= 2 (truncation) + 1.3 (relative) + 0.5 (rounding)
  const int32_t q1 = f2i_small(fmul(fmul(i2f_small((int32_t)(R >> 35)), r), 16777216.0f));
  R = (int64_t)(((uint64_t)R << 18) - mulw(q1, mb));                    // |R| <= 3.8 mb < 2^55
  // digit 2 (11 bits): q2 ~ R 2^11 / mb ~ (R >> 34) r 2^16, |q2| < 2^13; error < 0.51
  const int32_t q2 = f2i_small(fmul(fmul(i2f_small((int32_t)(R >> 34)), r), 65536.0f));
  R = (int64_t)(((uint64_t)R << 11) - mulw(q2, mb));                    // |R| < 0.51 mb
  // R = A 2^52 - Q mb exactly for Q = q0 2^29 + q1 2^11 + q2, |R| < 0.51 mb:
  // the exact quotient A 2^52 / mb is within 0.51 of Q, so its nearest integer
  // is Q + 1 when 2R > mb, Q - 1 when 2R < -mb and Q otherwise.  No tie
  // arises: the quotient of two binary floating-point numbers is never half
  // way between two representable ones.
  const int64_t twoR = R * 2, m = (int64_t)mb;                           // |2R| < 2^54.1
  const int32_t q2r = q2 + (twoR > m ? 1 : 0) - (twoR < -m ? 1 : 0);
  // the result's significand (in [2^52, 2^53]; 2^53 carries into the exponent
  // field) added to the exponent field of e - 1
  return dval(sgn | ((((uint64_t)(e - 1) << 52) + ((uint64_t)q0 << 29)) +
                     ((uint64_t)(int64_t)q1 << 11) + (uint64_t)(int64_t)q2r));
}

// RN(a / b) on the fast domain -- b normal, and a = +-0 or a normal with the
// quotient's exponent in [1, 2045] whichever way the significand quotient
// falls (so the result is normal) -- without a branch.  Outside that domain
// the result is unspecified and bad is set to 1.
SFP_FN double div_fast(double a, double b, unsigned &bad) {
  const uint64_t ua = dbits(a), ub = dbits(b);
  const uint64_t sgn = (ua ^ ub) & kSign;
  const uint32_t ea = (uint32_t)(ua >> 52) & 0x7ffu, eb = (uint32_t)(ub >> 52) & 0x7ffu;
  const int e0 = (int)ea - (int)eb + 1023;
  const bool b_normal = eb - 1u < 2046u;
  const bool a_zero = (ua & kAbs) == 0;
  bad |= (b_normal && (a_zero || (ea - 1u < 2046u && (unsigned)(e0 - 2) < 2044u))) ? 0u : 1u;
  const double q = div_core(ua, ub, sgn, e0);
  return a_zero ? dval(sgn) : q;
}

// RN(a / b) in double for two floats, given q32 = RN32(a / b), their quotient
// correctly rounded to single precision: the first 24 bits of the double
// quotient are q32's (or 2^24 when q32 rounded up into the next binade), and
// two more integer digits of 20 and 9 bits with exact residuals complete the
// 53, on 32-bit integers (the residuals are small, so arithmetic modulo 2^32
// gives them exactly).  div_ff_core assumes its domain: a = +-0 or normal, b
// normal, q32 normal (a quotient of floats is always a normal double);
// div_ff checks it, sets bad outside it (the result is then unspecified).
SFP_FN double div_ff_core(float a, float b, float q32) {
  const uint32_t ua = fbits(a), ub = fbits(b), uq = fbits(q32);
  const uint32_t sgn = (ua ^ ub) & 0x80000000u;
  const uint32_t ea = (ua >> 23) & 0xffu, eb = (ub >> 23) & 0xffu, eq = (uq >> 23) & 0xffu;
  const uint32_t ma = (ua & 0x7fffffu) | 0x800000u, mb = (ub & 0x7fffffu) | 0x800000u;
  const uint32_t lt = ma < mb ? 1u : 0u;
  const uint32_t A = ma << lt;                       // A / mb in [1, 2)
  const int e = (int)ea - (int)eb - (int)lt;         // floor(lg |a / b|)
  // q0 = RN(A 2^23 / mb) in [2^23, 2^24]: q32's significand, or 2^24 when q32
  // is 2^(e+1)
  const bool up = (int)eq == e + 128;
  const uint32_t q0 = up ? 0x1000000u : ((uq & 0x7fffffu) | 0x800000u);
  // E0 = A 2^23 - q0 mb, |E0| <= mb / 2 < 2^23 (q0 is the nearest integer)
  const int32_t E0 = (int32_t)((A << 23) - q0 * mb);
  // r ~ 1/mb to ~2^-22 relative (mb < 2^24 is exact in a float)
  const float r = rcp_approx(fval(0x4B000000u | (mb & 0x7FFFFFu)));
  // digit 1 (20 bits): q1 ~ E0 2^20 / mb ~ (E0 >> 2) r 2^22, |q1| < 2^19;
  // error <= 0.38 (truncation of E0) + 0.31 (r and roundings) + 0.5 (rounding)
  const int32_t q1 = f2i_small(fmul(fmul(i2f_small(E0 >> 2), r), 4194304.0f));
  const int32_t E1 = (int32_t)(((uint32_t)E0 << 20) - (uint32_t)q1 * mb);   // |E1| < 1.2 mb
  // digit 2 (9 bits): q2 ~ E1 2^9 / mb ~ (E1 >> 5) r 2^14, |q2| < 2^10;
  // error <= 2^-9 (truncation) + 2^-11 (r and roundings) + 0.5 (rounding) < 0.51
  const int32_t q2 = f2i_small(fmul(fmul(i2f_small(E1 >> 5), r), 16384.0f));
  const int32_t E2 = (int32_t)(((uint32_t)E1 << 9) - (uint32_t)q2 * mb);    // |E2| < 0.51 mb
  // A 2^52 / mb = Q + E2 / mb, Q = q0 2^29 + q1 2^9 + q2: the nearest integer
  // is Q + 1 when 2 E2 > mb, Q - 1 when 2 E2 < -mb, else Q (never a tie: a
  // quotient of 24-bit integers is not half way between 53-bit ones)
  const int32_t tE2 = E2 * 2, m = (int32_t)mb;
  const int32_t low = q1 * 512 + q2 + (tE2 > m ? 1 : 0) - (tE2 < -m ? 1 : 0);
  // significand in [2^52, 2^53] (2^53 carries into the exponent field) added
  // to the exponent field of e - 1
  const uint64_t sig = ((uint64_t)q0 << 29) + (uint64_t)(int64_t)low;
  const uint64_t r64 = (((uint64_t)(e + 1023 - 1)) << 52) + sig;
  const bool a_zero = (ua & 0x7fffffffu) == 0;
  return dval(((uint64_t)sgn << 32) | (a_zero ? 0ull : r64));
}
SFP_FN double div_ff(float a, float b, float q32, unsigned &bad) {
  const uint32_t ua = fbits(a), ub = fbits(b), uq = fbits(q32);
  const uint32_t ea = (ua >> 23) & 0xffu, eb = (ub >> 23) & 0xffu, eq = (uq >> 23) & 0xffu;
  const uint32_t ma = (ua & 0x7fffffu) | 0x800000u, mb = (ub & 0x7fffffu) | 0x800000u;
  const int e = (int)ea - (int)eb - (ma < mb ? 1 : 0);
  const bool a_zero = (ua & 0x7fffffffu) == 0;
  bad |= (a_zero || (ea - 1u < 254u && eq - 1u < 254u && ((int)eq == e + 128 || (int)eq == e + 127))) &&
                 eb - 1u < 254u ? 0u : 1u;
  return div_ff_core(a, b, q32);
}

// RN(a / b) for all operands: the hardware instruction outside the fast domain.
SFP_FN double div_rn(double a, double b) {
  const uint64_t ua = dbits(a), ub = dbits(b);
  const uint64_t sgn = (ua ^ ub) & kSign;
  const uint32_t ea = (uint32_t)(ua >> 52) & 0x7ffu, eb = (uint32_t)(ub >> 52) & 0x7ffu;
  const int e0 = (int)ea - (int)eb + 1023;
  const bool b_normal = eb - 1u < 2046u;
  if ((ua & kAbs) == 0 && b_normal) return dval(sgn);          // +-0 / normal
  if (!(ea - 1u < 2046u && b_normal && (unsigned)(e0 - 2) < 2044u)) return hw_div(a, b);
  return div_core(ua, ub, sgn, e0);
}

// RN(sqrt(x)) for x = dval(ux) positive and normal: three integer digits.
SFP_FN double sqrt_core(uint64_t ux) {
  const uint32_t ex = (uint32_t)(ux >> 52);
  const uint64_t mx = (ux & kFrac) | kImpl;
  const int E = (int)ex - 1023;
  const int odd = E & 1;
  const uint64_t X = mx << odd;                    // X in [2^52, 2^54), E - odd even
  const int er = ((E - odd) >> 1) + 1023;          // result exponent, always normal
  // S = floor(sqrt(X 2^52)) in [2^52, 2^53), built as s0 2^29 + d1 2^11 + d2.
  // fx = X / 2^30 to 24 bits: the top 24 bits of mx as a float in [2^23, 2^24),
  // halved (exponent field minus one) when X = mx, i.e. E even
  const float fx = fval((0x4B000000u | ((uint32_t)(mx >> 29) & 0x7FFFFFu)) - ((uint32_t)(odd ^ 1) << 23));
  const float y = rsqrt_approx(fx);                // ~fx^-1/2
  // digit 0 (24 bits): s0 ~ sqrt(fx) 2^12 ~ S / 2^29, within 8.5
  const uint32_t s0 = f_to_u24_clamped(fmul(fmul(fx, y), 4096.0f));
  // R1 = (X 2^52 - (s0 2^29)^2) / 2^52 = X - (8 s0)^2 exactly (8 s0 < 2^27); |R1| < 2^34.1
  const uint32_t s08 = s0 << 3;
  const int64_t R1 = (int64_t)(X - (uint64_t)s08 * s08);
  // digit 1 (18 bits): the Newton step S - s0 2^29 ~ R1 2^52 / (2 s0 2^29), in units of
  // 2^11: d1 ~ R1 / (2 s0) 2^12 ~ R1 y / 2 (1/s0 ~ y 2^-12); |d1| < 2^21.1;
  // error <= 2 (truncation) + 2.3 (y for 1/s0) + 1.1 (Newton's square term) + 0.5
  const int32_t d1 = f2i_small(fmul(fmul(i2f_small((int32_t)(R1 >> 13)), y), 4096.0f));
  const uint64_t S2 = ((uint64_t)s0 << 29) + ((uint64_t)(int64_t)d1 << 11);
  // R2 = (X 2^52 - S2^2) / 2^22 = R1 2^30 - s0 d1 2^19 - d1^2; |R2| < 2^45.6
  const int64_t R2 = (int64_t)(((uint64_t)R1 << 30) - ((uint64_t)((int64_t)s0 * d1) << 19) -
                               (uint64_t)((int64_t)d1 * d1));
  // digit 2 (11 bits): d2 ~ R2 2^22 / (2 S2) ~ (R2 >> 24) y 2^4, |d2| < 2^13.6; error < 0.53
  const int32_t d2 = f2i_small(fmul(fmul(i2f_small((int32_t)(R2 >> 24)), y), 16.0f));
  const int64_t si = (int64_t)(S2 + (uint64_t)(int64_t)d2);                 // S
  // R = X 2^52 - S^2 = R2 2^22 - 2 S2 d2 - d2^2, |R| < 2^55
  const int64_t R = (int64_t)(((uint64_t)R2 << 22) - (mulw(d2, S2) << 1) -
                              (uint64_t)((int64_t)d2 * d2));
  // the exact root t = sqrt(X 2^52) is within 0.53 of S, so its nearest
  // integer (t is never half way) is S + 1 when t > S + 1/2, i.e. R > S + 1/4,
  // i.e. R > S; S - 1 when t < S - 1/2, i.e. R < 1/4 - S, i.e. R <= -S; and
  // S otherwise (R integer); the adjustment joins the last digit
  const int32_t d2r = d2 + (R > si ? 1 : 0) - (R <= -si ? 1 : 0);
  return dval((((uint64_t)(er - 1) << 52) + S2) + (uint64_t)(int64_t)d2r);
}

// RN(sqrt(x)) for positive normal x, without a branch; for any other x (+-0,
// subnormal, negative, inf, NaN) the result is unspecified and bad is set.
SFP_FN double sqrt_fast(double x, unsigned &bad) {
  const uint64_t ux = dbits(x);
  bad |= ((uint32_t)(ux >> 52) - 1u < 2046u) ? 0u : 1u;   // the exponent field includes the sign
  return sqrt_core(ux);
}

// RN(a b) on the integer pipe, for a and b normal or zero and a product that is
// zero or normal; otherwise the result is unspecified and bad is set.  The
// 53-bit significands ma, mb are split at bit 32 (ma = ah 2^32 + al, ah < 2^21),
// the 106-bit product P = ma mb is formed from four 32 x 32 -> 64-bit products
// (P in [2^104, 2^106)), normalized to [2^105, 2^106) by one left shift when
// below, and rounded to nearest even at bit 53: the significand is P >> 53, the
// round bit bit 52, the sticky bits 0 - 51.  A carry of the rounding into 2^53
// moves into the exponent field.  (The FP64 pipe of GB300 executes 2
// operations per clock per SM; this trades one of them for integer
// instructions.)
SFP_FN double mul_fast(double a, double b, unsigned &bad) {
  const uint64_t ua = dbits(a), ub = dbits(b);
  const uint32_t ha = (uint32_t)(ua >> 32), hb = (uint32_t)(ub >> 32);
  const uint32_t la = (uint32_t)ua, lb = (uint32_t)ub;
  const uint32_t ea = (ha >> 20) & 0x7ffu, eb = (hb >> 20) & 0x7ffu;
  const uint32_t sgn = (ha ^ hb) & 0x80000000u;
  const bool zero = ((ua << 1) == 0) || ((ub << 1) == 0);
  const uint32_t mah = (ha & 0xfffffu) | 0x100000u, mbh = (hb & 0xfffffu) | 0x100000u;
  const uint64_t ll = (uint64_t)la * lb;
  const uint64_t mid = (uint64_t)la * mbh + (uint64_t)mah * lb;        // < 2^54
  const uint64_t lo = ll + (mid << 32);
  const uint64_t hi = (uint64_t)mah * mbh + (mid >> 32) + (lo < ll ? 1u : 0u);   // P >> 64, < 2^42
  // normalize: P < 2^105 (bit 41 of hi clear) moves up by one
  const uint32_t top = (uint32_t)(hi >> 41) & 1u;
  const uint64_t h2 = top ? hi : (hi << 1) | (lo >> 63);
  const uint64_t l2 = top ? lo : lo << 1;
  const uint64_t sig = (h2 << 11) | (l2 >> 53);                       // in [2^52, 2^53)
  const uint64_t rbit = (l2 >> 52) & 1u;
  const uint64_t sticky = (l2 << 12) != 0 ? 1u : 0u;
  const uint64_t inc = rbit & (sticky | (sig & 1u));
  const int e = (int)ea + (int)eb - 1023 + (int)top;                   // biased exponent
  const uint64_t r = ((uint64_t)(uint32_t)(e - 1) << 52) + sig + inc;
  const bool in_ok = (ea - 1u < 2046u || (ua << 1) == 0) && (eb - 1u < 2046u || (ub << 1) == 0);
  const bool out_ok = zero || (e >= 1 && (uint32_t)(r >> 52) - 1u < 2046u);
  bad |= (in_ok && out_ok) ? 0u : 1u;
  return dval(((uint64_t)sgn << 32) | (zero ? 0ull : r));
}

// RN(sqrt(x)) for all x: the hardware instruction outside the fast domain.
SFP_FN double sqrt_rn(double x) {
  const uint64_t ux = dbits(x);
  if (!((uint32_t)(ux >> 52) - 1u < 2046u)) return hw_sqrt(x);   // +-0, subnormal, negative, inf, NaN
  return sqrt_core(ux);
}

// Conversions between float and double on the integer pipe (the conversion
// instruction runs on the FP64 pipe).
// f2d: exact widening; normal numbers and zeros here, the instruction for
// subnormal, infinite and NaN inputs.
SFP_FN double f2d(float x) {
  const uint32_t b = fbits(x);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  if (e - 1u < 254u)
    return dval(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29));
  if ((b & 0x7fffffffu) == 0) return dval(sign);
  return (double)x;
}
// d2f: round to nearest float, ties to even, for results in the normal float
// range (a carry out of the significand moves to the next binade, and past
// FLT_MAX to infinity, as rounding to nearest does) and for zeros; the
// instruction for subnormal float results, infinities and NaNs.
SFP_FN float d2f(double x) {
  const uint64_t u = dbits(x);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t ef = ((hi >> 20) & 0x7ffu) - 896u;      // float biased exponent
  if (ef - 1u < 254u) {
    uint32_t r = (ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;                 // the 29 dropped bits
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
    return fval((hi & 0x80000000u) | r);
  }
  if (((hi & 0x7fffffffu) | lo) == 0) return fval(hi & 0x80000000u);
#if defined(__CUDA_ARCH__)
  return __double2float_rn(x);
#else
  return (float)x;
#endif
}

}  // namespace sfp
}  // namespace svd2
