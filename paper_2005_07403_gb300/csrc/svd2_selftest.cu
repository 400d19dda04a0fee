// svd2_arith_check: the library's double division and square root (computed on
// the integer and FP32 pipes, svd2_softfp.cuh) and its float <-> double
// conversions (integer pipe) next to the hardware's IEEE instructions, element
// by element, for testing on the device.
#include "svd2_common.cuh"
#include "svd2_math.cuh"
#include "svd2_softfp.cuh"

namespace {

__global__ void arith_check_kernel(int op, int64_t n, const double *x, const double *y,
                                   double *lib, double *hw) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = x[i];
    if (op == 0) {
      const double b = y[i];
      lib[i] = svd2::sfp::div_rn(a, b);
      hw[i] = __ddiv_rn(a, b);
    } else if (op == 1) {
      lib[i] = svd2::sfp::sqrt_rn(a);
      hw[i] = __dsqrt_rn(a);
    } else if (op == 2) {
      lib[i] = (double)svd2::sfp::d2f(a);
      hw[i] = (double)__double2float_rn(a);
    } else if (op == 3) {
      const float f = __uint_as_float((unsigned)__double2loint(a));
      lib[i] = svd2::sfp::f2d(f);
      hw[i] = (double)f;
    } else {
      // the double quotient of two floats (x, y rounded to float) completed from
      // their float quotient; NaN where it flags the operands
      const float fa = __double2float_rn(a), fb = __double2float_rn(y[i]);
      unsigned flag = 0;
      const double q = svd2::sfp::div_ff(fa, fb, __fdiv_rn(fa, fb), flag);
      lib[i] = flag ? __longlong_as_double(0x7ff8000000000000ll) : q;
      hw[i] = __ddiv_rn((double)fa, (double)fb);
    }
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {   // SplitMix64 finaliser
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// res[0] += mismatches, res[1] = min mismatching index, res[2] += cases checked.
__global__ void fp32_check_kernel(int op, uint64_t begin, uint64_t count,
                                  unsigned long long *res) {
  unsigned long long bad = 0, checked = 0, first = ~0ull;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint64_t k = begin + i;
    bool ok = true, in = true;
    if (op == 0) {
      const float b = __uint_as_float((uint32_t)k);
      ok = __float_as_uint(svd2::frcp_mk(b)) == __float_as_uint(__frcp_rn(b));
    } else if (op == 1) {
      const float x = __uint_as_float((uint32_t)k);
      ok = __float_as_uint(svd2::fsqrt_mk(x)) == __float_as_uint(__fsqrt_rn(x));
    } else if (op == 2) {        // significand pairs: a, b in [1, 2)
      const float a = __uint_as_float(0x3f800000u | (uint32_t)((k >> 23) & 0x7fffffu));
      const float b = __uint_as_float(0x3f800000u | (uint32_t)(k & 0x7fffffu));
      ok = __float_as_uint(svd2::fdiv_mk(a, b)) == __float_as_uint(__fdiv_rn(a, b));
    } else {                     // random bit patterns, checked on the stated domain
      const uint64_t r = mix64(k);
      const float a = __uint_as_float((uint32_t)r), b = __uint_as_float((uint32_t)(r >> 32));
      const float ab = fabsf(b);
      const double q = fabs((double)a / (double)b);
      in = ab >= 0x1p-125f && ab <= 0x1p125f &&
           (a == 0.0f || (fabsf(a) >= 0x1p-102f && q >= 0x1p-125 && q <= 0x1p127));
      if (in) ok = __float_as_uint(svd2::fdiv_mk(a, b)) == __float_as_uint(__fdiv_rn(a, b));
    }
    checked += in ? 1 : 0;
    if (!ok) {
      ++bad;
      first = k < first ? k : first;
    }
  }
  if (bad) {
    atomicAdd(&res[0], bad);
    atomicMin(&res[1], first);
  }
  atomicAdd(&res[2], checked);
}

}  // namespace

extern "C" int svd2_fp32_selfcheck(int op, uint64_t begin, uint64_t count, void *result,
                                   svd2_stream_t stream) {
  if (op < 0 || op > 3 || !result || !svd2::aligned(result, 8)) return SVD2_EINVAL;
  if (count == 0) return SVD2_OK;
  fp32_check_kernel<<<16 * svd2::sm_count(), 256, 0, (cudaStream_t)stream>>>(
      op, begin, count, static_cast<unsigned long long *>(result));
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}

extern "C" int svd2_arith_check(int op, int64_t n, const double *x, const double *y, double *lib,
                                double *hw, svd2_stream_t stream) {
  if (op < 0 || op > 4) return SVD2_EINVAL;
  if (n < 0) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!x || !lib || !hw || ((op == 0 || op == 4) && !y)) return SVD2_EINVAL;
  const int grid = 8 * svd2::sm_count();
  arith_check_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(op, n, x, y, lib, hw);
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}
