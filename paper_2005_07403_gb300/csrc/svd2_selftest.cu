// svd2_arith_check: the library's double division and square root (computed on
// the integer and FP32 pipes, svd2_softfp.cuh) and its float <-> double
// conversions (integer pipe) next to the hardware's IEEE instructions, element
// by element, for testing on the device.
#include "svd2_common.cuh"
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
    } else {
      const float f = __uint_as_float((unsigned)__double2loint(a));
      lib[i] = svd2::sfp::f2d(f);
      hw[i] = (double)f;
    }
  }
}

}  // namespace

extern "C" int svd2_arith_check(int op, int64_t n, const double *x, const double *y, double *lib,
                                double *hw, svd2_stream_t stream) {
  if (op < 0 || op > 3) return SVD2_EINVAL;
  if (n < 0) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!x || !lib || !hw || (op == 0 && !y)) return SVD2_EINVAL;
  const int grid = 8 * svd2::sm_count();
  arith_check_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(op, n, x, y, lib, hw);
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}
