// Plain forward form svd2_batch_z and its C ABI (kernel template in
// svd2_fwd_impl.cuh; one translation unit per form so they build in parallel).
#include "svd2_fwd_impl.cuh"

using namespace svd2;

extern "C" int svd2_batch_z(int64_t n, const double *const A[8], double *const U[8],
                            double *const V[8], double *smax, double *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  FwdArgs<double, 8> p{};
  return launch_fwd<double, true>(kOpZ, n, A, U, V, smax, smin, s, flags, (cudaStream_t)stream,
                                    p);
}

extern "C" int svd2_values_z(int64_t n, const double *const A[8], double *smax, double *smin,
                             int32_t *s, uint32_t flags, svd2_stream_t stream) {
  FwdArgs<double, 8> p{};
  return launch_fwd<double, true>(kOpZ, n, A, nullptr, nullptr, smax, smin, s, flags,
                               (cudaStream_t)stream, p, true);
}

extern "C" int svd2_batch_interleaved_z(int64_t n, const double *A, double *U, double *V, double *smax,
                                        double *smin, int32_t *s, uint32_t flags,
                                        svd2_stream_t stream) {
  if ((U == nullptr) != (V == nullptr)) return SVD2_EINVAL;
  return launch_interleaved<double, true>(kOpZ, n, A, U, V, smax, smin, s, flags,
                                        (cudaStream_t)stream, U == nullptr);
}
