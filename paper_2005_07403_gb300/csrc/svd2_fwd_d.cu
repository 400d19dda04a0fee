// Plain forward form svd2_batch_d and its C ABI (kernel template in
// svd2_fwd_impl.cuh; one translation unit per form so they build in parallel).
#include "svd2_fwd_impl.cuh"

using namespace svd2;

extern "C" int svd2_batch_d(int64_t n, const double *const A[4], double *const U[4],
                            double *const V[4], double *smax, double *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  FwdArgs<double, 4> p{};
  return launch_fwd<double, false>(kOpD, n, A, U, V, smax, smin, s, flags, (cudaStream_t)stream,
                                    p);
}

extern "C" int svd2_values_d(int64_t n, const double *const A[4], double *smax, double *smin,
                             int32_t *s, uint32_t flags, svd2_stream_t stream) {
  FwdArgs<double, 4> p{};
  return launch_fwd<double, false>(kOpD, n, A, nullptr, nullptr, smax, smin, s, flags,
                               (cudaStream_t)stream, p, true);
}

extern "C" int svd2_batch_interleaved_d(int64_t n, const double *A, double *U, double *V, double *smax,
                                        double *smin, int32_t *s, uint32_t flags,
                                        svd2_stream_t stream) {
  if ((U == nullptr) != (V == nullptr)) return SVD2_EINVAL;
  return launch_interleaved<double, false>(kOpD, n, A, U, V, smax, smin, s, flags,
                                        (cudaStream_t)stream, U == nullptr);
}
