// Plain forward form svd2_batch_c and its C ABI (kernel template in
// svd2_fwd_impl.cuh; one translation unit per form so they build in parallel).
#include "svd2_fwd_impl.cuh"

using namespace svd2;

extern "C" int svd2_batch_c(int64_t n, const float *const A[8], float *const U[8],
                            float *const V[8], float *smax, float *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  FwdArgs<float, 8> p{};
  return launch_fwd<float, true>(kOpC, n, A, U, V, smax, smin, s, flags, (cudaStream_t)stream,
                                    p);
}

extern "C" int svd2_values_c(int64_t n, const float *const A[8], float *smax, float *smin,
                             int32_t *s, uint32_t flags, svd2_stream_t stream) {
  FwdArgs<float, 8> p{};
  return launch_fwd<float, true>(kOpC, n, A, nullptr, nullptr, smax, smin, s, flags,
                               (cudaStream_t)stream, p, true);
}

extern "C" int svd2_batch_interleaved_c(int64_t n, const float *A, float *U, float *V, float *smax,
                                        float *smin, int32_t *s, uint32_t flags,
                                        svd2_stream_t stream) {
  if ((U == nullptr) != (V == nullptr)) return SVD2_EINVAL;
  return launch_interleaved<float, true>(kOpC, n, A, U, V, smax, smin, s, flags,
                                        (cudaStream_t)stream, U == nullptr);
}
