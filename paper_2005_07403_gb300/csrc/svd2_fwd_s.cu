// Plain forward form svd2_batch_s and its C ABI (kernel template in
// svd2_fwd_impl.cuh; one translation unit per form so they build in parallel).
#include "svd2_fwd_impl.cuh"

using namespace svd2;

extern "C" int svd2_batch_s(int64_t n, const float *const A[4], float *const U[4],
                            float *const V[4], float *smax, float *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  FwdArgs<float, 4> p{};
  return launch_fwd<float, false>(kOpS, n, A, U, V, smax, smin, s, flags, (cudaStream_t)stream,
                                    p);
}

extern "C" int svd2_values_s(int64_t n, const float *const A[4], float *smax, float *smin,
                             int32_t *s, uint32_t flags, svd2_stream_t stream) {
  FwdArgs<float, 4> p{};
  return launch_fwd<float, false>(kOpS, n, A, nullptr, nullptr, smax, smin, s, flags,
                               (cudaStream_t)stream, p, true);
}

extern "C" int svd2_batch_interleaved_s(int64_t n, const float *A, float *U, float *V, float *smax,
                                        float *smin, int32_t *s, uint32_t flags,
                                        svd2_stream_t stream) {
  if ((U == nullptr) != (V == nullptr)) return SVD2_EINVAL;
  return launch_interleaved<float, false>(kOpS, n, A, U, V, smax, smin, s, flags,
                                        (cudaStream_t)stream, U == nullptr);
}
