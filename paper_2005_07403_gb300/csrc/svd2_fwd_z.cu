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
