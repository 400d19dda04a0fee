// Plain forward forms and their C ABI: svd2_batch_{d,z,s,c}.  The kernel
// template lives in svd2_fwd_impl.cuh.
#include "svd2_fwd_impl.cuh"

using namespace svd2;

template <typename T, bool CPLX>
static int fwd(int op, int64_t n, const T *const *A, T *const *U, T *const *V, T *smax, T *smin,
               int32_t *s, uint32_t flags, svd2_stream_t stream) {
  FwdArgs<T, CPLX ? 8 : 4> p{};
  return launch_fwd<T, CPLX, false>(op, n, A, U, V, smax, smin, s, flags, (cudaStream_t)stream, p);
}

extern "C" int svd2_batch_d(int64_t n, const double *const A[4], double *const U[4],
                            double *const V[4], double *smax, double *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  return fwd<double, false>(kOpD, n, A, U, V, smax, smin, s, flags, stream);
}

extern "C" int svd2_batch_z(int64_t n, const double *const A[8], double *const U[8],
                            double *const V[8], double *smax, double *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  return fwd<double, true>(kOpZ, n, A, U, V, smax, smin, s, flags, stream);
}

extern "C" int svd2_batch_s(int64_t n, const float *const A[4], float *const U[4],
                            float *const V[4], float *smax, float *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  return fwd<float, false>(kOpS, n, A, U, V, smax, smin, s, flags, stream);
}

extern "C" int svd2_batch_c(int64_t n, const float *const A[8], float *const U[8],
                            float *const V[8], float *smax, float *smin, int32_t *s,
                            uint32_t flags, svd2_stream_t stream) {
  return fwd<float, true>(kOpC, n, A, U, V, smax, smin, s, flags, stream);
}
