// Real FP32 form with the FP64 tangent step: svd2_batch_s_tan64.
//
// The single-precision method (Sec. 1, Sec. 7) on every matrix, with one step
// taken in double where the matrix is ill-conditioned: when |r''_22| < 2^tau
// r11 at Eq. 7 (r''_22 / r11 is within a factor of two of sigma_min /
// sigma_max), -tan(alpha) = a'''_21 / a'''_11 and the fma of Eq. 7 are
// evaluated again in double.  In the real case the a''' are the scaled
// entries with signs changed -- exact in float -- so the cancellation of Eq. 7,
// where single precision loses sigma_min, is the double method's own.  The
// step is a branch inside the single-precision batch kernel: one integer
// double division, one FP64 fma and the conversions, with no second pass and
// no scratch memory.  The fix-up pass (as for svd2_batch_s) finishes the
// matrices the fast arithmetic could not, with the general arithmetic.
#include "svd2_fwd_impl.cuh"

namespace svd2 {

using Tan64Exact = Tan64Ar<ExactAr<float>>;

// Fix-up pass: the matrices with s = kRedoS recomputed with the general
// arithmetic at the paper's scale h (the tangent step included); counted.
__global__ void __launch_bounds__(256) tan64_fix_kernel(const __grid_constant__ FwdArgs<float, 4> p) {
  if (*p.redo == 0) return;
  unsigned nwide = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t k = k0; k < p.n; k += stride) {
    if (p.s[k] != kRedoS) continue;
    float a[4], u[4], v[4], sx, sn;
    int32_t so;
#pragma unroll
    for (int e = 0; e < 4; ++e) a[e] = p.a[e][k];
    Tan64Exact ar;
    ar.tau = p.tau;
    svd2_one<float, false>(ar, a, u, v, sx, sn, so);
    nwide += ar.wide;
    if (p.flags & SVD2_BACKSCALE) backscale(sx, sn, so);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      p.u[e][k] = u[e];
      p.v[e][k] = v[e];
    }
    p.smax[k] = sx;
    p.smin[k] = sn;
    p.s[k] = so;
  }
  if (p.count) warp_count_add(p.count, nwide);
}

template <int M, int U>
static FwdKernel<float, false> tan64_kernel() {
  return fwd_kernel<float, false, M, U, false, false, true>;
}

static FwdKernel<float, false> pick_tan64(int mpt, int unroll) {
#define SVD2_PICK(M_, U_) \
  if (mpt == M_ && unroll == U_) return tan64_kernel<M_, U_>();
  SVD2_PICK(1, 1) SVD2_PICK(1, 2) SVD2_PICK(2, 1) SVD2_PICK(2, 2) SVD2_PICK(4, 1) SVD2_PICK(4, 2)
#undef SVD2_PICK
  return nullptr;
}

}  // namespace svd2

using namespace svd2;

extern "C" int svd2_batch_s_tan64(int64_t n, const float *const A[4], float *const U[4],
                                  float *const V[4], float *smax, float *smin, int32_t *s,
                                  int tau_log2, uint32_t flags, unsigned long long *count,
                                  svd2_stream_t stream_) {
  const cudaStream_t stream = (cudaStream_t)stream_;
  if (n < 0 || tau_log2 < -100 || tau_log2 > 0 || (flags & ~SVD2_BACKSCALE)) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!A || !U || !V || !smax || !smin || !s) return SVD2_EINVAL;
  FwdArgs<float, 4> p{};
  bool vec_ok = aligned(smax, 16) && aligned(smin, 16) && aligned(s, 16);
  for (int e = 0; e < 4; ++e) {
    if (!A[e] || !U[e] || !V[e]) return SVD2_EINVAL;
    p.a[e] = A[e];
    p.u[e] = U[e];
    p.v[e] = V[e];
    vec_ok = vec_ok && aligned(A[e], 16) && aligned(U[e], 16) && aligned(V[e], 16);
  }
  p.smax = smax;
  p.smin = smin;
  p.s = s;
  p.n = n;
  p.flags = flags;
  p.stride = 1;
  p.tau = ldexpf(1.0f, tau_log2);
  p.count = count;
  Launch L = get_launch(kOpSTan64);
  if (!vec_ok) L.mpt = 1;
  FwdKernel<float, false> k = pick_tan64(L.mpt, L.unroll);
  if (!k) return SVD2_EINVAL;
  int resident = 0;
  SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, L.block, 0));
  const int64_t groups = n / L.mpt, tail = n % L.mpt;
  const int64_t loops = (groups + L.unroll - 1) / L.unroll;
  const int64_t grid = grid_for(loops > tail ? loops : tail, L, resident);
  void *flag = nullptr;
  int rc = flag_block(stream, &flag);
  if (rc != SVD2_OK) return rc;
  p.redo = static_cast<unsigned long long *>(flag);
  k<<<(unsigned)grid, (unsigned)L.block, 0, stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    tan64_fix_kernel<<<fix_grid(n), 256, 0, stream>>>(p);
    e = cudaGetLastError();
  }
  rc = flag_release(flag, stream);
  if (e != cudaSuccess) return record_cuda_error(e);
  return rc;
}
