// FP32 form with FP64 re-run: svd2_batch_s_rerun / svd2_batch_c_rerun.
//
// Pass 1 is the single-precision method (Sec. 1, Sec. 7) over all matrices;
// it flags every matrix whose scaled singular values satisfy
// sigma'_min < 2^tau sigma'_max (compared in float; the product by the power of
// two is exact) and appends its index to a list in the workspace with one
// atomic per warp.  Pass 2 re-runs the flagged matrices only, on full warps,
// with the double-precision method on the exactly widened input, and writes
// the double results rounded to float, sigma' brought to the float run's
// scale: sigma'_32 = RN32(sigma'_64 2^(s32 - s64)).  Both passes run on the
// caller's stream with no host synchronisation; pass 2 reads the list length
// from device memory and covers it with a grid-stride loop.
#include "svd2_fwd_impl.cuh"

namespace svd2 {

// Workspace layout: [0] total re-run count of the call (uint64), [1] count of
// the current chunk (uint64), then from byte 256 the uint32 index list of the
// current chunk (chunk-relative indices).
constexpr size_t kListOffset = 256;
constexpr int64_t kChunk = int64_t(1) << 31;

template <int NA>
struct RerunArgs {
  const float *a[NA];
  float *u[NA];
  float *v[NA];
  float *smax;
  float *smin;
  const uint32_t *list;
  const unsigned long long *count;
  unsigned long long *total;
  uint32_t flags;
};

template <bool CPLX>
__global__ void __launch_bounds__(256) rerun_kernel(const RerunArgs<CPLX ? 8 : 4> p) {
  constexpr int NA = CPLX ? 8 : 4;
  const unsigned long long cnt = *p.count;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (unsigned long long i = tid; i < cnt; i += stride) {
    const uint32_t k = p.list[i];
    float a[NA];
    double ad[NA];
    unsigned mx = 0;
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      a[e] = p.a[e][k];
      ad[e] = (double)a[e];
      const unsigned b = fp<float>::bits(a[e]) & fp<float>::kAbs;
      mx = b > mx ? b : mx;
    }
    int32_t s32 = scale_exponent<float>(mx);
    double u[NA], v[NA], sx, sn;
    int32_t s64;
    int piv;
    if constexpr (CPLX)
      svd2_cplx<double>(ad, u, v, sx, sn, s64, piv);
    else
      svd2_real<double>(ad, u, v, sx, sn, s64, piv);
    float fx = __double2float_rn(scalef(sx, s32 - s64));
    float fn = __double2float_rn(scalef(sn, s32 - s64));
    if (p.flags & SVD2_BACKSCALE) backscale(fx, fn, s32);
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      p.u[e][k] = __double2float_rn(u[e]);
      p.v[e][k] = __double2float_rn(v[e]);
    }
    p.smax[k] = fx;
    p.smin[k] = fn;
  }
  if (tid == 0) *p.total += cnt;
}

template <bool CPLX>
static int rerun_form(int op, int64_t n, const float *const *A, float *const *U, float *const *V,
                      float *smax, float *smin, int32_t *s, int tau_log2, uint32_t flags,
                      void *workspace, size_t ws_bytes, cudaStream_t stream) {
  constexpr int NA = CPLX ? 8 : 4;
  if (n < 0 || tau_log2 < -100 || tau_log2 > 0 || (flags & ~SVD2_BACKSCALE)) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!workspace || !aligned(workspace, 16) || ws_bytes < svd2_rerun_workspace_bytes(n))
    return SVD2_EINVAL;
  if (!A || !U || !V) return SVD2_EINVAL;
  auto *ws = static_cast<unsigned char *>(workspace);
  auto *total = reinterpret_cast<unsigned long long *>(ws);
  auto *count = total + 1;
  auto *list = reinterpret_cast<uint32_t *>(ws + kListOffset);
  SVD2_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(unsigned long long), stream));
  // pass 2 covers a device-resident count with a grid-stride loop: one
  // resident wave of blocks, enough warps to hide its scattered accesses
  int resident = 0;
  SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, rerun_kernel<CPLX>, 256, 0));
  const int grid2 = sm_count() * (resident > 0 ? resident : 1);
  for (int64_t base = 0; base < n; base += kChunk) {
    const int64_t m = (n - base < kChunk) ? (n - base) : kChunk;
    const float *a[NA];
    float *u[NA], *v[NA];
    for (int e = 0; e < NA; ++e) {
      if (!A[e] || !U[e] || !V[e]) return SVD2_EINVAL;
      a[e] = A[e] + base;
      u[e] = U[e] + base;
      v[e] = V[e] + base;
    }
    if (!smax || !smin || !s) return SVD2_EINVAL;
    SVD2_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream));
    FwdArgs<float, NA> p{};
    p.tau = ldexpf(1.0f, tau_log2);
    p.list = list;
    p.count = count;
    int rc = launch_fwd<float, CPLX, true>(op, m, a, u, v, smax + base, smin + base, s + base,
                                           flags, stream, p);
    if (rc != SVD2_OK) return rc;
    RerunArgs<NA> q{};
    for (int e = 0; e < NA; ++e) {
      q.a[e] = a[e];
      q.u[e] = u[e];
      q.v[e] = v[e];
    }
    q.smax = smax + base;
    q.smin = smin + base;
    q.list = list;
    q.count = count;
    q.total = total;
    q.flags = flags;
    rerun_kernel<CPLX><<<grid2, 256, 0, stream>>>(q);
    SVD2_CUDA_TRY(cudaGetLastError());
  }
  return SVD2_OK;
}

}  // namespace svd2

using namespace svd2;

extern "C" size_t svd2_rerun_workspace_bytes(int64_t n) {
  if (n <= 0) return kListOffset;
  const int64_t m = n < kChunk ? n : kChunk;
  return kListOffset + (size_t)m * sizeof(uint32_t);
}

extern "C" int svd2_batch_s_rerun(int64_t n, const float *const A[4], float *const U[4],
                                  float *const V[4], float *smax, float *smin, int32_t *s,
                                  int tau_log2, uint32_t flags, void *workspace,
                                  size_t workspace_bytes, svd2_stream_t stream) {
  return rerun_form<false>(kOpS, n, A, U, V, smax, smin, s, tau_log2, flags, workspace,
                           workspace_bytes, (cudaStream_t)stream);
}

extern "C" int svd2_batch_c_rerun(int64_t n, const float *const A[8], float *const U[8],
                                  float *const V[8], float *smax, float *smin, int32_t *s,
                                  int tau_log2, uint32_t flags, void *workspace,
                                  size_t workspace_bytes, svd2_stream_t stream) {
  return rerun_form<true>(kOpC, n, A, U, V, smax, smin, s, tau_log2, flags, workspace,
                          workspace_bytes, (cudaStream_t)stream);
}

extern "C" int svd2_rerun_count(const void *workspace, int64_t *count) {
  if (!workspace || !count) return SVD2_EINVAL;
  unsigned long long c = 0;
  SVD2_CUDA_TRY(cudaMemcpy(&c, workspace, sizeof(c), cudaMemcpyDeviceToHost));
  *count = (int64_t)c;
  return SVD2_OK;
}
