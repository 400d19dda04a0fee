// FP32 form with FP64 re-run: svd2_batch_s_rerun / svd2_batch_c_rerun.
//
// Four launches on the caller's stream:
//  1. the single-precision batch kernel (fwd_kernel, as svd2_batch_s / _c, Sec.
//     1, Sec. 7) over all n matrices, which also marks (s = kRerunMark) every
//     matrix whose scaled singular values satisfy sigma'_min < 2^tau sigma'_max
//     (compared in float; the product by the power of two is exact);
//  2. compact_kernel: the marked indices, in increasing order within each
//     chunk, appended to a list in the workspace (reads s, 4 bytes a matrix);
//  3. list_rerun_kernel: every listed matrix decomposed again, one per thread
//     on full warps, by the double-precision method on the exactly widened
//     input, its outputs replaced by the double results rounded to float with
//     sigma' brought to the float run's scale: sigma'_32 = RN32(sigma'_64
//     2^(s32 - s64));
//  4. the fix-up pass, which finishes the matrices the fast single-precision
//     arithmetic could not (reads one word otherwise).
// Passes 1 and 3 are separate kernels so that each gets its own register
// budget and occupancy: the single-precision kernel is bound by HBM, the
// re-run by the FP64 and integer pipes.  The re-run's gathers and scattered
// 4-byte stores touch about 0.7 sectors per array and re-run matrix (one in
// ten matrices at the 2^-8 threshold on the ill-conditioned mix).
#include <type_traits>

#include "svd2_fwd_impl.cuh"

namespace svd2 {

// Workspace layout: [0] re-run count of the call (uint64), [8] the fix-up
// flag of the call (uint64), [16] the list length of the current chunk
// (uint64); from byte 256 the index list, 4 bytes per matrix of a chunk.
constexpr size_t kListOffset = 256;
constexpr int64_t kChunk = int64_t(1) << 31;

// Re-run of one matrix in double precision with the arithmetic policy
// Ar; float outputs u, v, sigma' stored (s is left to the caller).  Returns the
// final s of the matrix (the float run's exponent, or 0 after back-scaling).
// With FastAr, ar.bad set means the stored outputs are unspecified.
template <bool CPLX, typename Ar>
__device__ __forceinline__ int32_t rerun_one(Ar &ar, const FwdArgs<float, CPLX ? 8 : 4> &p,
                                             int64_t k, const float *a) {
  constexpr int NA = CPLX ? 8 : 4;
  double ad[NA];
  unsigned mx = 0;
#pragma unroll
  for (int e = 0; e < NA; ++e) {
    ad[e] = sfp::f2d(a[e]);   // float <-> double on the integer pipe
    const unsigned b = fp<float>::bits(a[e]) & fp<float>::kAbs;
    mx = b > mx ? b : mx;
  }
  int32_t s32 = scale_exponent<float>(mx);
  double u[NA], v[NA], sx, sn;
  int32_t s64;
  svd2_one<double, CPLX>(ar, ad, u, v, sx, sn, s64);
  float fx = sfp::d2f(ar.scale(sx, s32 - s64));
  float fn = sfp::d2f(ar.scale(sn, s32 - s64));
  if (p.flags & SVD2_BACKSCALE) {
    if (s32 != kZeroS) {
      fx = ar.template scale_as<float>(fx, -s32);
      fn = ar.template scale_as<float>(fn, -s32);
    }
    s32 = 0;
  }
#pragma unroll
  for (int e = 0; e < NA; ++e) {
    p.u[e][k] = sfp::d2f(u[e]);
    p.v[e][k] = sfp::d2f(v[e]);
  }
  p.smax[k] = fx;
  p.smin[k] = fn;
  return s32;
}

// Arithmetic of the double-precision re-run; its division and square root run
// on the integer pipe either way, so that the FP64 pipe (2 results per clock
// per SM) executes only the method's own operations.  Complex: the batch
// kernels' branch-free fast arithmetic (a matrix outside its domain gets
// s = kRedoRerun and the fix-up pass re-runs it with the general arithmetic);
// real: the general arithmetic.  Measured on the list of the 2^24 batch: real
// 198 us general against 221 us fast, complex (2^23) 254 us general against
// 239 us fast.
template <bool CPLX>
using RerunAr = typename std::conditional<CPLX, FastAr<double>, ExactAr<double>>::type;

// Pass 2: the indices k with s[k] == kRerunMark, in increasing order within
// each chunk of 16 * blockDim.x matrices (one warp-scan and one block-scan of
// the per-thread counts), each chunk appended to the list with one atomic on
// its length.  vec: s is 16-byte aligned (vector loads).
__global__ void __launch_bounds__(256) compact_kernel(const int32_t *s, int64_t n, uint32_t *list,
                                                      unsigned long long *len, bool vec) {
  __shared__ int warp_sum[8];
  __shared__ unsigned long long base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk = 16 * (int64_t)blockDim.x;
  for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < n; c0 += (int64_t)gridDim.x * chunk) {
    const int64_t k0 = c0 + 16 * (int64_t)threadIdx.x;
    unsigned bits = 0;
    if (vec && k0 + 16 <= n) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int4 w = __ldcs(reinterpret_cast<const int4 *>(s + k0) + q);
        bits |= (unsigned)(w.x == kRerunMark) << (4 * q) | (unsigned)(w.y == kRerunMark) << (4 * q + 1) |
                (unsigned)(w.z == kRerunMark) << (4 * q + 2) | (unsigned)(w.w == kRerunMark) << (4 * q + 3);
      }
    } else {
      for (int j = 0; j < 16 && k0 + j < n; ++j) bits |= (unsigned)(s[k0 + j] == kRerunMark) << j;
    }
    const int cnt = __popc(bits);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const int x = warp_sum[w];
        warp_sum[w] = tot;
        tot += x;
      }
      base = tot ? atomicAdd(len, (unsigned long long)tot) : 0;
    }
    __syncthreads();
    uint64_t pos = base + warp_sum[warp] + (incl - cnt);
    while (bits) {
      const int j = __ffs(bits) - 1;
      bits &= bits - 1;
      list[pos++] = (uint32_t)(k0 + j);
    }
    __syncthreads();
  }
}

// Pass 3: the listed matrices re-run in double precision, one per thread
// (full warps), outputs and s stored over the single-precision ones; the list
// length is read on the device, so the grid is one resident wave.
template <bool CPLX>
__global__ void __launch_bounds__(512, 2)
    list_rerun_kernel(const __grid_constant__ FwdArgs<float, CPLX ? 8 : 4> p, const uint32_t *list,
                      const unsigned long long *len) {
  constexpr int NA = CPLX ? 8 : 4;
  const int64_t L = (int64_t)*len;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += step) {
    const uint32_t k = list[i];
    float a[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) a[e] = p.a[e][k];
    RerunAr<CPLX> ar;
    const int32_t s32 = rerun_one<CPLX>(ar, p, k, a);
    if (ar.bad) {                       // the fix-up kernel re-runs it exactly
      p.s[k] = kRedoRerun;
      *p.redo = 1;
    } else {
      p.s[k] = s32;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(p.count, (unsigned long long)L);
}

// Fix-up pass of the re-run form (same stream, after the re-run pass): s =
// kRedoS -- the single-precision method with the general arithmetic, then the
// re-run test and, if it asks, the double-precision re-run (counted);
// s = kRedoRerun -- the double-precision re-run with the general arithmetic
// (already counted).  Reads one word and ends when nothing was flagged.
template <bool CPLX>
__global__ void __launch_bounds__(256)
    rerun_fix_kernel(const __grid_constant__ FwdArgs<float, CPLX ? 8 : 4> p) {
  constexpr int NA = CPLX ? 8 : 4;
  if (*p.redo == 0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.n; k += stride) {
    const int32_t sk = p.s[k];
    if (sk != kRedoS && sk != kRedoRerun) continue;
    bool rerun = sk == kRedoRerun;
    if (!rerun) {
      const SigmaPair<float> r =
          exact_one<float, CPLX>(p.a, p.u, p.v, p.smax, p.smin, p.s, p.flags, k);
      rerun = r.smin < fp<float>::mul(p.tau, r.smax);
      if (rerun) atomicAdd(p.count, 1ull);
    }
    if (rerun) {
      float a[NA];
#pragma unroll
      for (int e = 0; e < NA; ++e) a[e] = p.a[e][k];
      ExactAr<double> ar;
      p.s[k] = rerun_one<CPLX>(ar, p, k, a);
    }
  }
}

// Pass 1 kernels: fwd_kernel with the re-run marks, in the launch shapes of
// the plain single-precision form.
template <bool CPLX>
static FwdKernel<float, CPLX> pick_mark(int mpt, int unroll) {
#define SVD2_PICK(M_, U_) \
  if (mpt == M_ && unroll == U_) return fwd_kernel<float, CPLX, M_, U_, false, true>;
  SVD2_PICK(1, 1) SVD2_PICK(1, 2) SVD2_PICK(2, 1) SVD2_PICK(2, 2) SVD2_PICK(4, 1) SVD2_PICK(4, 2)
#undef SVD2_PICK
  return nullptr;
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
  if (!A || !U || !V || !smax || !smin || !s) return SVD2_EINVAL;
  auto *count = static_cast<unsigned long long *>(workspace);
  auto *list = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(workspace) + kListOffset);
  Launch L = get_launch(op);
  bool vec_ok = aligned(smax, 16) && aligned(smin, 16) && aligned(s, 16);
  for (int e = 0; e < NA; ++e) {
    if (!A[e] || !U[e] || !V[e]) return SVD2_EINVAL;
    vec_ok = vec_ok && aligned(A[e], 16) && aligned(U[e], 16) && aligned(V[e], 16);
  }
  if (!vec_ok) L.mpt = 1;
  auto k = pick_mark<CPLX>(L.mpt, L.unroll);
  if (!k) return SVD2_EINVAL;
  int resident = 0, resident2 = 0;
  SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, L.block, 0));
  SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident2, list_rerun_kernel<CPLX>, 512, 0));
  SVD2_CUDA_TRY(cudaMemsetAsync(count, 0, 2 * sizeof(unsigned long long), stream));
  for (int64_t base = 0; base < n; base += kChunk) {
    const int64_t m = (n - base < kChunk) ? (n - base) : kChunk;
    SVD2_CUDA_TRY(cudaMemsetAsync(count + 2, 0, sizeof(unsigned long long), stream));
    FwdArgs<float, NA> p{};
    for (int e = 0; e < NA; ++e) {
      p.a[e] = A[e] + base;
      p.u[e] = U[e] + base;
      p.v[e] = V[e] + base;
    }
    p.smax = smax + base;
    p.smin = smin + base;
    p.s = s + base;
    p.n = m;
    p.flags = flags;
    p.tau = ldexpf(1.0f, tau_log2);
    p.count = count;
    p.redo = count + 1;
    p.stride = 1;
    const int64_t groups = m / L.mpt, tail = m % L.mpt;
    const int64_t loops = (groups + L.unroll - 1) / L.unroll;
    const int64_t grid = grid_for(loops > tail ? loops : tail, L, resident);
    k<<<(unsigned)grid, L.block, 0, stream>>>(p);
    SVD2_CUDA_TRY(cudaGetLastError());
    const int64_t chunks = (m + 4095) / 4096;
    const int64_t cgrid = chunks < (int64_t)sm_count() * 8 ? chunks : (int64_t)sm_count() * 8;
    compact_kernel<<<(unsigned)cgrid, 256, 0, stream>>>(p.s, m, list, count + 2, aligned(p.s, 16));
    SVD2_CUDA_TRY(cudaGetLastError());
    const int64_t want = (m + 511) / 512;
    const int64_t cap = (int64_t)sm_count() * (resident2 > 0 ? resident2 : 1);
    list_rerun_kernel<CPLX><<<(unsigned)(want < cap ? want : cap), 512, 0, stream>>>(p, list, count + 2);
    SVD2_CUDA_TRY(cudaGetLastError());
    rerun_fix_kernel<CPLX><<<fix_grid(m), 256, 0, stream>>>(p);
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
