// FP32 form with FP64 re-run: svd2_batch_s_rerun / svd2_batch_c_rerun.
//
// Each block takes tiles of consecutive matrices; for a tile it first runs the
// single-precision method (Sec. 1, Sec. 7) on every matrix and flags each
// matrix whose scaled singular values satisfy sigma'_min < 2^tau sigma'_max
// (compared in float; the product by the power of two is exact), queueing its
// index and input elements in shared memory.  Once the queue holds a block's
// worth (and at the end), the whole block re-runs the queued matrices, on
// full warps, with the double-precision method on the exactly widened input,
// and overwrites their outputs with the double results rounded to float,
// sigma' brought to the float run's scale: sigma'_32 = RN32(sigma'_64
// 2^(s32 - s64)).  The re-run reads its inputs from shared memory; its
// scattered stores rewrite lines the block wrote a few tiles earlier, part of
// which have left L2 by then (measured: +74% DRAM reads, +27% writes over
// the algorithmic bytes).  The number of re-run matrices is accumulated in
// the workspace.  A second kernel, the fix-up pass, finishes the matrices the
// fast arithmetic of either precision could not (reads one word otherwise).
#include "svd2_fwd_impl.cuh"

namespace svd2 {

// Workspace layout: [0] re-run count of the call (uint64), [8] the fix-up
// flag of the call (uint64).  The size formula (256 bytes plus 4 per matrix)
// also leaves room for an index list, which this form keeps in shared memory.
constexpr size_t kListOffset = 256;
constexpr int64_t kChunk = int64_t(1) << 31;

// Re-run of one queued matrix in double precision with the arithmetic policy
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
    ad[e] = (double)a[e];
    const unsigned b = fp<float>::bits(a[e]) & fp<float>::kAbs;
    mx = b > mx ? b : mx;
  }
  int32_t s32 = scale_exponent<float>(mx);
  double u[NA], v[NA], sx, sn;
  int32_t s64;
  svd2_one<double, CPLX>(ar, ad, u, v, sx, sn, s64);
  float fx = __double2float_rn(ar.scale(sx, s32 - s64));
  float fn = __double2float_rn(ar.scale(sn, s32 - s64));
  if (p.flags & SVD2_BACKSCALE) {
    if (s32 != kZeroS) {
      fx = ar.template scale_as<float>(fx, -s32);
      fn = ar.template scale_as<float>(fn, -s32);
    }
    s32 = 0;
  }
#pragma unroll
  for (int e = 0; e < NA; ++e) {
    p.u[e][k] = __double2float_rn(u[e]);
    p.v[e][k] = __double2float_rn(v[e]);
  }
  p.smax[k] = fx;
  p.smin[k] = fn;
  return s32;
}

// Queue matrix k (index and input elements) for the double-precision re-run.
template <int NA>
__device__ __forceinline__ void enqueue(uint32_t k, const float *a, uint32_t *q_idx, float *q_a,
                                        int qcap, int *q_n) {
  const int pos = atomicAdd(q_n, 1);      // shared memory; pos < qcap (one slot per matrix)
  q_idx[pos] = k;
#pragma unroll
  for (int e = 0; e < NA; ++e) q_a[e * qcap + pos] = a[e];
}

// The single-precision method on M matrices from k0, queueing the matrices
// whose sigma' ask for the re-run; a matrix the fast arithmetic cannot finish
// gets s = kRedoS (the fix-up kernel then decides its re-run).
template <bool CPLX, int M>
__device__ __forceinline__ void fp32_group(const FwdArgs<float, CPLX ? 8 : 4> &p, int64_t k0,
                                           const float (&in)[CPLX ? 8 : 4][M], uint32_t *q_idx,
                                           float *q_a, int qcap, int *q_n) {
  constexpr int NA = CPLX ? 8 : 4;
  float uo[NA][M], vo[NA][M], sx[M], sn[M];
  int32_t so[M];
  unsigned bad = 0;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    float a[NA], u[NA], v[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) a[e] = in[e][m];
    HotAr<float, CPLX> ar;
    svd2_one<float, CPLX>(ar, a, u, v, sx[m], sn[m], so[m]);
    if (!ar.bad && sn[m] < fp<float>::mul(p.tau, sx[m]))
      enqueue<NA>((uint32_t)(k0 + m), a, q_idx, q_a, qcap, q_n);
    if (p.flags & SVD2_BACKSCALE) backscale(ar, sx[m], sn[m], so[m]);
    so[m] = ar.bad ? kRedoS : so[m];
    bad |= ar.bad;
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      uo[e][m] = u[e];
      vo[e][m] = v[e];
    }
  }
#pragma unroll
  for (int e = 0; e < NA; ++e) store_vec<float, M>(p.u[e] + k0, uo[e]);
#pragma unroll
  for (int e = 0; e < NA; ++e) store_vec<float, M>(p.v[e] + k0, vo[e]);
  store_vec<float, M>(p.smax + k0, sx);
  store_vec<float, M>(p.smin + k0, sn);
  store_vec<int32_t, M>(p.s + k0, so);
  if (bad) *p.redo = 1;
}

// Drain the block's queue -- every queued matrix re-run in double precision --
// once it holds at least `min_fill` entries (0: whatever it holds).  Called by
// every thread of the block; the decision is uniform.
template <bool CPLX>
__device__ __forceinline__ void drain(const FwdArgs<float, CPLX ? 8 : 4> &p, const uint32_t *q_idx,
                                      const float *q_a, int qcap, int *q_n, int min_fill) {
  constexpr int NA = CPLX ? 8 : 4;
  __syncthreads();
  const int qn = *q_n;
  if (qn == 0 || qn < min_fill) return;
  for (int i = threadIdx.x; i < qn; i += blockDim.x) {
    float a[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) a[e] = q_a[e * qcap + i];
    FastAr<double> ar;
    rerun_one<CPLX>(ar, p, q_idx[i], a);
    if (ar.bad) {                       // the fix-up kernel re-runs it exactly
      p.s[q_idx[i]] = kRedoRerun;
      *p.redo = 1;
    }
  }
  if (threadIdx.x == 0) atomicAdd(p.count, (unsigned long long)qn);
  __syncthreads();
  if (threadIdx.x == 0) *q_n = 0;
  __syncthreads();
}

// Tiles of blockDim * M * UNR matrices; every thread of a block runs the same
// number of tile iterations, so the barriers of drain() are uniform.  The
// queue holds one tile plus one block of matrices and is drained when it has
// a block's worth (full warps in the double-precision pass), and at the end.
template <bool CPLX, int M, int UNR>
__global__ void __launch_bounds__(512)
    fused_rerun_kernel(const __grid_constant__ FwdArgs<float, CPLX ? 8 : 4> p) {
  constexpr int NA = CPLX ? 8 : 4;
  extern __shared__ __align__(16) unsigned char smem[];
  const int qcap = blockDim.x * (M * UNR + 1);
  int *q_n = reinterpret_cast<int *>(smem);
  uint32_t *q_idx = reinterpret_cast<uint32_t *>(smem + 16);
  float *q_a = reinterpret_cast<float *>(smem + 16 + (size_t)qcap * sizeof(uint32_t));
  if (threadIdx.x == 0) *q_n = 0;
  __syncthreads();
  const int64_t ngroups = p.n / M;
  const int64_t per_tile = (int64_t)blockDim.x * UNR;      // groups per tile
  const int64_t ntiles = (ngroups + per_tile - 1) / per_tile;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    float in[UNR][NA][M];
#pragma unroll
    for (int r = 0; r < UNR; ++r) {
      const int64_t g = t * per_tile + (int64_t)r * blockDim.x + threadIdx.x;
      if (g < ngroups) {
#pragma unroll
        for (int e = 0; e < NA; ++e) load_vec<float, M>(p.a[e] + g * M, in[r][e]);
      }
    }
#pragma unroll
    for (int r = 0; r < UNR; ++r) {
      const int64_t g = t * per_tile + (int64_t)r * blockDim.x + threadIdx.x;
      if (g < ngroups) fp32_group<CPLX, M>(p, g * M, in[r], q_idx, q_a, qcap, q_n);
    }
    drain<CPLX>(p, q_idx, q_a, qcap, q_n, blockDim.x);
  }
  // the n mod M tail, one matrix per thread of block 0
  const int64_t tail = p.n - ngroups * M;
  if (blockIdx.x == 0 && tail > 0 && threadIdx.x < tail) {
    const int64_t k = ngroups * M + threadIdx.x;
    float in1[NA][1];
#pragma unroll
    for (int e = 0; e < NA; ++e) in1[e][0] = p.a[e][k];
    fp32_group<CPLX, 1>(p, k, in1, q_idx, q_a, qcap, q_n);
  }
  drain<CPLX>(p, q_idx, q_a, qcap, q_n, 0);
}

using FusedKernel4 = void (*)(const FwdArgs<float, 4>);
using FusedKernel8 = void (*)(const FwdArgs<float, 8>);

// Fix-up pass of the re-run form (same stream, after the fused kernel): s =
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

template <bool CPLX>
static auto pick_fused(int mpt, int unroll) -> void (*)(const FwdArgs<float, CPLX ? 8 : 4>) {
#define SVD2_PICK(M_, U_) \
  if (mpt == M_ && unroll == U_) return fused_rerun_kernel<CPLX, M_, U_>;
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
  SVD2_CUDA_TRY(cudaMemsetAsync(count, 0, 2 * sizeof(unsigned long long), stream));
  Launch L = get_launch(op);
  bool vec_ok = aligned(smax, 16) && aligned(smin, 16) && aligned(s, 16);
  for (int e = 0; e < NA; ++e) {
    if (!A[e] || !U[e] || !V[e]) return SVD2_EINVAL;
    vec_ok = vec_ok && aligned(A[e], 16) && aligned(U[e], 16) && aligned(V[e], 16);
  }
  if (!vec_ok) L.mpt = 1;
  auto k = pick_fused<CPLX>(L.mpt, L.unroll);
  if (!k) return SVD2_EINVAL;
  const size_t qcap = (size_t)L.block * (L.mpt * L.unroll + 1);
  const size_t shmem = 16 + qcap * sizeof(uint32_t) + qcap * NA * sizeof(float);
  SVD2_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem));
  int resident = 0;
  SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, L.block, shmem));
  for (int64_t base = 0; base < n; base += kChunk) {
    const int64_t m = (n - base < kChunk) ? (n - base) : kChunk;
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
    const int64_t tiles = (m / L.mpt + (int64_t)L.block * L.unroll - 1) / ((int64_t)L.block * L.unroll);
    const int64_t cap = (int64_t)sm_count() * (resident > 0 ? resident : 1) * (L.waves > 0 ? L.waves : 1 << 20);
    int64_t grid = tiles < 1 ? 1 : tiles;
    if (grid > cap) grid = cap;
    k<<<(unsigned)grid, L.block, shmem, stream>>>(p);
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
