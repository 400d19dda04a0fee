// Forward kernel template of the plain forms (svd2_fwd_{d,z,s,c}.cu); its
// argument block, vector helpers and back-scaling are shared with the FP32 form
// with FP64 re-run (svd2_rerun.cu).
//
// One thread owns `mpt` consecutive matrices of the split layout (Sec. 3) per
// load group and keeps everything in registers from the load of A to the
// store of U, V, Sigma' and s -- the register-resident pipeline of Sec. 4,
// with a CUDA thread in place of an AVX-512 lane.  Loads and stores are
// 16-byte streaming accesses on every element array, so each warp moves whole
// 32-byte sectors of each of the 4 (real) or 8 (complex) input and 11 or 19
// output streams.
#pragma once
#include "svd2_common.cuh"
#include "svd2_math.cuh"

namespace svd2 {

template <typename T, int NA>
struct FwdArgs {
  const T *a[NA];
  T *u[NA];
  T *v[NA];
  T *smax;
  T *smin;
  int32_t *s;
  int64_t n;
  uint32_t flags;
  // FP32 form with FP64 re-run only: re-run threshold and re-run counter.
  T tau;
  unsigned long long *count;
};

// Optional back-scaling of Fig. 1: Sigma = 2^-s Sigma' (correctly rounded,
// may overflow or underflow), then s = 0.
template <typename T>
__device__ __forceinline__ void backscale(T &smax, T &smin, int32_t &s) {
  if (s != kZeroS) {
    smax = scalef(smax, -s);
    smin = scalef(smin, -s);
  }
  s = 0;
}

template <typename T, bool CPLX, int M>
__device__ __forceinline__ void process_group(const FwdArgs<T, CPLX ? 8 : 4> &p, int64_t k0,
                                              const T (&in)[CPLX ? 8 : 4][M]) {
  constexpr int NA = CPLX ? 8 : 4;
  T uo[NA][M], vo[NA][M], sx[M], sn[M];
  int32_t so[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    T a[NA], u[NA], v[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) a[e] = in[e][m];
    int piv;
    if constexpr (CPLX)
      svd2_cplx<T>(a, u, v, sx[m], sn[m], so[m], piv);
    else
      svd2_real<T>(a, u, v, sx[m], sn[m], so[m], piv);
    if (p.flags & SVD2_BACKSCALE) backscale(sx[m], sn[m], so[m]);
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      uo[e][m] = u[e];
      vo[e][m] = v[e];
    }
  }
#pragma unroll
  for (int e = 0; e < NA; ++e) store_vec<T, M>(p.u[e] + k0, uo[e]);
#pragma unroll
  for (int e = 0; e < NA; ++e) store_vec<T, M>(p.v[e] + k0, vo[e]);
  store_vec<T, M>(p.smax + k0, sx);
  store_vec<T, M>(p.smin + k0, sn);
  store_vec<int32_t, M>(p.s + k0, so);
}

// Minimum resident 512-thread blocks per SM the compiler must allow for: the
// complex FP64 kernel is bound by arithmetic latency and runs best at 64
// registers (32 warps per SM at 256 threads); the others may use up to 128.
template <typename T, bool CPLX> constexpr int kMinBlocks = (sizeof(T) == 8 && CPLX) ? 2 : 1;

template <typename T, bool CPLX, int M, int UNR>
__global__ void __launch_bounds__(512, kMinBlocks<T, CPLX>) fwd_kernel(const FwdArgs<T, CPLX ? 8 : 4> p) {
  constexpr int NA = CPLX ? 8 : 4;
  const int64_t ngroups = p.n / M;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t g0 = tid; g0 < ngroups; g0 += stride * UNR) {
    T in[UNR][NA][M];
#pragma unroll
    for (int r = 0; r < UNR; ++r) {
      const int64_t g = g0 + r * stride;
      if (g < ngroups) {
#pragma unroll
        for (int e = 0; e < NA; ++e) load_vec<T, M>(p.a[e] + g * M, in[r][e]);
      }
    }
#pragma unroll
    for (int r = 0; r < UNR; ++r) {
      const int64_t g = g0 + r * stride;
      if (g < ngroups) process_group<T, CPLX, M>(p, g * M, in[r]);
    }
  }
  // the n mod M tail, one matrix per thread
  const int64_t k = ngroups * M + tid;
  if (tid < p.n - ngroups * M) {
    T in1[NA][1];
#pragma unroll
    for (int e = 0; e < NA; ++e) in1[e][0] = p.a[e][k];
    process_group<T, CPLX, 1>(p, k, in1);
  }
}

template <typename T, bool CPLX>
using FwdKernel = void (*)(const FwdArgs<T, CPLX ? 8 : 4>);

template <typename T, bool CPLX>
inline FwdKernel<T, CPLX> pick_kernel(int mpt, int unroll) {
#define SVD2_PICK(M_, U_) \
  if (mpt == M_ && unroll == U_) return fwd_kernel<T, CPLX, M_, U_>;
  SVD2_PICK(1, 1) SVD2_PICK(1, 2) SVD2_PICK(2, 1) SVD2_PICK(2, 2) SVD2_PICK(4, 1) SVD2_PICK(4, 2)
#undef SVD2_PICK
  return nullptr;
}

// Validate the arguments, fill p and launch the forward kernel for op on n
// matrices.  Returns an SVD2_* code.
template <typename T, bool CPLX>
inline int launch_fwd(int op, int64_t n, const T *const *A, T *const *Uo, T *const *Vo, T *smax,
                      T *smin, int32_t *s, uint32_t flags, cudaStream_t stream,
                      FwdArgs<T, CPLX ? 8 : 4> &p) {
  constexpr int NA = CPLX ? 8 : 4;
  if (n < 0 || (flags & ~SVD2_BACKSCALE)) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!A || !Uo || !Vo || !smax || !smin || !s) return SVD2_EINVAL;
  bool vec_ok = aligned(smax, 16) && aligned(smin, 16) && aligned(s, 16);
  for (int e = 0; e < NA; ++e) {
    if (!A[e] || !Uo[e] || !Vo[e]) return SVD2_EINVAL;
    p.a[e] = A[e];
    p.u[e] = Uo[e];
    p.v[e] = Vo[e];
    vec_ok = vec_ok && aligned(A[e], 16) && aligned(Uo[e], 16) && aligned(Vo[e], 16);
  }
  p.smax = smax;
  p.smin = smin;
  p.s = s;
  p.n = n;
  p.flags = flags;
  Launch L = get_launch(op);
  if (!vec_ok) L.mpt = 1;
  FwdKernel<T, CPLX> k = pick_kernel<T, CPLX>(L.mpt, L.unroll);
  if (!k) return SVD2_EINVAL;
  int resident = 0;
  SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, L.block, 0));
  const int64_t groups = n / L.mpt;
  const int64_t tail = n % L.mpt;
  const int64_t loops = (groups + L.unroll - 1) / L.unroll;
  const int64_t units = loops > tail ? loops : tail;   // threads needed
  const int64_t grid = grid_for(units, L, resident);
  k<<<(unsigned)grid, L.block, 0, stream>>>(p);
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}

}  // namespace svd2
