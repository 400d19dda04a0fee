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
  // FP32 forms with FP64 re-run or FP64 tangent step only: the threshold and
  // the counter of the matrices that took the double-precision work.
  T tau;
  unsigned long long *count;
  // Set to nonzero by the fast kernel when it flagged a matrix (see fix_kernel).
  unsigned long long *redo;
  // Elements between consecutive matrices in every array of A, U and V: 1 for
  // the split layout, 4 or 8 for the interleaved (n, 2, 2) layout, where each
  // pointer addresses one element of the first matrix.  smax, smin, s: 1.
  int64_t stride;
};

// s written by the fast kernel for a matrix it could not finish: its outputs
// are recomputed by the fix-up kernel.  (Valid s are -2 .. 2095 and kZeroS.)
constexpr int32_t kRedoS = INT32_MIN;
// FP32 form with re-run: the single-precision results stand but the
// double-precision re-run left its fast domain.
constexpr int32_t kRedoRerun = INT32_MIN + 1;
// FP32 form with re-run, first pass: the matrix asks for the re-run (its
// single-precision sigma' satisfy sigma'_min < 2^tau sigma'_max).
constexpr int32_t kRerunMark = INT32_MIN + 2;

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
// The same with the policy's scaling (FastAr flags results that leave the
// normal range; the fix-up pass then back-scales them exactly).
template <typename T, typename Ar>
__device__ __forceinline__ void backscale(Ar &ar, T &smax, T &smin, int32_t &s) {
  if (s != kZeroS) {
    smax = ar.scale(smax, -s);
    smin = ar.scale(smin, -s);
  }
  s = 0;
}

// One matrix with the given arithmetic policy (Sec. 2 - Sec. 7, Eq. 29; with
// SINE, U by Eq. 31; with VALS, the singular values and s only -- u and v are
// then left zero in the complex method and unspecified in the real one).
template <typename T, bool CPLX, bool SINE = false, bool VALS = false, typename Ar>
__device__ __forceinline__ void svd2_one(Ar &ar, const T *a, T *u, T *v, T &smax, T &smin,
                                         int32_t &s) {
  int piv;
  if constexpr (CPLX)
    svd2_cplx<T, SINE, VALS>(ar, a, u, v, smax, smin, s, piv);
  else
    svd2_real<T, SINE>(ar, a, u, v, smax, smin, s, piv);
}

template <typename T> struct SigmaPair {
  T smax, smin;
};

// Matrix k recomputed with the general arithmetic (ExactAr), its outputs
// stored over whatever the fast kernel stored for it; returns sigma'_max and
// sigma'_min before any back-scaling.  The element arrays may live in any
// address space.
template <typename T, bool CPLX, bool VALS = false, bool SINE = false>
__device__ __forceinline__ SigmaPair<T> exact_one(const T *const *a, T *const *u, T *const *v,
                                                  T *smax, T *smin, int32_t *s, uint32_t flags,
                                                  int64_t k, int64_t stride = 1) {
  constexpr int NA = CPLX ? 8 : 4;
  T ai[NA], uo[NA], vo[NA], sx, sn;
  int32_t so;
#pragma unroll
  for (int e = 0; e < NA; ++e) ai[e] = a[e][k * stride];
  ExactAr<T> ar;
  svd2_one<T, CPLX, SINE, VALS>(ar, ai, uo, vo, sx, sn, so);
  const SigmaPair<T> r{sx, sn};
  if (flags & SVD2_BACKSCALE) backscale(sx, sn, so);
  if constexpr (!VALS) {
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      u[e][k * stride] = uo[e];
      v[e][k * stride] = vo[e];
    }
  }
  smax[k] = sx;
  smin[k] = sn;
  s[k] = so;
  return r;
}

// M matrices from k0 with the batch arithmetic HotAr, stored with vector
// stores; a matrix the fast arithmetic cannot finish gets s = kRedoS and
// raises p.redo.
// MARK (first pass of the FP32 form with re-run): a matrix whose
// single-precision sigma' ask for the double-precision re-run gets
// s = kRerunMark.
// TAN64 (real FP32 form with the FP64 tangent step): the tangent step of
// Eq. 6 - Eq. 7 in double where |r''_22| < p.tau r11; returns the number of
// matrices (not flagged for the fix-up pass) that took it.
template <typename T, bool CPLX, bool TAN64>
struct GroupArOf { using type = HotAr<T, CPLX>; };
template <>
struct GroupArOf<float, false, true> { using type = Tan64Ar<HotAr<float, false>>; };

template <typename T, bool CPLX, int M, bool VALS = false, bool MARK = false, bool TAN64 = false,
          bool SINE = false>
__device__ __forceinline__ unsigned process_group(const FwdArgs<T, CPLX ? 8 : 4> &p, int64_t k0,
                                                  const T (&in)[CPLX ? 8 : 4][M]) {
  constexpr int NA = CPLX ? 8 : 4;
  T uo[NA][M], vo[NA][M], sx[M], sn[M];
  int32_t so[M];
  unsigned bad = 0, nwide = 0;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    T a[NA], u[NA], v[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) a[e] = in[e][m];
    typename GroupArOf<T, CPLX, TAN64>::type ar;
    if constexpr (TAN64) ar.tau = p.tau;
    svd2_one<T, CPLX, SINE, VALS>(ar, a, u, v, sx[m], sn[m], so[m]);
    bool mark = false;
    if constexpr (MARK) mark = sn[m] < fp<T>::mul(p.tau, sx[m]);
    if (p.flags & SVD2_BACKSCALE) backscale(ar, sx[m], sn[m], so[m]);
    // (a matrix handed to the fix-up pass is counted there)
    if constexpr (TAN64) nwide += ar.bad ? 0u : ar.wide;
    so[m] = ar.bad ? kRedoS : mark ? kRerunMark : so[m];
    bad |= ar.bad;
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      uo[e][m] = u[e];
      vo[e][m] = v[e];
    }
  }
  if constexpr (!VALS) {
#pragma unroll
    for (int e = 0; e < NA; ++e) store_vec<T, M>(p.u[e] + k0, uo[e]);
#pragma unroll
    for (int e = 0; e < NA; ++e) store_vec<T, M>(p.v[e] + k0, vo[e]);
  }
  store_vec<T, M>(p.smax + k0, sx);
  store_vec<T, M>(p.smin + k0, sn);
  store_vec<int32_t, M>(p.s + k0, so);
  if (bad) *p.redo = 1;
  return nwide;
}

// Adds each warp's count to *count (one atomic per warp); every lane of the
// warp calls it.
__device__ __forceinline__ void warp_count_add(unsigned long long *count, unsigned c) {
  const unsigned t = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && t) atomicAdd(count, (unsigned long long)t);
}

// Fix-up pass after the fast kernel, on the same stream: if the fast kernel
// flagged any matrix, every matrix with s = kRedoS is recomputed with the
// general arithmetic.  Flagged matrices are those with a zero or subnormal
// divisor or scaled entry, or an exponent out of the fast range: zero columns,
// zero matrices, entries spanning more than the exponent range.  Otherwise the
// pass reads one word and ends.
template <typename T, bool CPLX, bool VALS>
__global__ void __launch_bounds__(256) fix_kernel(const __grid_constant__ FwdArgs<T, CPLX ? 8 : 4> p) {
  if (*p.redo == 0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool sine = (p.flags & SVD2_SINE) != 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.n; k += stride)
    if (p.s[k] == kRedoS) {
      if (sine)
        exact_one<T, CPLX, VALS, true>(p.a, p.u, p.v, p.smax, p.smin, p.s, p.flags, k, p.stride);
      else
        exact_one<T, CPLX, VALS>(p.a, p.u, p.v, p.smax, p.smin, p.s, p.flags, k, p.stride);
    }
}

// Blocks of the fix-up pass: enough to scan a batch quickly when it has work.
inline unsigned fix_grid(int64_t n) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 4;
  return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Minimum resident 512-thread blocks per SM the compiler must allow for: the
// FP64 kernels and the complex FP32 one are bound by arithmetic latency and
// run best at 64 registers (32 warps per SM; complex FP32 at 76 registers
// measured 5% slower); the real FP32 one may use up to 128 (capping it at 32
// registers for full occupancy measured no faster), except with the FP64
// tangent step, whose 76 registers at two matrices per thread left 16 warps
// per SM: at 64 registers it runs 19% faster (56.2 -> 67.0 G matrices/s).
template <typename T, bool CPLX, bool TAN64 = false>
constexpr int kMinBlocks = (sizeof(T) == 8 || CPLX || TAN64) ? 2 : 1;
// The same register budget stated as (threads, 1): 1024 threads for a 64-register
// kernel (two 512-thread blocks' worth), which also admits 1024-thread blocks.
template <typename T, bool CPLX, bool TAN64 = false>
constexpr int kMaxThreads = kMinBlocks<T, CPLX, TAN64> == 2 ? 1024 : 512;

template <typename T, bool CPLX, int M, int UNR, bool VALS = false, bool MARK = false,
          bool TAN64 = false, bool SINE = false>
__global__ void __launch_bounds__((kMaxThreads<T, CPLX, TAN64>), 1)
    fwd_kernel(const __grid_constant__ FwdArgs<T, CPLX ? 8 : 4> p) {
  constexpr int NA = CPLX ? 8 : 4;
  unsigned nwide = 0;
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
      if (g < ngroups)
        nwide += process_group<T, CPLX, M, VALS, MARK, TAN64, SINE>(p, g * M, in[r]);
    }
  }
  // the n mod M tail, one matrix per thread
  const int64_t k = ngroups * M + tid;
  if (tid < p.n - ngroups * M) {
    T in1[NA][1];
#pragma unroll
    for (int e = 0; e < NA; ++e) in1[e][0] = p.a[e][k];
    nwide += process_group<T, CPLX, 1, VALS, MARK, TAN64, SINE>(p, k, in1);
  }
  if constexpr (TAN64) {
    if (p.count) warp_count_add(p.count, nwide);
  }
}

// The interleaved layout (p.stride == NA, each matrix one contiguous record):
// one matrix per thread.  REC: the record is moved with 16-byte vector loads
// and stores (every base pointer 16-byte aligned; a record is 16, 32 or 64
// bytes) and permuted to the record order of Sec. 8 in registers; otherwise
// element loads and stores at the layout's stride.
template <bool CPLX> constexpr int interleaved_offset(int e);

template <typename T, bool CPLX, bool VALS, bool REC>
__global__ void __launch_bounds__(256, 2 * kMinBlocks<T, CPLX>) strided_kernel(const __grid_constant__ FwdArgs<T, CPLX ? 8 : 4> p) {
  constexpr int NA = CPLX ? 8 : 4;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.n; k += step) {
    T a[NA], u[NA], v[NA], sx, sn;
    int32_t so;
    if constexpr (REC) {
      T rec[NA];
      load_vec<T, NA>(p.a[0] + k * NA, rec);
#pragma unroll
      for (int e = 0; e < NA; ++e) a[e] = rec[interleaved_offset<CPLX>(e)];
    } else {
#pragma unroll
      for (int e = 0; e < NA; ++e) a[e] = __ldcs(p.a[e] + k * p.stride);
    }
    HotAr<T, CPLX> ar;
    svd2_one<T, CPLX, false, VALS>(ar, a, u, v, sx, sn, so);
    if (p.flags & SVD2_BACKSCALE) backscale(ar, sx, sn, so);
    if constexpr (!VALS) {
      if constexpr (REC) {
        T ru[NA], rv[NA];
#pragma unroll
        for (int e = 0; e < NA; ++e) {
          ru[interleaved_offset<CPLX>(e)] = u[e];
          rv[interleaved_offset<CPLX>(e)] = v[e];
        }
        store_vec<T, NA>(p.u[0] + k * NA, ru);
        store_vec<T, NA>(p.v[0] + k * NA, rv);
      } else {
#pragma unroll
        for (int e = 0; e < NA; ++e) {
          __stcs(p.u[e] + k * p.stride, u[e]);
          __stcs(p.v[e] + k * p.stride, v[e]);
        }
      }
    }
    __stcs(p.smax + k, sx);
    __stcs(p.smin + k, sn);
    __stcs(p.s + k, ar.bad ? kRedoS : so);
    if (ar.bad) *p.redo = 1;
  }
}

template <typename T, bool CPLX>
using FwdKernel = void (*)(const FwdArgs<T, CPLX ? 8 : 4>);

// The values-only kernels and those with the assembly of Eq. 31 exist for one
// load group in flight only.
template <typename T, bool CPLX>
inline FwdKernel<T, CPLX> pick_kernel(int mpt, int unroll, bool vals, bool sine = false) {
  if (sine) {
    if (mpt == 1) return fwd_kernel<T, CPLX, 1, 1, false, false, false, true>;
    if (mpt == 2) return fwd_kernel<T, CPLX, 2, 1, false, false, false, true>;
    if (mpt == 4) return fwd_kernel<T, CPLX, 4, 1, false, false, false, true>;
    return nullptr;
  }
#define SVD2_PICK(M_, U_) \
  if (mpt == M_ && unroll == U_) return fwd_kernel<T, CPLX, M_, U_, false>;
  if (!vals) {
    SVD2_PICK(1, 1) SVD2_PICK(1, 2) SVD2_PICK(2, 1) SVD2_PICK(2, 2) SVD2_PICK(4, 1) SVD2_PICK(4, 2)
    return nullptr;
  }
#undef SVD2_PICK
  if (mpt == 1) return fwd_kernel<T, CPLX, 1, 1, true>;
  if (mpt == 2) return fwd_kernel<T, CPLX, 2, 1, true>;
  if (mpt == 4) return fwd_kernel<T, CPLX, 4, 1, true>;
  return nullptr;
}

// Validate the arguments, fill p and launch the forward kernel for op on n
// matrices.  vals: singular values only (U, V neither computed nor stored,
// Uo and Vo may be NULL).  stride: elements between consecutive matrices in
// the arrays of A, U and V (1: split layout).  Returns an SVD2_* code.
template <typename T, bool CPLX>
inline int launch_fwd(int op, int64_t n, const T *const *A, T *const *Uo, T *const *Vo, T *smax,
                      T *smin, int32_t *s, uint32_t flags, cudaStream_t stream,
                      FwdArgs<T, CPLX ? 8 : 4> &p, bool vals = false, int64_t stride = 1) {
  constexpr int NA = CPLX ? 8 : 4;
  if (n < 0 || stride < 1 || (flags & ~(SVD2_BACKSCALE | SVD2_SINE))) return SVD2_EINVAL;
  // Eq. 31 is an assembly of U: for the split layout's full forms only
  if ((flags & SVD2_SINE) && (stride > 1 || vals)) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!A || (!vals && (!Uo || !Vo)) || !smax || !smin || !s) return SVD2_EINVAL;
  bool vec_ok = stride == 1 && aligned(smax, 16) && aligned(smin, 16) && aligned(s, 16);
  for (int e = 0; e < NA; ++e) {
    if (!A[e] || (!vals && (!Uo[e] || !Vo[e]))) return SVD2_EINVAL;
    p.a[e] = A[e];
    p.u[e] = vals ? nullptr : Uo[e];
    p.v[e] = vals ? nullptr : Vo[e];
    vec_ok = vec_ok && aligned(A[e], 16) && (vals || (aligned(Uo[e], 16) && aligned(Vo[e], 16)));
  }
  p.smax = smax;
  p.smin = smin;
  p.s = s;
  p.n = n;
  p.flags = flags;
  p.stride = stride;
  FwdKernel<T, CPLX> k = nullptr;
  int64_t grid = 0;
  unsigned block = 256;
  if (stride > 1) {
    // whole records when the layout is the interleaved one and every base is aligned
    const bool rec = stride == NA && aligned(A[0], 16) &&
                     (vals || (aligned(Uo[0], 16) && aligned(Vo[0], 16)));
    if (rec)
      k = vals ? strided_kernel<T, CPLX, true, true> : strided_kernel<T, CPLX, false, true>;
    else
      k = vals ? strided_kernel<T, CPLX, true, false> : strided_kernel<T, CPLX, false, false>;
    const int64_t want = (n + 255) / 256;
    grid = want < 0x7fffffffLL ? want : 0x7fffffffLL;
  } else {
    Launch L = get_launch(op);
    const bool sine = (flags & SVD2_SINE) && !vals;
    if (!vec_ok) L.mpt = 1;
    if (vals || sine) L.unroll = 1;
    k = pick_kernel<T, CPLX>(L.mpt, L.unroll, vals, sine);
    if (!k) return SVD2_EINVAL;
    int resident = 0;
    SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, L.block, 0));
    const int64_t groups = n / L.mpt;
    const int64_t tail = n % L.mpt;
    const int64_t loops = (groups + L.unroll - 1) / L.unroll;
    const int64_t units = loops > tail ? loops : tail;   // threads needed
    grid = grid_for(units, L, resident);
    block = (unsigned)L.block;
  }
  // the batch kernel, then the fix-up pass, which reads the flag word and
  // ends unless the batch kernel flagged a matrix
  void *flag = nullptr;
  int rc = flag_block(stream, &flag);
  if (rc != SVD2_OK) return rc;
  p.redo = static_cast<unsigned long long *>(flag);
  k<<<(unsigned)grid, block, 0, stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    if (vals)
      fix_kernel<T, CPLX, true><<<fix_grid(n), 256, 0, stream>>>(p);
    else
      fix_kernel<T, CPLX, false><<<fix_grid(n), 256, 0, stream>>>(p);
    e = cudaGetLastError();
  }
  rc = flag_release(flag, stream);
  if (e != cudaSuccess) return record_cuda_error(e);
  return rc;
}

// The interleaved layout of a (n, 2, 2) row-major array (torch's layout for a
// batch of 2x2 real or complex matrices): matrix k's entries are contiguous,
// real: a11 a12 a21 a22; complex: Re a11, Im a11, Re a12, Im a12, Re a21,
// Im a21, Re a22, Im a22.  Offset of the record-order element e (Sec. 8:
// a11, a21, a12, a22, real and imaginary parts interleaved) in one matrix.
template <bool CPLX> constexpr int interleaved_offset(int e) {
  if (CPLX) {
    const int elem = e >> 1, part = e & 1;             // elem: a11, a21, a12, a22
    const int rm = (elem == 1) ? 2 : (elem == 2) ? 1 : elem;   // row-major position
    return 2 * rm + part;
  }
  return (e == 1) ? 2 : (e == 2) ? 1 : e;
}

// launch_fwd on an interleaved batch at base pointers A, U, V.
template <typename T, bool CPLX>
inline int launch_interleaved(int op, int64_t n, const T *A, T *U, T *V, T *smax, T *smin,
                              int32_t *s, uint32_t flags, cudaStream_t stream, bool vals) {
  constexpr int NA = CPLX ? 8 : 4;
  if (n < 0 || (flags & ~SVD2_BACKSCALE)) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!A || (!vals && (!U || !V))) return SVD2_EINVAL;
  const T *a[NA];
  T *u[NA], *v[NA];
  for (int e = 0; e < NA; ++e) {
    a[e] = A + interleaved_offset<CPLX>(e);
    u[e] = vals ? nullptr : U + interleaved_offset<CPLX>(e);
    v[e] = vals ? nullptr : V + interleaved_offset<CPLX>(e);
  }
  FwdArgs<T, NA> p{};
  return launch_fwd<T, CPLX>(op, n, a, u, v, smax, smin, s, flags, stream, p, vals, NA);
}

}  // namespace svd2
