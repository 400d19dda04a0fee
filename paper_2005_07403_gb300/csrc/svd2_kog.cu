// One parallel step of the Kogbetliantz method (Sec. 1): svd2_kog_step_{d,z,s,c}.
//
// The iteration matrix G of order m = 2n and n pivot pairs (p_k, q_k) (a
// permutation of 0 .. m-1).  The batch of Sec. 1 is the n pivot blocks
// A^[k] = [[G(p,p), G(p,q)], [G(q,p), G(q,q)]]; after A^[k] = U Sigma V^*,
// G is updated from the left by U^* on rows p_k, q_k and from the right by V
// on columns p_k, q_k.  Rows p_k, q_k and columns p_j, q_j meet in a 2x2
// block, so the update is one independent product per block,
//   G'[{p_k, q_k}, {p_j, q_j}] = (U^[k])^* G[{p_k, q_k}, {p_j, q_j}] V^[j],
// and the pivot block (j = k) becomes Sigma^[k] exactly (off-diagonal pivot
// positions annihilated).  Two kernels on the caller's stream:
//  kog_pivot_kernel   one thread per pair: gather A^[k], the method with the
//                     general arithmetic and the back-scaling of Fig. 1, U, V,
//                     Sigma into the workspace (split layout);
//  kog_update_kernel  in place, 2x2 blocks: read the block, multiply by U^*
//                     and V, store.  Threads along x take the pairs of the
//                     unit-stride dimension (rows of a column-major G, columns
//                     of a row-major one) and up to 8 blocks each along y, so
//                     a warp reads and writes contiguous runs -- with one
//                     vector access per two neighbours -- when the pairs are
//                     (2i, 2i+1); each thread keeps its own U^[k] (or V^[j])
//                     and the other factor is uniform across the warp.
// The update reads and writes G once: 2 m^2 elements of HBM traffic; in
// double precision it is bound by the FP64 pipe (64 operations per complex
// block, 16 per real one).
#include "svd2_fwd_impl.cuh"

namespace svd2 {

template <typename T, bool CPLX>
struct KogArgs {
  T *g;                    // real: G(r, c) = g[r rs + c cs]; complex: Re, Im at 2 (r rs + c cs) + 0, 1
  int64_t rs, cs;
  const int32_t *pairs;    // p_0, q_0, p_1, q_1, ...
  int64_t m, npairs;
  T *u[CPLX ? 8 : 4];      // workspace: U^[k], V^[k] in the record order of Sec. 8
  T *v[CPLX ? 8 : 4];
  T *smax, *smin;          // Sigma^[k] (back-scaled)
  unsigned long long *skipped;
};

template <typename T, bool CPLX>
__device__ __forceinline__ void g_load(const KogArgs<T, CPLX> &p, int64_t r, int64_t c, T &re,
                                       T &im) {
  const int64_t o = r * p.rs + c * p.cs;
  if constexpr (CPLX) {
    re = p.g[2 * o];
    im = p.g[2 * o + 1];
  } else {
    re = p.g[o];
    im = T(0);
  }
}

template <typename T, bool CPLX>
__device__ __forceinline__ void g_store(const KogArgs<T, CPLX> &p, int64_t r, int64_t c, T re,
                                        T im) {
  const int64_t o = r * p.rs + c * p.cs;
  if constexpr (CPLX) {
    p.g[2 * o] = re;
    p.g[2 * o + 1] = im;
  } else {
    p.g[o] = re;
  }
}

__device__ __forceinline__ bool pair_ok(int32_t a, int32_t b, int64_t m) {
  return a >= 0 && b >= 0 && a < m && b < m && a != b;
}

template <typename T, bool CPLX>
__global__ void __launch_bounds__(256) kog_pivot_kernel(const __grid_constant__ KogArgs<T, CPLX> p) {
  constexpr int NA = CPLX ? 8 : 4;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.npairs; k += step) {
    const int32_t pk = p.pairs[2 * k], qk = p.pairs[2 * k + 1];
    if (!pair_ok(pk, qk, p.m)) {
      atomicAdd(p.skipped, 1ull);
      continue;
    }
    // A^[k] column by column (Sec. 1): a11 = G(p,p), a21 = G(q,p), a12 = G(p,q), a22 = G(q,q)
    T a[NA];
    const int32_t rr[4] = {pk, qk, pk, qk}, cc[4] = {pk, pk, qk, qk};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      T re, im;
      g_load(p, rr[e], cc[e], re, im);
      if constexpr (CPLX) {
        a[2 * e] = re;
        a[2 * e + 1] = im;
      } else {
        a[e] = re;
      }
    }
    T u[NA], v[NA], sx, sn;
    int32_t s;
    ExactAr<T> ar;
    svd2_one<T, CPLX>(ar, a, u, v, sx, sn, s);
    backscale(sx, sn, s);
#pragma unroll
    for (int e = 0; e < NA; ++e) {
      p.u[e][k] = u[e];
      p.v[e][k] = v[e];
    }
    p.smax[k] = sx;
    p.smin[k] = sn;
  }
}

// The multiplication that starts each fma chain of the update: the hardware
// instruction, or for doubles the integer-pipe form (sfp::mul_fast, the same
// bits; it sets bad for operands or a product outside the normal range), which
// moves that operation off the FP64 pipe (2 operations per clock per SM).
struct HwMul {
  template <typename T> __device__ __forceinline__ T operator()(T a, T b) const {
    return fp<T>::mul(a, b);
  }
};
struct IntMul {
  unsigned &bad;
  __device__ __forceinline__ double operator()(double a, double b) const {
    return sfp::mul_fast(a, b, bad);
  }
};

// Complex 2x2 entries: (re, im) pairs in the record order of Sec. 8
// (x11, x21, x12, x22).  Sums of two products as fma chains.
template <typename T, typename Mul>
__device__ __forceinline__ void conj_dot2(T xr1, T xi1, T yr1, T yi1, T xr2, T xi2, T yr2, T yi2,
                                          T &re, T &im, const Mul &mul) {
  using F = fp<T>;
  // conj(x1) y1 + conj(x2) y2
  re = F::fma(xr1, yr1, F::fma(xi1, yi1, F::fma(xr2, yr2, mul(xi2, yi2))));
  im = F::fma(xr1, yi1, F::fma(f_neg(xi1), yr1, F::fma(xr2, yi2, f_neg(mul(xi2, yr2)))));
}
template <typename T, typename Mul>
__device__ __forceinline__ void dot2(T xr1, T xi1, T yr1, T yi1, T xr2, T xi2, T yr2, T yi2,
                                     T &re, T &im, const Mul &mul) {
  using F = fp<T>;
  // x1 y1 + x2 y2
  re = F::fma(xr1, yr1, F::fma(f_neg(xi1), yi1, F::fma(xr2, yr2, f_neg(mul(xi2, yi2)))));
  im = F::fma(xr1, yi1, F::fma(xi1, yr1, F::fma(xr2, yi2, mul(xi2, yr2))));
}

// B' = U^* B V for 2x2 matrices (element order x11, x21, x12, x22; complex:
// separate real and imaginary arrays).
template <typename T, bool CPLX, typename Mul, typename Mul2 = Mul>
__device__ __forceinline__ void two_sided(const T *ur, const T *ui, const T *vr, const T *vi,
                                          T *br, T *bi, const Mul &mul, const Mul2 &mul2) {
  using F = fp<T>;
  T tr[4], ti[4];
  // T = U^* B: t_xy = conj(u_0x) b_0y + conj(u_1x) b_1y (0-based x, y; the
  // element (x, y) has index x + 2 y)
#pragma unroll
  for (int x = 0; x < 2; ++x) {
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int t = x + 2 * y, u1 = 2 * x, u2 = 2 * x + 1, b1 = 2 * y, b2 = 2 * y + 1;
      if constexpr (CPLX) {
        conj_dot2(ur[u1], ui[u1], br[b1], bi[b1], ur[u2], ui[u2], br[b2], bi[b2], tr[t], ti[t], mul);
      } else {
        tr[t] = F::fma(ur[u1], br[b1], mul(ur[u2], br[b2]));
        ti[t] = T(0);
      }
    }
  }
  // B' = T V: b'_xy = t_x1 v_1y + t_x2 v_2y
#pragma unroll
  for (int x = 0; x < 2; ++x) {
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int o = x + 2 * y, t1 = x, t2 = x + 2, v1 = 2 * y, v2 = 2 * y + 1;
      if constexpr (CPLX) {
        dot2(tr[t1], ti[t1], vr[v1], vi[v1], tr[t2], ti[t2], vr[v2], vi[v2], br[o], bi[o], mul2);
      } else {
        br[o] = F::fma(tr[t1], vr[v1], mul2(tr[t2], vr[v2]));
      }
    }
  }
}

template <typename T, bool CPLX>
__device__ __forceinline__ void load_factor(T *const *w, int64_t k, T *r, T *i) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if constexpr (CPLX) {
      r[e] = w[2 * e][k];
      i[e] = w[2 * e + 1][k];
    } else {
      r[e] = w[e][k];
      i[e] = T(0);
    }
  }
}

// Two entries that are neighbours along the unit-stride dimension (linear
// offsets o and o + 1): one vector access when `vec` (the pair (o, o + 1) is
// aligned to its size, or to 16 bytes for complex doubles), else two.
template <typename T, bool CPLX>
__device__ __forceinline__ void g_load2(const KogArgs<T, CPLX> &p, int64_t o, bool vec, T &r0,
                                        T &i0, T &r1, T &i1) {
  if (vec) {
    if constexpr (CPLX) {
      T w[4];
      load_vec<T, 4>(p.g + 2 * o, w);
      r0 = w[0]; i0 = w[1]; r1 = w[2]; i1 = w[3];
    } else {
      T w[2];
      load_vec<T, 2>(p.g + o, w);
      r0 = w[0]; r1 = w[1];
      i0 = i1 = T(0);
    }
  } else if constexpr (CPLX) {
    r0 = p.g[2 * o]; i0 = p.g[2 * o + 1]; r1 = p.g[2 * o + 2]; i1 = p.g[2 * o + 3];
  } else {
    r0 = p.g[o]; r1 = p.g[o + 1];
    i0 = i1 = T(0);
  }
}

template <typename T, bool CPLX>
__device__ __forceinline__ void g_store2(const KogArgs<T, CPLX> &p, int64_t o, bool vec, T r0,
                                         T i0, T r1, T i1) {
  if (vec) {
    if constexpr (CPLX) {
      const T w[4] = {r0, i0, r1, i1};
      store_vec<T, 4>(p.g + 2 * o, w);
    } else {
      const T w[2] = {r0, r1};
      store_vec<T, 2>(p.g + o, w);
    }
  } else if constexpr (CPLX) {
    p.g[2 * o] = r0; p.g[2 * o + 1] = i0; p.g[2 * o + 2] = r1; p.g[2 * o + 3] = i1;
  } else {
    p.g[o] = r0; p.g[o + 1] = r1;
  }
}

// Launch shape of the update kernel, by measurement at m = 8192 (column-major,
// pairs (2i, 2i+1)): complex doubles in blocks of 128 with at least 5 resident
// per SM (96 registers; 1.38 ms against 1.49 at 2 blocks of 256 and 122
// registers, 1.41 at 3 blocks and 80); real doubles 4 blocks of 256 (64
// registers; 0.38 ms against 0.39 at 3 blocks and 76); floats as the compiler
// allots.
template <typename T, bool CPLX> struct KogShape {
  static constexpr int block = (CPLX && sizeof(T) == 8) ? 128 : 256;
  static constexpr int min_blocks = sizeof(T) != 8 ? 0 : CPLX ? 5 : 4;
};

template <typename T, bool CPLX, bool ROWS_FAST>
__global__ void __launch_bounds__(KogShape<T, CPLX>::block, KogShape<T, CPLX>::min_blocks)
    kog_update_kernel(const __grid_constant__ KogArgs<T, CPLX> p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.npairs) return;
  const int32_t pi = p.pairs[2 * i], qi = p.pairs[2 * i + 1];
  if (!pair_ok(pi, qi, p.m)) return;
  // the thread's own pair lies along the unit-stride dimension: rows of a
  // column-major G, columns of a row-major one
  const bool adjacent = qi == pi + 1;
  constexpr uintptr_t kAlign = (!CPLX && sizeof(T) == 4) ? 8 : 16;
  const int64_t ostride = ROWS_FAST ? p.cs : p.rs;   // step between the other dimension's lines
  // the thread's own factor: U^[i] (rows fast) or V^[i] (columns fast)
  T fr[4], fi[4];
  load_factor<T, CPLX>(ROWS_FAST ? p.u : p.v, i, fr, fi);
  for (int64_t jj = blockIdx.y; jj < p.npairs; jj += gridDim.y) {
    const int32_t pj = p.pairs[2 * jj], qj = p.pairs[2 * jj + 1];
    if (!pair_ok(pj, qj, p.m)) continue;
    const int64_t k = ROWS_FAST ? i : jj;
    const int32_t pk = ROWS_FAST ? pi : pj, qk = ROWS_FAST ? qi : qj;   // row pair
    if (i == jj) {   // the pivot block: Sigma^[k]
      g_store(p, pk, pk, p.smax[k], T(0));
      g_store(p, qk, pk, T(0), T(0));
      g_store(p, pk, qk, T(0), T(0));
      g_store(p, qk, qk, p.smin[k], T(0));
      continue;
    }
    // the two lines of the other dimension (columns pj, qj of a column-major
    // G): offsets of the own pair's first entry on each line
    const int64_t o0 = (int64_t)pi + (int64_t)pj * ostride;
    const int64_t o1 = (int64_t)pi + (int64_t)qj * ostride;
    const bool v0 = adjacent && (reinterpret_cast<uintptr_t>(p.g + (CPLX ? 2 : 1) * o0) % kAlign) == 0;
    const bool v1 = adjacent && (reinterpret_cast<uintptr_t>(p.g + (CPLX ? 2 : 1) * o1) % kAlign) == 0;
    // block in the record order (x11, x21, x12, x22) of rows (pk, qk) x columns (pc, qc)
    T gr[4], gi[4];
    auto load_block = [&]() {
    if (adjacent) {
      // rows fast: line pj holds (pk,pc),(qk,pc) = record 0, 1; line qj holds 2, 3.
      // columns fast: line pj (a row) holds (pk,pc),(pk,qc) = record 0, 2; line qj holds 1, 3.
      if constexpr (ROWS_FAST) {
        g_load2(p, o0, v0, gr[0], gi[0], gr[1], gi[1]);
        g_load2(p, o1, v1, gr[2], gi[2], gr[3], gi[3]);
      } else {
        g_load2(p, o0, v0, gr[0], gi[0], gr[2], gi[2]);
        g_load2(p, o1, v1, gr[1], gi[1], gr[3], gi[3]);
      }
    } else {
      const int32_t pc = ROWS_FAST ? pj : pi, qc = ROWS_FAST ? qj : qi;   // column pair
      g_load(p, pk, pc, gr[0], gi[0]);
      g_load(p, qk, pc, gr[1], gi[1]);
      g_load(p, pk, qc, gr[2], gi[2]);
      g_load(p, qk, qc, gr[3], gi[3]);
    }
    };
    load_block();
    T or_[4], oi[4];   // the other factor, uniform across the warp
    load_factor<T, CPLX>(ROWS_FAST ? p.v : p.u, jj, or_, oi);
    auto apply = [&](const auto &mul, const auto &mul2) {
      if constexpr (ROWS_FAST)
        two_sided<T, CPLX>(fr, fi, or_, oi, gr, gi, mul, mul2);
      else
        two_sided<T, CPLX>(or_, oi, fr, fi, gr, gi, mul, mul2);
    };
    if constexpr (sizeof(T) == 8) {
      // doubles: leading products of the fma chains on the integer pipe --
      // all 16 of a complex block (64 FP64 operations; 1.85 -> 1.49 ms at
      // m = 8192 in the same launch shape), the 4 of the first stage of a
      // real one (16 operations; 0.49 -> 0.38 ms); a block with an operand or
      // product outside the multiply's domain (zero, subnormal, overflow) is
      // read again and done with the hardware multiplication (nothing is
      // stored before this point)
      unsigned bad = 0;
      if constexpr (CPLX)
        apply(IntMul{bad}, IntMul{bad});
      else   // the 4 products of U^* B (all 8: 0.49 ms against 0.38)
        apply(IntMul{bad}, HwMul{});
      if (__any_sync(__activemask(), bad != 0)) {
        if (bad) {
          asm volatile("" ::: "memory");   // a fresh read, not the first one's registers
          load_block();
          apply(HwMul{}, HwMul{});
        }
      }
    } else {
      apply(HwMul{}, HwMul{});
    }
    if (adjacent) {
      if constexpr (ROWS_FAST) {
        g_store2(p, o0, v0, gr[0], gi[0], gr[1], gi[1]);
        g_store2(p, o1, v1, gr[2], gi[2], gr[3], gi[3]);
      } else {
        g_store2(p, o0, v0, gr[0], gi[0], gr[2], gi[2]);
        g_store2(p, o1, v1, gr[1], gi[1], gr[3], gi[3]);
      }
    } else {
      const int32_t pc = ROWS_FAST ? pj : pi, qc = ROWS_FAST ? qj : qi;
      g_store(p, pk, pc, gr[0], gi[0]);
      g_store(p, qk, pc, gr[1], gi[1]);
      g_store(p, pk, qc, gr[2], gi[2]);
      g_store(p, qk, qc, gr[3], gi[3]);
    }
  }
}

constexpr size_t kKogHeader = 256;

inline size_t round256(size_t b) { return (b + 255) / 256 * 256; }

template <typename T, bool CPLX>
size_t kog_ws_bytes(int64_t m) {
  constexpr int NA = CPLX ? 8 : 4;
  const int64_t n = m / 2;
  return kKogHeader + (size_t)(2 * NA + 2) * round256((size_t)n * sizeof(T));
}

template <typename T, bool CPLX>
int kog_step(int64_t m, T *G, int64_t rs, int64_t cs, const int32_t *pairs, void *ws,
             size_t ws_bytes, cudaStream_t st) {
  constexpr int NA = CPLX ? 8 : 4;
  if (m < 2 || (m & 1) || !G || !pairs || !ws || !aligned(ws, 256)) return SVD2_EINVAL;
  // column-major (rs = 1, cs >= m) or row-major (cs = 1, rs >= m)
  const bool rows_fast = rs == 1 && cs >= m;
  if (!rows_fast && !(cs == 1 && rs >= m)) return SVD2_EINVAL;
  if (ws_bytes < kog_ws_bytes<T, CPLX>(m)) return SVD2_EINVAL;
  KogArgs<T, CPLX> p{};
  p.g = G;
  p.rs = rs;
  p.cs = cs;
  p.pairs = pairs;
  p.m = m;
  p.npairs = m / 2;
  auto *base = static_cast<unsigned char *>(ws);
  p.skipped = reinterpret_cast<unsigned long long *>(base);
  const size_t arr = round256((size_t)p.npairs * sizeof(T));
  size_t off = kKogHeader;
  for (int e = 0; e < NA; ++e, off += arr) p.u[e] = reinterpret_cast<T *>(base + off);
  for (int e = 0; e < NA; ++e, off += arr) p.v[e] = reinterpret_cast<T *>(base + off);
  p.smax = reinterpret_cast<T *>(base + off);
  p.smin = reinterpret_cast<T *>(base + off + arr);
  SVD2_CUDA_TRY(cudaMemsetAsync(p.skipped, 0, sizeof(unsigned long long), st));
  const int64_t pb = (p.npairs + 255) / 256;
  kog_pivot_kernel<T, CPLX><<<(unsigned)(pb < 65535 ? pb : 65535), 256, 0, st>>>(p);
  SVD2_CUDA_TRY(cudaGetLastError());
  // each thread takes up to 8 blocks of its line (amortises its own factor)
  const int64_t gy = (p.npairs + 7) / 8;
  constexpr int ub = KogShape<T, CPLX>::block;
  const dim3 grid((unsigned)((p.npairs + ub - 1) / ub), (unsigned)(gy < 65535 ? gy : 65535));
  if (rows_fast)
    kog_update_kernel<T, CPLX, true><<<grid, ub, 0, st>>>(p);
  else
    kog_update_kernel<T, CPLX, false><<<grid, ub, 0, st>>>(p);
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}

}  // namespace svd2

using namespace svd2;

extern "C" size_t svd2_kog_workspace_bytes(int op, int64_t m) {
  if (m < 2) m = 2;
  switch (op) {
    case kOpD: return kog_ws_bytes<double, false>(m);
    case kOpZ: return kog_ws_bytes<double, true>(m);
    case kOpS: return kog_ws_bytes<float, false>(m);
    case kOpC: return kog_ws_bytes<float, true>(m);
    default: return 0;
  }
}

extern "C" int svd2_kog_step_d(int64_t m, double *G, int64_t rs, int64_t cs, const int32_t *pairs,
                               void *workspace, size_t workspace_bytes, svd2_stream_t stream) {
  return kog_step<double, false>(m, G, rs, cs, pairs, workspace, workspace_bytes,
                                 (cudaStream_t)stream);
}
extern "C" int svd2_kog_step_z(int64_t m, double *G, int64_t rs, int64_t cs, const int32_t *pairs,
                               void *workspace, size_t workspace_bytes, svd2_stream_t stream) {
  return kog_step<double, true>(m, G, rs, cs, pairs, workspace, workspace_bytes,
                                (cudaStream_t)stream);
}
extern "C" int svd2_kog_step_s(int64_t m, float *G, int64_t rs, int64_t cs, const int32_t *pairs,
                               void *workspace, size_t workspace_bytes, svd2_stream_t stream) {
  return kog_step<float, false>(m, G, rs, cs, pairs, workspace, workspace_bytes,
                                (cudaStream_t)stream);
}
extern "C" int svd2_kog_step_c(int64_t m, float *G, int64_t rs, int64_t cs, const int32_t *pairs,
                               void *workspace, size_t workspace_bytes, svd2_stream_t stream) {
  return kog_step<float, true>(m, G, rs, cs, pairs, workspace, workspace_bytes,
                               (cudaStream_t)stream);
}

extern "C" int svd2_kog_skipped(const void *workspace, int64_t *count) {
  if (!workspace || !count) return SVD2_EINVAL;
  unsigned long long c = 0;
  SVD2_CUDA_TRY(cudaMemcpy(&c, workspace, sizeof(c), cudaMemcpyDeviceToHost));
  *count = (int64_t)c;
  return SVD2_OK;
}
