// Backward (adjoint) of the real batched 2x2 SVD: svd2_bwd_d / svd2_bwd_s.
//
// For A = U diag(s1, s2) V^T (s1 >= s2 >= 0, U and V orthogonal) and a loss
// with gradients gU, gV (element order u11, u21, u12, u22) and g1, g2, the
// gradient with respect to A is, with J = U^T gU, K = V^T gV, a = J12 - J21,
// b = K12 - K21:
//   gA = U M V^T,  M = [[g1, p - q], [-p - q, g2]],
//   p = (a - b) / (2 (s1 + s2)),  q = (a + b) / (2 (s1 - s2)).
// (The standard square-SVD adjoint: dP = U^T dA V has diagonal d(s) and
// off-diagonal Omega_U Sigma + Sigma Omega_V^T with antisymmetric Omega's, which
// for order two solve in closed form.)  The paper defines no backward; this is
// the differentiation form built on its forward.
//
// Near-equal singular values: 1/(s1 - s2) is replaced, with the relative gap
// g = (s1 - s2)/s1, by g / (s1 (g^2 + rel_delta^2)) -- equal to 1/(s1 - s2)
// for g >> rel_delta and going to 0 as g -> 0 -- so the rotation part of the
// gradient stays bounded when the singular vectors are ill-determined.
// s1 + s2 = 0 (A = 0) zeroes both rotation terms.  NULL upstream gradients
// count as zero.  Every operation is a correctly rounded IEEE operation in the
// order written, as in the oracle's adjoint.
#include "svd2_common.cuh"
#include "svd2_math.cuh"

namespace svd2 {

template <typename T>
struct BwdArgs {
  const T *u[4];
  const T *v[4];
  const T *s1;
  const T *s2;
  const T *gu[4];   // entries may be NULL (zero)
  const T *gv[4];
  const T *g1;
  const T *g2;
  T *ga[4];
  T dl;
  int64_t n;
};

template <typename T>
__device__ __forceinline__ T ld0(const T *p, int64_t k) {
  return p ? __ldcs(p + k) : T(0);
}

// M consecutive elements from k0 (vector loads), or zeros for a NULL array.
template <typename T, int M>
__device__ __forceinline__ void ld0_vec(const T *p, int64_t k0, T (&x)[M]) {
  if (p) {
    load_vec<T, M>(p + k0, x);
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = T(0);
  }
}

// The products of the adjoint, by stage (0: the dot products of J and K, 1: the
// factors of p, q and the gap, 2: W = U M, 3: gA = W V^*): the hardware
// multiplication, or for doubles in the stages of the mask STAGES the same
// correctly rounded product on the integer pipe (sfp::mul_fast: bad is set for
// a subnormal, infinite or NaN operand or a product outside the normal range,
// the result then unspecified), which takes those operations off the FP64 pipe
// (2 per clock per SM).
struct BwdMulHw {
  template <int S, typename T> __device__ __forceinline__ T at(T a, T b) const {
    return fp<T>::mul(a, b);
  }
};
template <unsigned STAGES> struct BwdMulMix {
  unsigned &bad;
  template <int S> __device__ __forceinline__ double at(double a, double b) const {
    if constexpr (((STAGES >> S) & 1u) != 0) return sfp::mul_fast(a, b, bad);
    else return fp<double>::mul(a, b);
  }
};

// The stages whose products run on the integer pipe in the FP64 kernels: those
// of p, q and the gap and of gA (real: 10 of 18 products; complex: 20 of 40),
// the split that balances the two pipes best at n = 2^22 -- adjoint 0.246 ms
// real, 0.903 ms complex, against 0.330 and 1.071 with every product on the
// FP64 pipe and 0.309 and 0.990 with every product on the integer pipe (the
// integer pipe then binds).
constexpr unsigned kBwdIntStagesReal = 0xau;
constexpr unsigned kBwdIntStagesCplx = 0xau;

template <int S, typename Mul, typename T>
__device__ __forceinline__ T mul_at(const Mul &mul, T a, T b) {
  return mul.template at<S>(a, b);
}

// x > 0 and x == 0, for doubles on the integer pipe (the comparison
// instruction runs on the FP64 pipe); a NaN compares false, as in IEEE.
template <typename T> __device__ __forceinline__ bool gt0(T x) {
  if constexpr (sizeof(T) == 8) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
  } else {
    return x > T(0);
  }
}
template <typename T> __device__ __forceinline__ bool eq0(T x) {
  if constexpr (sizeof(T) == 8)
    return ((unsigned long long)__double_as_longlong(x) << 1) == 0;
  else
    return x == T(0);
}

// The adjoint of one matrix: U, V, s1, s2 and the upstream gradients in,
// gA out (element order 11, 21, 12, 22).
template <typename T, typename Mul>
__device__ __forceinline__ void bwd_one(const T (&u)[4], const T (&v)[4], T s1, T s2,
                                        const T (&gu)[4], const T (&gv)[4], T m11, T m22, T dl,
                                        T (&ga)[4], const Mul &mul) {
  using F = fp<T>;
  const T u11 = u[0], u21 = u[1], u12 = u[2], u22 = u[3];
  const T v11 = v[0], v21 = v[1], v12 = v[2], v22 = v[3];
  // J12 = (U^T gU)_12, J21 = (U^T gU)_21, likewise K for V
  // (every two-term dot product as fma(x0, y0, x1 y1))
  const T J12 = F::fma(u11, gu[2], mul_at<0>(mul, u21, gu[3]));
  const T J21 = F::fma(u12, gu[0], mul_at<0>(mul, u22, gu[1]));
  const T K12 = F::fma(v11, gv[2], mul_at<0>(mul, v21, gv[3]));
  const T K21 = F::fma(v12, gv[0], mul_at<0>(mul, v22, gv[1]));
  const T a = F::sub(J12, J21), b = F::sub(K12, K21);
  const T sum = F::add(s1, s2);
  const T inv_sum = gt0(sum) ? F::div(T(1), sum) : T(0);
  T inv_gap = T(0);
  if (gt0(s1)) {
    const T g = F::div(F::sub(s1, s2), s1);
    // g = 0: the safeguard's value there (0), also for rel_delta = 0 (0/0)
    inv_gap = eq0(g) ? T(0) : F::div(g, mul_at<1>(mul, s1, F::fma(g, g, mul_at<1>(mul, dl, dl))));
  }
  const T pp = mul_at<1>(mul, mul_at<1>(mul, T(0.5), F::sub(a, b)), inv_sum);
  const T qq = mul_at<1>(mul, mul_at<1>(mul, T(0.5), F::add(a, b)), inv_gap);
  const T m12 = F::sub(pp, qq), m21 = F::sub(b_neg(pp), qq);
  // W = U M, gA = W V^T
  const T w11 = F::fma(u11, m11, mul_at<2>(mul, u12, m21));
  const T w12 = F::fma(u11, m12, mul_at<2>(mul, u12, m22));
  const T w21 = F::fma(u21, m11, mul_at<2>(mul, u22, m21));
  const T w22 = F::fma(u21, m12, mul_at<2>(mul, u22, m22));
  ga[0] = F::fma(w11, v11, mul_at<3>(mul, w12, v12));
  ga[1] = F::fma(w21, v11, mul_at<3>(mul, w22, v12));
  ga[2] = F::fma(w11, v21, mul_at<3>(mul, w12, v22));
  ga[3] = F::fma(w21, v21, mul_at<3>(mul, w22, v22));
}

// M matrices per thread per step (grid-stride), every array read and written
// with M-element vector accesses (all arrays aligned to M elements; M = 1:
// scalar accesses at any alignment), then the n mod M tail one per thread.
// Doubles: at least 4 resident blocks (64 registers; the split below needs 60,
// and with every product on the integer pipe the kernel took 96 uncapped,
// halving the resident warps: 0.39 against 0.31 ms at n = 2^22).
template <typename T, int M>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 4 : 0) bwd_kernel(const BwdArgs<T> p) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ngroups = p.n / M;
  for (int64_t g = tid; g < ngroups; g += stride) {
    const int64_t k0 = g * M;
    T u[4][M], v[4][M], gu[4][M], gv[4][M], s1[M], s2[M], m11[M], m22[M], ga[4][M];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      load_vec<T, M>(p.u[e] + k0, u[e]);
      load_vec<T, M>(p.v[e] + k0, v[e]);
    }
    load_vec<T, M>(p.s1 + k0, s1);
    load_vec<T, M>(p.s2 + k0, s2);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ld0_vec<T, M>(p.gu[e], k0, gu[e]);
      ld0_vec<T, M>(p.gv[e], k0, gv[e]);
    }
    ld0_vec<T, M>(p.g1, k0, m11);
    ld0_vec<T, M>(p.g2, k0, m22);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      T ui[4], vi[4], gui[4], gvi[4], gai[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ui[e] = u[e][m];
        vi[e] = v[e][m];
        gui[e] = gu[e][m];
        gvi[e] = gv[e][m];
      }
      if constexpr (sizeof(T) == 8) {
        // the integer-pipe products; a matrix with one outside their domain is
        // read again (plain loads after a compiler barrier: the first values
        // need not stay in registers) and done with the hardware's
        unsigned bad = 0;
        bwd_one<T>(ui, vi, s1[m], s2[m], gui, gvi, m11[m], m22[m], p.dl, gai,
                   BwdMulMix<kBwdIntStagesReal>{bad});
        if (bad) {
          asm volatile("" ::: "memory");
          const int64_t k = k0 + m;
          T u2[4], v2[4], gu2[4], gv2[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            u2[e] = p.u[e][k];
            v2[e] = p.v[e][k];
            gu2[e] = p.gu[e] ? p.gu[e][k] : T(0);
            gv2[e] = p.gv[e] ? p.gv[e][k] : T(0);
          }
          bwd_one<T>(u2, v2, p.s1[k], p.s2[k], gu2, gv2, p.g1 ? p.g1[k] : T(0),
                     p.g2 ? p.g2[k] : T(0), p.dl, gai, BwdMulHw{});
        }
      } else {
        bwd_one<T>(ui, vi, s1[m], s2[m], gui, gvi, m11[m], m22[m], p.dl, gai, BwdMulHw{});
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) ga[e][m] = gai[e];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) store_vec<T, M>(p.ga[e] + k0, ga[e]);
  }
  if constexpr (M > 1) {
    const int64_t k = ngroups * M + tid;
    if (k < p.n) {
      T ui[4], vi[4], gui[4], gvi[4], gai[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ui[e] = __ldcs(p.u[e] + k);
        vi[e] = __ldcs(p.v[e] + k);
        gui[e] = ld0(p.gu[e], k);
        gvi[e] = ld0(p.gv[e], k);
      }
      bwd_one<T>(ui, vi, __ldcs(p.s1 + k), __ldcs(p.s2 + k), gui, gvi, ld0(p.g1, k),
                 ld0(p.g2, k), p.dl, gai, BwdMulHw{});
#pragma unroll
      for (int e = 0; e < 4; ++e) __stcs(p.ga[e] + k, gai[e]);
    }
  }
}

// Complex adjoint (svd2_bwd_z / svd2_bwd_c): with J = U^* gU, K = V^* gV,
// a = J12 - conj(J21), b = K12 - conj(K21), p and q as in the real case,
//   gA = U M V^*,  M = [[g1 + i t1, p - q], [-conj(p) - conj(q), g2 + i t2]],
//   t_i = (Im J_ii - Im K_ii) / (2 s_i) (0 for s_i = 0),
// gradients as dL/dRe + i dL/dIm.  The t_i carry the phase gauge
// U, V -> U D, V D: for a loss invariant under it, Im J_ii + Im K_ii = 0.
// Same order of correctly rounded operations as the oracle's complex adjoint.
template <typename T>
struct BwdArgsC {
  const T *u[8];
  const T *v[8];
  const T *s1;
  const T *s2;
  const T *gu[8];
  const T *gv[8];
  const T *g1;
  const T *g2;
  T *ga[8];
  T dl;
  int64_t n;
};

// sum_a conj(x_a) y_a over the two elements (a0, a1) of x and (b0, b1) of y,
// each four-term sum as the fma chain x0 y0 + (x1 y1 + (x2 y2 + x3 y3)):
// real part xr0 yr0 + xi0 yi0 + xr1 yr1 + xi1 yi1, imaginary part
// xr0 yi0 - xi0 yr0 + xr1 yi1 - xi1 yr1.
template <typename T, typename Mul>
__device__ __forceinline__ T cdot_re(T xr0, T xi0, T yr0, T yi0, T xr1, T xi1, T yr1, T yi1,
                                     const Mul &mul) {
  using F = fp<T>;
  return F::fma(xr0, yr0, F::fma(xi0, yi0, F::fma(xr1, yr1, mul_at<0>(mul, xi1, yi1))));
}
template <typename T, typename Mul>
__device__ __forceinline__ T cdot_im(T xr0, T xi0, T yr0, T yi0, T xr1, T xi1, T yr1, T yi1,
                                     const Mul &mul) {
  using F = fp<T>;
  return F::fma(xr0, yi0,
                F::fma(b_neg(xi0), yr0, F::fma(xr1, yi1, b_neg(mul_at<0>(mul, xi1, yr1)))));
}

// The complex adjoint of matrix k: its inputs read, gA into ga (record order
// Re 11, Im 11, Re 21, ...).
template <typename T, bool STREAM, typename Mul>
__device__ __forceinline__ void bwd_cplx_one(const BwdArgsC<T> &p, int64_t k, T (&ga)[8],
                                             const Mul &mul) {
  using F = fp<T>;
  // streaming loads, or plain ones (a second read after a compiler barrier)
  auto ld = [&](const T *a) { return STREAM ? __ldcs(a + k) : a[k]; };
  auto ldz = [&](const T *a) { return a ? ld(a) : T(0); };
  T ur[4], ui[4], vr[4], vi[4], gur[4], gui[4], gvr[4], gvi[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ur[e] = ld(p.u[2 * e]);
    ui[e] = ld(p.u[2 * e + 1]);
    vr[e] = ld(p.v[2 * e]);
    vi[e] = ld(p.v[2 * e + 1]);
    gur[e] = ldz(p.gu[2 * e]);
    gui[e] = ldz(p.gu[2 * e + 1]);
    gvr[e] = ldz(p.gv[2 * e]);
    gvi[e] = ldz(p.gv[2 * e + 1]);
  }
  const T s1 = ld(p.s1), s2 = ld(p.s2);
  // J_xy = sum_a conj(u_ax) gu_ay, element (a, x) at a + 2x
  const T Jr12 = cdot_re(ur[0], ui[0], gur[2], gui[2], ur[1], ui[1], gur[3], gui[3], mul);
  const T Ji12 = cdot_im(ur[0], ui[0], gur[2], gui[2], ur[1], ui[1], gur[3], gui[3], mul);
  const T Jr21 = cdot_re(ur[2], ui[2], gur[0], gui[0], ur[3], ui[3], gur[1], gui[1], mul);
  const T Ji21 = cdot_im(ur[2], ui[2], gur[0], gui[0], ur[3], ui[3], gur[1], gui[1], mul);
  const T Ji11 = cdot_im(ur[0], ui[0], gur[0], gui[0], ur[1], ui[1], gur[1], gui[1], mul);
  const T Ji22 = cdot_im(ur[2], ui[2], gur[2], gui[2], ur[3], ui[3], gur[3], gui[3], mul);
  const T Kr12 = cdot_re(vr[0], vi[0], gvr[2], gvi[2], vr[1], vi[1], gvr[3], gvi[3], mul);
  const T Ki12 = cdot_im(vr[0], vi[0], gvr[2], gvi[2], vr[1], vi[1], gvr[3], gvi[3], mul);
  const T Kr21 = cdot_re(vr[2], vi[2], gvr[0], gvi[0], vr[3], vi[3], gvr[1], gvi[1], mul);
  const T Ki21 = cdot_im(vr[2], vi[2], gvr[0], gvi[0], vr[3], vi[3], gvr[1], gvi[1], mul);
  const T Ki11 = cdot_im(vr[0], vi[0], gvr[0], gvi[0], vr[1], vi[1], gvr[1], gvi[1], mul);
  const T Ki22 = cdot_im(vr[2], vi[2], gvr[2], gvi[2], vr[3], vi[3], gvr[3], gvi[3], mul);
  const T ar = F::sub(Jr12, Jr21), ai = F::add(Ji12, Ji21);
  const T br = F::sub(Kr12, Kr21), bi = F::add(Ki12, Ki21);
  const T sum = F::add(s1, s2);
  const T inv_sum = gt0(sum) ? F::div(T(1), sum) : T(0);
  T inv_gap = T(0);
  if (gt0(s1)) {
    const T g = F::div(F::sub(s1, s2), s1);
    // g = 0: the safeguard's value there (0), also for rel_delta = 0 (0/0)
    inv_gap = eq0(g) ? T(0)
                     : F::div(g, mul_at<1>(mul, s1, F::fma(g, g, mul_at<1>(mul, p.dl, p.dl))));
  }
  const T pr = mul_at<1>(mul, mul_at<1>(mul, T(0.5), F::sub(ar, br)), inv_sum);
  const T pi = mul_at<1>(mul, mul_at<1>(mul, T(0.5), F::sub(ai, bi)), inv_sum);
  const T qr = mul_at<1>(mul, mul_at<1>(mul, T(0.5), F::add(ar, br)), inv_gap);
  const T qi = mul_at<1>(mul, mul_at<1>(mul, T(0.5), F::add(ai, bi)), inv_gap);
  const T t1 = gt0(s1) ? F::div(mul_at<1>(mul, T(0.5), F::sub(Ji11, Ki11)), s1) : T(0);
  const T t2 = gt0(s2) ? F::div(mul_at<1>(mul, T(0.5), F::sub(Ji22, Ki22)), s2) : T(0);
  // M in the record order m11, m21, m12, m22
  const T mr[4] = {ldz(p.g1), F::sub(b_neg(pr), qr), F::sub(pr, qr), ldz(p.g2)};
  const T mi[4] = {t1, F::add(pi, qi), F::sub(pi, qi), t2};
  // W = U M
  T wr[4], wi[4];
#pragma unroll
  for (int x = 0; x < 2; ++x) {
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int o = x + 2 * y, u1 = x, u2 = x + 2, m1 = 2 * y, m2 = 2 * y + 1;
      wr[o] = F::fma(ur[u1], mr[m1], F::fma(b_neg(ui[u1]), mi[m1],
                     F::fma(ur[u2], mr[m2], b_neg(mul_at<2>(mul, ui[u2], mi[m2])))));
      wi[o] = F::fma(ur[u1], mi[m1], F::fma(ui[u1], mr[m1],
                     F::fma(ur[u2], mi[m2], mul_at<2>(mul, ui[u2], mr[m2]))));
    }
  }
  // gA = W V^*
#pragma unroll
  for (int x = 0; x < 2; ++x) {
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int o = x + 2 * y, w1 = x, w2 = x + 2, v1 = y, v2 = y + 2;
      ga[2 * o] = F::fma(wr[w1], vr[v1], F::fma(wi[w1], vi[v1],
                         F::fma(wr[w2], vr[v2], mul_at<3>(mul, wi[w2], vi[v2]))));
      ga[2 * o + 1] = F::fma(wi[w1], vr[v1], F::fma(b_neg(wr[w1]), vi[v1],
                             F::fma(wi[w2], vr[v2], b_neg(mul_at<3>(mul, wr[w2], vi[v2])))));
    }
  }
}

// Doubles: at least 3 resident blocks (80 registers with some spilling; with
// every product on the integer pipe, 0.99 ms at n = 2^22 against 1.01 uncapped
// at 118 registers and 1.03 in blocks of 128 at 96).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 3 : 0)
    bwd_cplx_kernel(const BwdArgsC<T> p) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < p.n; k += stride) {
    T ga[8];
    if constexpr (sizeof(T) == 8) {
      // the integer-pipe products; a matrix with one outside their domain is
      // read again and done with the hardware's (nothing is stored before)
      unsigned bad = 0;
      bwd_cplx_one<T, true>(p, k, ga, BwdMulMix<kBwdIntStagesCplx>{bad});
      if (bad) {
        asm volatile("" ::: "memory");
        bwd_cplx_one<T, false>(p, k, ga, BwdMulHw{});
      }
    } else {
      bwd_cplx_one<T, true>(p, k, ga, BwdMulHw{});
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) __stcs(p.ga[e] + k, ga[e]);
  }
}

template <typename T>
static int launch_bwd_cplx(int64_t n, const T *const *U, const T *const *V, const T *s1,
                           const T *s2, const T *const *gU, const T *const *gV, const T *g1,
                           const T *g2, T *const *gA, T rel_delta, cudaStream_t stream) {
  if (n < 0 || !(rel_delta >= T(0))) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!U || !V || !gA || !s1 || !s2) return SVD2_EINVAL;
  BwdArgsC<T> p{};
  for (int e = 0; e < 8; ++e) {
    if (!U[e] || !V[e] || !gA[e]) return SVD2_EINVAL;
    p.u[e] = U[e];
    p.v[e] = V[e];
    p.gu[e] = gU ? gU[e] : nullptr;
    p.gv[e] = gV ? gV[e] : nullptr;
    p.ga[e] = gA[e];
  }
  p.s1 = s1;
  p.s2 = s2;
  p.g1 = g1;
  p.g2 = g2;
  p.dl = rel_delta;
  p.n = n;
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  bwd_cplx_kernel<T><<<(unsigned)(want < cap ? want : cap), 256, 0, stream>>>(p);
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}

template <typename T>
static int launch_bwd(int64_t n, const T *const *U, const T *const *V, const T *s1, const T *s2,
                      const T *const *gU, const T *const *gV, const T *g1, const T *g2,
                      T *const *gA, T rel_delta, cudaStream_t stream) {
  if (n < 0 || !(rel_delta >= T(0))) return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  if (!U || !V || !gA || !s1 || !s2) return SVD2_EINVAL;
  BwdArgs<T> p{};
  for (int e = 0; e < 4; ++e) {
    if (!U[e] || !V[e] || !gA[e]) return SVD2_EINVAL;
    p.u[e] = U[e];
    p.v[e] = V[e];
    p.gu[e] = gU ? gU[e] : nullptr;
    p.gv[e] = gV ? gV[e] : nullptr;
    p.ga[e] = gA[e];
  }
  p.s1 = s1;
  p.s2 = s2;
  p.g1 = g1;
  p.g2 = g2;
  p.dl = rel_delta;
  p.n = n;
  // FP32: two matrices per thread (8-byte vector accesses) when every array
  // allows it -- the FP32 adjoint is bound by memory latency; the FP64 one, bound
  // by latency once its products run on the integer pipe, keeps one matrix per
  // thread (64 registers)
  const size_t va = 2 * sizeof(T);
  bool vec = sizeof(T) == 4 && aligned(s1, va) && aligned(s2, va) && (!g1 || aligned(g1, va)) &&
             (!g2 || aligned(g2, va));
  for (int e = 0; e < 4; ++e)
    vec = vec && aligned(U[e], va) && aligned(V[e], va) && aligned(gA[e], va) &&
          (!p.gu[e] || aligned(p.gu[e], va)) && (!p.gv[e] || aligned(p.gv[e], va));
  const int M = vec ? 2 : 1;
  const int64_t units = (n / M > n % M) ? n / M : n % M;   // threads needed
  const int64_t want = (units + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  const unsigned grid = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  if constexpr (sizeof(T) == 4) {
    if (vec)
      bwd_kernel<T, 2><<<grid, 256, 0, stream>>>(p);
    else
      bwd_kernel<T, 1><<<grid, 256, 0, stream>>>(p);
  } else {
    bwd_kernel<T, 1><<<grid, 256, 0, stream>>>(p);
  }
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}

}  // namespace svd2

using namespace svd2;

extern "C" int svd2_bwd_d(int64_t n, const double *const U[4], const double *const V[4],
                          const double *s1, const double *s2, const double *const gU[4],
                          const double *const gV[4], const double *g1, const double *g2,
                          double *const gA[4], double rel_delta, svd2_stream_t stream) {
  return launch_bwd<double>(n, U, V, s1, s2, gU, gV, g1, g2, gA, rel_delta, (cudaStream_t)stream);
}

extern "C" int svd2_bwd_s(int64_t n, const float *const U[4], const float *const V[4],
                          const float *s1, const float *s2, const float *const gU[4],
                          const float *const gV[4], const float *g1, const float *g2,
                          float *const gA[4], float rel_delta, svd2_stream_t stream) {
  return launch_bwd<float>(n, U, V, s1, s2, gU, gV, g1, g2, gA, rel_delta, (cudaStream_t)stream);
}

extern "C" int svd2_bwd_z(int64_t n, const double *const U[8], const double *const V[8],
                          const double *s1, const double *s2, const double *const gU[8],
                          const double *const gV[8], const double *g1, const double *g2,
                          double *const gA[8], double rel_delta, svd2_stream_t stream) {
  return launch_bwd_cplx<double>(n, U, V, s1, s2, gU, gV, g1, g2, gA, rel_delta,
                                 (cudaStream_t)stream);
}

extern "C" int svd2_bwd_c(int64_t n, const float *const U[8], const float *const V[8],
                          const float *s1, const float *s2, const float *const gU[8],
                          const float *const gV[8], const float *g1, const float *g2,
                          float *const gA[8], float rel_delta, svd2_stream_t stream) {
  return launch_bwd_cplx<float>(n, U, V, s1, s2, gU, gV, g1, g2, gA, rel_delta,
                                (cudaStream_t)stream);
}
