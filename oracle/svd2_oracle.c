/*
 * CPU oracle for the batched 2x2 SVD of V. Novakovic, arXiv 2005.07403.
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, obviously-correct scalar C used by the
 * tests, by the smoke check and by the bench's CPU-baseline leg to check and to
 * time the CUDA library.  It shares no code, header, table or constant with the
 * CUDA path and neither side includes the other.  Build (see oracle/__init__.py):
 *     gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -fPIC -shared
 * -ffp-contract=off is required: every fused multiply-add of the paper is
 * written as an explicit fma call and no other product may be fused.
 *
 * Two tiers:
 *  O1 (step oracle): the paper's algorithm, Sec. 2 - Sec. 7 and Eq. 29, one
 *     matrix at a time, in double, float and binary128 (the latter gives a
 *     reference decomposition accurate to ~1e-33 for the gradient checks);
 *  O2 (truth tier): closed forms of the singular values and the error metrics
 *     of Sec. 8 (Eq. 32 - Eq. 35), evaluated in binary128.
 *
 * Parity status (what pins each function; details in the tests):
 *  - scale exponent s (Eq. 2): pinned by hand-computed exponents of golden
 *    cases and by the bound -2 <= s;
 *  - singular values: pinned to the binary128 closed form and to brute force
 *    (mpmath) on all small integer matrices;
 *  - U and V: pinned by the backward error and the orthogonality of Sec. 8,
 *    by closed forms (diagonal and rotated diagonal matrices) and by the
 *    structure Eq. 29 fixes (real non-negative cos(psi) first row of V before
 *    P_c, etc.);
 *  - the adjoint: pinned by central finite differences of O1 itself;
 *  - the element-by-element rounding sequence of U and V (which of the
 *    equally valid minimal-rounding orders of Eq. 29 is used) has no pin
 *    beyond those properties: parity unpinned for that choice.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- binary128: __float128 on x86-64 (libquadmath), long double on AArch64. */
#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 quad;
#define Q_FMA fmaq
#define Q_SQRT sqrtq
#define Q_FABS fabsq
#define Q_COPYSIGN copysignq
#define Q_LOGB logbq
#define Q_SCALBN scalbnq
#define Q_MAX FLT128_MAX
#define Q_TRUE_MIN FLT128_DENORM_MIN
#define Q_MAX_EXP FLT128_MAX_EXP
#elif defined(__aarch64__)
typedef long double quad;
_Static_assert(LDBL_MANT_DIG == 113, "AArch64 long double must be binary128");
#define Q_FMA fmal
#define Q_SQRT sqrtl
#define Q_FABS fabsl
#define Q_COPYSIGN copysignl
#define Q_LOGB logbl
#define Q_SCALBN scalbnl
#define Q_MAX LDBL_MAX
#define Q_TRUE_MIN LDBL_TRUE_MIN
#define Q_MAX_EXP LDBL_MAX_EXP
#else
#error "binary128 support needed"
#endif

#define ZERO_S INT32_MAX   /* int32 stand-in for the s = DBL_MAX of the zero matrix (Eq. 2) */

/* ------------------------------------------------------------- double ---- */
#define T double
#define SFX(name) name##_d
#define T_MAX DBL_MAX
#define T_TRUE_MIN DBL_TRUE_MIN
#define T_MAX_EXP DBL_MAX_EXP
/* Fig. 10 prints sqrt(DBL_MAX) as 1.34078079299425956E+154; the tests check that
 * this literal and sqrt(DBL_MAX) are the same double. */
#define T_SQRT_MAX 1.34078079299425956E+154
#define T_FMA fma
#define T_SQRT sqrt
#define T_FABS fabs
#define T_COPYSIGN copysign
#define T_LOGB logb
#define T_SCALBN scalbn
#include "svd2_oracle_body.h"
#undef T
#undef SFX
#undef T_MAX
#undef T_TRUE_MIN
#undef T_MAX_EXP
#undef T_SQRT_MAX
#undef T_FMA
#undef T_SQRT
#undef T_FABS
#undef T_COPYSIGN
#undef T_LOGB
#undef T_SCALBN

/* -------------------------------------------------------------- float ---- */
/* Single precision as remarked in Sec. 1 and Sec. 7: FLT_* constants and
 * sqrt(FLT_MAX) as the bound of Eq. 14. */
#define T float
#define SFX(name) name##_s
#define T_MAX FLT_MAX
#define T_TRUE_MIN FLT_TRUE_MIN
#define T_MAX_EXP FLT_MAX_EXP
#define T_SQRT_MAX sqrtf(FLT_MAX)
#define T_FMA fmaf
#define T_SQRT sqrtf
#define T_FABS fabsf
#define T_COPYSIGN copysignf
#define T_LOGB logbf
#define T_SCALBN scalbnf
#define T_WIDE double
#define T_WIDE_FMA fma
#include "svd2_oracle_body.h"
#undef T_WIDE
#undef T_WIDE_FMA
#undef T
#undef SFX
#undef T_MAX
#undef T_TRUE_MIN
#undef T_MAX_EXP
#undef T_SQRT_MAX
#undef T_FMA
#undef T_SQRT
#undef T_FABS
#undef T_COPYSIGN
#undef T_LOGB
#undef T_SCALBN

/* ---------------------------------------------------------- binary128 ---- */
#define T quad
#define SFX(name) name##_q
#define T_MAX Q_MAX
#define T_TRUE_MIN Q_TRUE_MIN
#define T_MAX_EXP Q_MAX_EXP
#define T_SQRT_MAX Q_SQRT(Q_MAX)
#define T_FMA Q_FMA
#define T_SQRT Q_SQRT
#define T_FABS Q_FABS
#define T_COPYSIGN Q_COPYSIGN
#define T_LOGB Q_LOGB
#define T_SCALBN Q_SCALBN
#include "svd2_oracle_body.h"

/* ------------------------------------------------------------ helpers ---- */

static int32_t s_to_i32_d(double s) { return s == DBL_MAX ? ZERO_S : (int32_t)s; }
static int32_t s_to_i32_s(float s) { return s == FLT_MAX ? ZERO_S : (int32_t)s; }

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int svd2o_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Fig. 1: optional backscaling Sigma = 2^-s Sigma', after which s reads 0. */
#define SVD2O_BACKSCALE 1u
/* U assembled by Eq. 31 (sines and cosines) instead of Eq. 29 (tangents). */
#define SVD2O_SINE 2u

/* ----------------------------------------------- O1 batch entry points ---- */
/*
 * Split layout of Sec. 3: one array per matrix element, in the order of the
 * records of Sec. 8: A[0..3] = a11, a21, a12, a22 (real), and for complex
 * A[0..7] = Re a11, Im a11, Re a21, Im a21, Re a12, Im a12, Re a22, Im a22.
 * U and V use the same element order.  piv may be NULL.  The loop over the
 * matrices is the OpenMP parallel for of Fig. 2.
 */
void svd2o_batch_d(int64_t n, const double *const A[4], double *const U[4],
                   double *const V[4], double *smax, double *smin, int32_t *s,
                   uint8_t *piv, uint32_t flags, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double a[2][2] = { { A[0][k], A[2][k] }, { A[1][k], A[3][k] } };
        double u[2][2], v[2][2], sx, sn, sc;
        int p;
        int w;
        svd2_real_t_d(a, u, v, &sx, &sn, &sc, &p, 0.0, &w, (flags & SVD2O_SINE) != 0);
        U[0][k] = u[0][0]; U[1][k] = u[1][0]; U[2][k] = u[0][1]; U[3][k] = u[1][1];
        V[0][k] = v[0][0]; V[1][k] = v[1][0]; V[2][k] = v[0][1]; V[3][k] = v[1][1];
        int32_t si = s_to_i32_d(sc);
        if ((flags & SVD2O_BACKSCALE) && si != ZERO_S) {
            sx = scalbn(sx, -si);
            sn = scalbn(sn, -si);
        }
        if (flags & SVD2O_BACKSCALE)
            si = 0;
        smax[k] = sx; smin[k] = sn; s[k] = si;
        if (piv) piv[k] = (uint8_t)p;
    }
}

void svd2o_batch_s(int64_t n, const float *const A[4], float *const U[4],
                   float *const V[4], float *smax, float *smin, int32_t *s,
                   uint8_t *piv, uint32_t flags, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        float a[2][2] = { { A[0][k], A[2][k] }, { A[1][k], A[3][k] } };
        float u[2][2], v[2][2], sx, sn, sc;
        int p;
        int w;
        svd2_real_t_s(a, u, v, &sx, &sn, &sc, &p, 0.0f, &w, (flags & SVD2O_SINE) != 0);
        U[0][k] = u[0][0]; U[1][k] = u[1][0]; U[2][k] = u[0][1]; U[3][k] = u[1][1];
        V[0][k] = v[0][0]; V[1][k] = v[1][0]; V[2][k] = v[0][1]; V[3][k] = v[1][1];
        int32_t si = s_to_i32_s(sc);
        if ((flags & SVD2O_BACKSCALE) && si != ZERO_S) {
            sx = scalbnf(sx, -si);
            sn = scalbnf(sn, -si);
        }
        if (flags & SVD2O_BACKSCALE)
            si = 0;
        smax[k] = sx; smin[k] = sn; s[k] = si;
        if (piv) piv[k] = (uint8_t)p;
    }
}

void svd2o_batch_z(int64_t n, const double *const A[8], double *const U[8],
                   double *const V[8], double *smax, double *smin, int32_t *s,
                   uint8_t *piv, uint32_t flags, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double ar[2][2] = { { A[0][k], A[4][k] }, { A[2][k], A[6][k] } };
        double ai[2][2] = { { A[1][k], A[5][k] }, { A[3][k], A[7][k] } };
        double ur[2][2], ui[2][2], vr[2][2], vi[2][2], sx, sn, sc;
        int p;
        svd2_cplx_t_d(ar, ai, ur, ui, vr, vi, &sx, &sn, &sc, &p, (flags & SVD2O_SINE) != 0);
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const int e = 2 * (2 * j + i);   /* element (i,j) -> record slot */
                U[e][k] = ur[i][j]; U[e + 1][k] = ui[i][j];
                V[e][k] = vr[i][j]; V[e + 1][k] = vi[i][j];
            }
        int32_t si = s_to_i32_d(sc);
        if ((flags & SVD2O_BACKSCALE) && si != ZERO_S) {
            sx = scalbn(sx, -si);
            sn = scalbn(sn, -si);
        }
        if (flags & SVD2O_BACKSCALE)
            si = 0;
        smax[k] = sx; smin[k] = sn; s[k] = si;
        if (piv) piv[k] = (uint8_t)p;
    }
}

void svd2o_batch_c(int64_t n, const float *const A[8], float *const U[8],
                   float *const V[8], float *smax, float *smin, int32_t *s,
                   uint8_t *piv, uint32_t flags, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        float ar[2][2] = { { A[0][k], A[4][k] }, { A[2][k], A[6][k] } };
        float ai[2][2] = { { A[1][k], A[5][k] }, { A[3][k], A[7][k] } };
        float ur[2][2], ui[2][2], vr[2][2], vi[2][2], sx, sn, sc;
        int p;
        svd2_cplx_t_s(ar, ai, ur, ui, vr, vi, &sx, &sn, &sc, &p, (flags & SVD2O_SINE) != 0);
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const int e = 2 * (2 * j + i);
                U[e][k] = ur[i][j]; U[e + 1][k] = ui[i][j];
                V[e][k] = vr[i][j]; V[e + 1][k] = vi[i][j];
            }
        int32_t si = s_to_i32_s(sc);
        if ((flags & SVD2O_BACKSCALE) && si != ZERO_S) {
            sx = scalbnf(sx, -si);
            sn = scalbnf(sn, -si);
        }
        if (flags & SVD2O_BACKSCALE)
            si = 0;
        smax[k] = sx; smin[k] = sn; s[k] = si;
        if (piv) piv[k] = (uint8_t)p;
    }
}

/*
 * FP32 form with FP64 re-run (the precision variant of the single-precision
 * remark of Sec. 1 and Sec. 7).  Every matrix is first decomposed in float.  A
 * matrix is flagged when sigma'_min < 2^tau_log2 * sigma'_max, evaluated in
 * float (the product by a power of two is exact).  A flagged matrix is
 * decomposed again by the double method on its exactly upcast elements; its
 * float outputs are then the double results rounded to float, with sigma'
 * brought to the float run's scale: sigma'_32 = RN32(sigma'_64 * 2^(s32 - s64)).
 * flagged[k] (may be NULL) receives 1 for re-run matrices.  With
 * SVD2O_BACKSCALE in flags, Fig. 1 is applied to these final float results
 * (sigma = 2^-s sigma'_32 in float, then s = 0).  Returns the count.
 */
static void backscale_f(float *sx, float *sn, int32_t *s)
{
    if (*s != ZERO_S) {
        *sx = scalbnf(*sx, -*s);
        *sn = scalbnf(*sn, -*s);
    }
    *s = 0;
}

int64_t svd2o_batch_s_rerun(int64_t n, const float *const A[4], float *const U[4],
                            float *const V[4], float *smax, float *smin, int32_t *s,
                            uint8_t *flagged, int tau_log2, uint32_t flags, int nthreads)
{
    set_threads(nthreads);
    int64_t count = 0;
    const float tau = ldexpf(1.0f, tau_log2);
#pragma omp parallel for schedule(static) reduction(+ : count)
    for (int64_t k = 0; k < n; ++k) {
        float a[2][2] = { { A[0][k], A[2][k] }, { A[1][k], A[3][k] } };
        float u[2][2], v[2][2], sx, sn, sc;
        int p;
        svd2_real_s(a, u, v, &sx, &sn, &sc, &p);
        const int32_t s32 = s_to_i32_s(sc);
        const int flag = sn < tau * sx;
        if (flag) {
            double ad[2][2] = { { a[0][0], a[0][1] }, { a[1][0], a[1][1] } };
            double ud[2][2], vd[2][2], sxd, snd, scd;
            int pd;
            svd2_real_d(ad, ud, vd, &sxd, &snd, &scd, &pd);
            const int32_t s64 = s_to_i32_d(scd);
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    u[i][j] = (float)ud[i][j];
                    v[i][j] = (float)vd[i][j];
                }
            sx = (float)scalbn(sxd, s32 - s64);
            sn = (float)scalbn(snd, s32 - s64);
            ++count;
        }
        U[0][k] = u[0][0]; U[1][k] = u[1][0]; U[2][k] = u[0][1]; U[3][k] = u[1][1];
        V[0][k] = v[0][0]; V[1][k] = v[1][0]; V[2][k] = v[0][1]; V[3][k] = v[1][1];
        int32_t so = s32;
        if (flags & SVD2O_BACKSCALE)
            backscale_f(&sx, &sn, &so);
        smax[k] = sx; smin[k] = sn; s[k] = so;
        if (flagged) flagged[k] = (uint8_t)flag;
    }
    return count;
}

/*
 * FP32 form with the FP64 tangent step (the precision variant of the
 * single-precision remark of Sec. 1 and Sec. 7 that keeps double precision
 * only where the method's stability needs it).  Every matrix is decomposed in
 * float; a matrix with |r''_22| < 2^tau_log2 r11 at Eq. 7 has -tan(alpha) and
 * the fma of Eq. 7 evaluated in double (svd2_real_t with T_WIDE = double).  In
 * the real case every value that enters that fma is exact in float, so its
 * double result is the double method's r''_22 / cos(alpha), up to the power of
 * two between the two scales of Eq. 2, whenever both take the same pivots;
 * it is the cancellation of Eq. 7 that costs sigma_min its accuracy in float.
 * wide[k] (may be NULL) receives 1 for the matrices that took the step.
 * Returns their count.
 */
int64_t svd2o_batch_s_tan64(int64_t n, const float *const A[4], float *const U[4],
                            float *const V[4], float *smax, float *smin, int32_t *s,
                            uint8_t *wide, int tau_log2, uint32_t flags, int nthreads)
{
    set_threads(nthreads);
    int64_t count = 0;
    const float tau = ldexpf(1.0f, tau_log2);
#pragma omp parallel for schedule(static) reduction(+ : count)
    for (int64_t k = 0; k < n; ++k) {
        float a[2][2] = { { A[0][k], A[2][k] }, { A[1][k], A[3][k] } };
        float u[2][2], v[2][2], sx, sn, sc;
        int p, w;
        svd2_real_t_s(a, u, v, &sx, &sn, &sc, &p, tau, &w, 0);
        U[0][k] = u[0][0]; U[1][k] = u[1][0]; U[2][k] = u[0][1]; U[3][k] = u[1][1];
        V[0][k] = v[0][0]; V[1][k] = v[1][0]; V[2][k] = v[0][1]; V[3][k] = v[1][1];
        int32_t so = s_to_i32_s(sc);
        if (flags & SVD2O_BACKSCALE)
            backscale_f(&sx, &sn, &so);
        smax[k] = sx; smin[k] = sn; s[k] = so;
        if (wide) wide[k] = (uint8_t)w;
        count += w;
    }
    return count;
}

/* Complex counterpart of svd2o_batch_s_rerun. */
int64_t svd2o_batch_c_rerun(int64_t n, const float *const A[8], float *const U[8],
                            float *const V[8], float *smax, float *smin, int32_t *s,
                            uint8_t *flagged, int tau_log2, uint32_t flags, int nthreads)
{
    set_threads(nthreads);
    int64_t count = 0;
    const float tau = ldexpf(1.0f, tau_log2);
#pragma omp parallel for schedule(static) reduction(+ : count)
    for (int64_t k = 0; k < n; ++k) {
        float ar[2][2] = { { A[0][k], A[4][k] }, { A[2][k], A[6][k] } };
        float ai[2][2] = { { A[1][k], A[5][k] }, { A[3][k], A[7][k] } };
        float ur[2][2], ui[2][2], vr[2][2], vi[2][2], sx, sn, sc;
        int p;
        svd2_cplx_s(ar, ai, ur, ui, vr, vi, &sx, &sn, &sc, &p);
        const int32_t s32 = s_to_i32_s(sc);
        const int flag = sn < tau * sx;
        if (flag) {
            double adr[2][2], adi[2][2], udr[2][2], udi[2][2], vdr[2][2], vdi[2][2];
            double sxd, snd, scd;
            int pd;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    adr[i][j] = ar[i][j];
                    adi[i][j] = ai[i][j];
                }
            svd2_cplx_d(adr, adi, udr, udi, vdr, vdi, &sxd, &snd, &scd, &pd);
            const int32_t s64 = s_to_i32_d(scd);
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    ur[i][j] = (float)udr[i][j]; ui[i][j] = (float)udi[i][j];
                    vr[i][j] = (float)vdr[i][j]; vi[i][j] = (float)vdi[i][j];
                }
            sx = (float)scalbn(sxd, s32 - s64);
            sn = (float)scalbn(snd, s32 - s64);
            ++count;
        }
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const int e = 2 * (2 * j + i);
                U[e][k] = ur[i][j]; U[e + 1][k] = ui[i][j];
                V[e][k] = vr[i][j]; V[e + 1][k] = vi[i][j];
            }
        int32_t so = s32;
        if (flags & SVD2O_BACKSCALE)
            backscale_f(&sx, &sn, &so);
        smax[k] = sx; smin[k] = sn; s[k] = so;
        if (flagged) flagged[k] = (uint8_t)flag;
    }
    return count;
}

/* ------------------------------------------------ O2: binary128 truth ---- */

static void q_split(quad q, double *hi, double *lo)
{
    const double h = (double)q;
    *hi = h;
    *lo = (double)(q - (quad)h);
}

/*
 * Closed-form singular values in binary128.  With F^2 = ||A||_F^2 and
 * d = |det A|: sigma_max = (sqrt(F^2 + 2d) + sqrt(F^2 - 2d)) / 2 and
 * sigma_min = d / sigma_max (sigma_max sigma_min = |det A|,
 * sigma_max^2 + sigma_min^2 = ||A||_F^2).  Products of doubles are exact in
 * binary128 (53 + 53 < 113 bits), so for real A the determinant carries a
 * single rounding.  Results are returned as hi + lo double pairs; when s is
 * not NULL they are first multiplied by 2^s[k] in binary128 (s[k] = ZERO_S:
 * unscaled), so the truth of Sigma' = 2^s Sigma stays representable in double
 * even where Sigma itself is subnormal or above DBL_MAX.
 */
static void truth_from_fd(quad F2, quad d, quad *sx, quad *sn)
{
    quad disc = F2 - 2 * d;
    if (disc < 0)
        disc = 0;
    const quad smax = (Q_SQRT(F2 + 2 * d) + Q_SQRT(disc)) / 2;
    *sx = smax;
    *sn = smax > 0 ? d / smax : 0;
}

static void truth_scale(quad *sx, quad *sn, const int32_t *s, int64_t k)
{
    if (s && s[k] != ZERO_S) {
        *sx = Q_SCALBN(*sx, s[k]);
        *sn = Q_SCALBN(*sn, s[k]);
    }
}

void svd2o_truth_d(int64_t n, const double *const A[4], const int32_t *s,
                   double *smax_hi, double *smax_lo, double *smin_hi, double *smin_lo)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const quad a11 = A[0][k], a21 = A[1][k], a12 = A[2][k], a22 = A[3][k];
        const quad F2 = a11 * a11 + a21 * a21 + a12 * a12 + a22 * a22;
        const quad d = Q_FABS(a11 * a22 - a12 * a21);
        quad sx, sn;
        truth_from_fd(F2, d, &sx, &sn);
        truth_scale(&sx, &sn, s, k);
        q_split(sx, &smax_hi[k], &smax_lo[k]);
        q_split(sn, &smin_hi[k], &smin_lo[k]);
    }
}

void svd2o_truth_z(int64_t n, const double *const A[8], const int32_t *s,
                   double *smax_hi, double *smax_lo, double *smin_hi, double *smin_lo)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const quad r11 = A[0][k], i11 = A[1][k], r21 = A[2][k], i21 = A[3][k];
        const quad r12 = A[4][k], i12 = A[5][k], r22 = A[6][k], i22 = A[7][k];
        const quad F2 = r11 * r11 + i11 * i11 + r21 * r21 + i21 * i21 +
                        r12 * r12 + i12 * i12 + r22 * r22 + i22 * i22;
        /* det = a11 a22 - a12 a21 */
        const quad dr = (r11 * r22 - i11 * i22) - (r12 * r21 - i12 * i21);
        const quad di = (r11 * i22 + i11 * r22) - (r12 * i21 + i12 * r21);
        const quad d = Q_SQRT(dr * dr + di * di);
        quad sx, sn;
        truth_from_fd(F2, d, &sx, &sn);
        truth_scale(&sx, &sn, s, k);
        q_split(sx, &smax_hi[k], &smax_lo[k]);
        q_split(sn, &smin_hi[k], &smin_lo[k]);
    }
}

/*
 * Error metrics of Sec. 8 in binary128, per matrix: kappa (Eq. 32),
 * rho = ||U Sigma V* - A||_F / ||A||_F (Eq. 33, 0 for A = 0),
 * delta = ||U* U - I||_F (Eq. 34), eta = ||V* V - I||_F (Eq. 35).
 * Sigma = 2^-s Sigma' is formed in binary128, where it cannot overflow.
 * Complex inputs use the 8-array record order; real ones pass Ai = Ui = Vi
 * = NULL.
 */
static void metrics_one(const quad ar[2][2], const quad ai[2][2],
                        const quad ur[2][2], const quad ui[2][2],
                        const quad vr[2][2], const quad vi[2][2],
                        quad sx, quad sn, double *rho, double *delta,
                        double *eta, double *kappa)
{
    quad num = 0, den = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            /* (U Sigma V*)_ij = sum_k U_ik sigma_k conj(V_jk) */
            quad er = 0, ei = 0;
            for (int k = 0; k < 2; ++k) {
                const quad sg = k == 0 ? sx : sn;
                const quad pr = ur[i][k] * vr[j][k] + ui[i][k] * vi[j][k];
                const quad pi = ui[i][k] * vr[j][k] - ur[i][k] * vi[j][k];
                er += sg * pr;
                ei += sg * pi;
            }
            er -= ar[i][j];
            ei -= ai[i][j];
            num += er * er + ei * ei;
            den += ar[i][j] * ar[i][j] + ai[i][j] * ai[i][j];
        }
    *rho = den > 0 ? (double)Q_SQRT(num / den) : (double)Q_SQRT(num);
    quad du = 0, dv = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            /* (X* X)_ij = sum_k conj(X_ki) X_kj */
            quad gr = 0, gi = 0, hr = 0, hi = 0;
            for (int k = 0; k < 2; ++k) {
                gr += ur[k][i] * ur[k][j] + ui[k][i] * ui[k][j];
                gi += ur[k][i] * ui[k][j] - ui[k][i] * ur[k][j];
                hr += vr[k][i] * vr[k][j] + vi[k][i] * vi[k][j];
                hi += vr[k][i] * vi[k][j] - vi[k][i] * vr[k][j];
            }
            if (i == j) {
                gr -= 1;
                hr -= 1;
            }
            du += gr * gr + gi * gi;
            dv += hr * hr + hi * hi;
        }
    *delta = (double)Q_SQRT(du);
    *eta = (double)Q_SQRT(dv);
    *kappa = sn > 0 ? (double)(sx / sn) : INFINITY;
}

static quad q_backscale(double sig, int32_t s)
{
    if (s == ZERO_S)
        return (quad)sig;
    return Q_SCALBN((quad)sig, -s);
}

void svd2o_metrics_d(int64_t n, const double *const A[4], const double *const U[4],
                     const double *const V[4], const double *smax, const double *smin,
                     const int32_t *s, double *rho, double *delta, double *eta,
                     double *kappa)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const quad ar[2][2] = { { A[0][k], A[2][k] }, { A[1][k], A[3][k] } };
        const quad ur[2][2] = { { U[0][k], U[2][k] }, { U[1][k], U[3][k] } };
        const quad vr[2][2] = { { V[0][k], V[2][k] }, { V[1][k], V[3][k] } };
        const quad z[2][2] = { { 0, 0 }, { 0, 0 } };
        metrics_one(ar, z, ur, z, vr, z, q_backscale(smax[k], s[k]),
                    q_backscale(smin[k], s[k]), &rho[k], &delta[k], &eta[k], &kappa[k]);
    }
}

void svd2o_metrics_z(int64_t n, const double *const A[8], const double *const U[8],
                     const double *const V[8], const double *smax, const double *smin,
                     const int32_t *s, double *rho, double *delta, double *eta,
                     double *kappa)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        quad ar[2][2], ai[2][2], ur[2][2], ui[2][2], vr[2][2], vi[2][2];
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const int e = 2 * (2 * j + i);
                ar[i][j] = A[e][k]; ai[i][j] = A[e + 1][k];
                ur[i][j] = U[e][k]; ui[i][j] = U[e + 1][k];
                vr[i][j] = V[e][k]; vi[i][j] = V[e + 1][k];
            }
        metrics_one(ar, ai, ur, ui, vr, vi, q_backscale(smax[k], s[k]),
                    q_backscale(smin[k], s[k]), &rho[k], &delta[k], &eta[k], &kappa[k]);
    }
}

/* ------------------------------------------------- adjoint (backward) ---- */
/* Batched adjoint (see adjoint in the body): U, V, gU, gV, gA in the element
 * order of svd2o_batch_d; s1, s2 are the back-scaled singular values. */
void svd2o_bwd_d(int64_t n, const double *const U[4], const double *const V[4],
                 const double *s1, const double *s2, const double *const gU[4],
                 const double *const gV[4], const double *g1, const double *g2,
                 double *const gA[4], double rel_delta)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const double u[4] = { U[0][k], U[1][k], U[2][k], U[3][k] };
        const double v[4] = { V[0][k], V[1][k], V[2][k], V[3][k] };
        const double gu[4] = { gU[0][k], gU[1][k], gU[2][k], gU[3][k] };
        const double gv[4] = { gV[0][k], gV[1][k], gV[2][k], gV[3][k] };
        double ga[4];
        adjoint_d(u, v, s1[k], s2[k], gu, gv, g1[k], g2[k], rel_delta, ga);
        for (int e = 0; e < 4; ++e)
            gA[e][k] = ga[e];
    }
}

void svd2o_bwd_s(int64_t n, const float *const U[4], const float *const V[4],
                 const float *s1, const float *s2, const float *const gU[4],
                 const float *const gV[4], const float *g1, const float *g2,
                 float *const gA[4], float rel_delta)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const float u[4] = { U[0][k], U[1][k], U[2][k], U[3][k] };
        const float v[4] = { V[0][k], V[1][k], V[2][k], V[3][k] };
        const float gu[4] = { gU[0][k], gU[1][k], gU[2][k], gU[3][k] };
        const float gv[4] = { gV[0][k], gV[1][k], gV[2][k], gV[3][k] };
        float ga[4];
        adjoint_s(u, v, s1[k], s2[k], gu, gv, g1[k], g2[k], rel_delta, ga);
        for (int e = 0; e < 4; ++e)
            gA[e][k] = ga[e];
    }
}

/* Complex adjoint over a split-layout batch (8 rows: Re, Im of x11, x21, x12, x22). */
#define SVD2O_BWD_CPLX(SUF, TT)                                                          \
void svd2o_bwd_##SUF(int64_t n, const TT *const U[8], const TT *const V[8],              \
                     const TT *s1, const TT *s2, const TT *const gU[8],                  \
                     const TT *const gV[8], const TT *g1, const TT *g2,                  \
                     TT *const gA[8], TT rel_delta)                                      \
{                                                                                        \
    _Pragma("omp parallel for schedule(static)")                                         \
    for (int64_t k = 0; k < n; ++k) {                                                    \
        TT ur[4], ui[4], vr[4], vi[4], gur[4], gui[4], gvr[4], gvi[4], gar[4], gai[4];   \
        for (int e = 0; e < 4; ++e) {                                                    \
            ur[e] = U[2 * e][k]; ui[e] = U[2 * e + 1][k];                                \
            vr[e] = V[2 * e][k]; vi[e] = V[2 * e + 1][k];                                \
            gur[e] = gU[2 * e][k]; gui[e] = gU[2 * e + 1][k];                            \
            gvr[e] = gV[2 * e][k]; gvi[e] = gV[2 * e + 1][k];                            \
        }                                                                                \
        adjoint_cplx_##SUF##_body(ur, ui, vr, vi, s1[k], s2[k], gur, gui, gvr, gvi,      \
                                  g1[k], g2[k], rel_delta, gar, gai);                    \
        for (int e = 0; e < 4; ++e) {                                                    \
            gA[2 * e][k] = gar[e];                                                       \
            gA[2 * e + 1][k] = gai[e];                                                   \
        }                                                                                \
    }                                                                                    \
}
#define adjoint_cplx_z_body adjoint_cplx_d
#define adjoint_cplx_c_body adjoint_cplx_s
SVD2O_BWD_CPLX(z, double)
SVD2O_BWD_CPLX(c, float)

/*
 * Reference gradient in binary128: the paper's method run in binary128 on the
 * exactly widened double input gives U, Sigma, V to ~1e-33; the adjoint is
 * then evaluated in binary128 with the given upstream gradients.  Output as
 * hi + lo double pairs.
 */
void svd2o_refgrad_d(int64_t n, const double *const A[4], const double *const gU[4],
                     const double *const gV[4], const double *g1, const double *g2,
                     double *const gA_hi[4], double *const gA_lo[4], double rel_delta)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const quad a[2][2] = { { A[0][k], A[2][k] }, { A[1][k], A[3][k] } };
        quad u[2][2], v[2][2], sx, sn, sc;
        int p;
        svd2_real_q(a, u, v, &sx, &sn, &sc, &p);
        if (sc != Q_MAX) {
            sx = Q_SCALBN(sx, -(int)sc);
            sn = Q_SCALBN(sn, -(int)sc);
        }
        const quad uq[4] = { u[0][0], u[1][0], u[0][1], u[1][1] };
        const quad vq[4] = { v[0][0], v[1][0], v[0][1], v[1][1] };
        const quad gu[4] = { gU[0][k], gU[1][k], gU[2][k], gU[3][k] };
        const quad gv[4] = { gV[0][k], gV[1][k], gV[2][k], gV[3][k] };
        quad ga[4];
        adjoint_q(uq, vq, sx, sn, gu, gv, g1[k], g2[k], rel_delta, ga);
        for (int e = 0; e < 4; ++e)
            q_split(ga[e], &gA_hi[e][k], &gA_lo[e][k]);
    }
}

/* Binary128 run of the paper's method on a double input (the O1 steps at
 * T = binary128), for reference singular vectors.  Outputs hi + lo pairs of
 * U, V and of the back-scaled singular values; piv receives the pivot bits. */
void svd2o_batch_q_from_d(int64_t n, const double *const A[4], double *const U_hi[4],
                          double *const U_lo[4], double *const V_hi[4],
                          double *const V_lo[4], double *smax_hi, double *smax_lo,
                          double *smin_hi, double *smin_lo, uint8_t *piv)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        const quad a[2][2] = { { A[0][k], A[2][k] }, { A[1][k], A[3][k] } };
        quad u[2][2], v[2][2], sx, sn, sc;
        int p;
        svd2_real_q(a, u, v, &sx, &sn, &sc, &p);
        if (sc != Q_MAX) {
            sx = Q_SCALBN(sx, -(int)sc);
            sn = Q_SCALBN(sn, -(int)sc);
        }
        const int map[4][2] = { { 0, 0 }, { 1, 0 }, { 0, 1 }, { 1, 1 } };
        for (int e = 0; e < 4; ++e) {
            q_split(u[map[e][0]][map[e][1]], &U_hi[e][k], &U_lo[e][k]);
            q_split(v[map[e][0]][map[e][1]], &V_hi[e][k], &V_lo[e][k]);
        }
        q_split(sx, &smax_hi[k], &smax_lo[k]);
        q_split(sn, &smin_hi[k], &smin_lo[k]);
        if (piv) piv[k] = (uint8_t)p;
    }
}

/* Constants the tests compare with the paper's printed values. */
double svd2o_const_sqrt_dbl_max_literal(void) { return 1.34078079299425956E+154; }
double svd2o_const_sqrt_dbl_max(void) { return sqrt(DBL_MAX); }
float svd2o_const_sqrt_flt_max(void) { return sqrtf(FLT_MAX); }
