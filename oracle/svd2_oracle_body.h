/*
 * Precision-generic body of the CPU oracle for the batched 2x2 SVD of
 * V. Novakovic, "Batched computation of the singular value decompositions of
 * order two by the AVX-512 vectorization" (arXiv 2005.07403).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is included by svd2_oracle.c once per
 * floating type; it is plain, slow, scalar C that follows the paper's steps in
 * the paper's order and notation, one matrix at a time.  It shares nothing with
 * the CUDA path.  Only tests, the smoke check and the bench's CPU baseline use it.
 *
 * Before inclusion the includer defines:
 *   T            the floating type
 *   SFX(name)    name mangling for this type (e.g. name##_d)
 *   T_MAX        largest finite T           (DBL_MAX in the paper)
 *   T_TRUE_MIN   smallest positive T        (DBL_TRUE_MIN in the paper, Eq. 1)
 *   T_MAX_EXP    T's MAX_EXP                (h = T_MAX_EXP - 3, Sec. 2.1)
 *   T_SQRT_MAX   RN(sqrt(T_MAX))            (bound in Eq. 14)
 *   T_FMA, T_SQRT, T_FABS, T_COPYSIGN, T_LOGB, T_SCALBN
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - hypot is the paper's own naive formula (Sec. 5, text before Fig. 4), so the
 *    result is a fixed sequence of correctly rounded operations;
 *  - invsqrt(x) = 1/sqrt(x) with IEEE sqrt and IEEE division (Sec. 6, the first
 *    remedy named before Fig. 8);
 *  - min/max are the relaxed fmin/fmax defined in Sec. 2 after Eq. 1 (the
 *    VMINPD/VMAXPD semantics): pmin(a,b) = a < b ? a : b and pmax(a,b) =
 *    a > b ? a : b, so a NaN first argument, or two zeros of either sign,
 *    yield the second argument;
 *  - exp2 of Sec. 2.1 is logb (floor(lg|a|), exact for subnormals, -inf for 0);
 *    SCALEF is scalbn (round to nearest for subnormal results);
 *  - s stays a T as in Eq. 2, with T_MAX for the all-zero matrix;
 *  - the d's of the real case are +-1 carrying the sign bit (Eq. 10; Fig. 7
 *    applies them by XOR, which is the same as multiplying by +-1);
 *  - the U expansion after Eq. 29 is used as printed: inner complex value, then
 *    the complex product with d_ii (Eq. 5), then the real factor c; the V of
 *    Eq. 29 is formed as v11 = cos(psi), v12 = cos(psi) tan(psi),
 *    v21 = -d~22 (cos(psi) tan(psi)), v22 = d~22 cos(psi).
 */

/* Sec. 2, the relaxed fmin and fmax defined after Eq. 1: the smaller (larger)
 * of two non-NaN arguments, else the second argument. */
static inline T SFX(pmin)(T a, T b)
{
    return a < b ? a : b;
}

static inline T SFX(pmax)(T a, T b)
{
    return a > b ? a : b;
}

/* ---- Sec. 2 and Sec. 5 (before Fig. 4): hypot(a,b) without exponent
 * adjustment.  a' = max(|a|,|b|), b' = min(|a|,|b|), a+ = max(a', TRUE_MIN),
 * q+ = b'/a+ <= 1, c = a' * sqrt(fma(q+, q+, 1)).  hypot(a,b) = 0 iff a = b = 0. */
static inline T SFX(hypot_naive)(T a, T b)
{
    T aa = T_FABS(a), ab = T_FABS(b);
    T ap = SFX(pmax)(aa, ab);
    T bp = SFX(pmin)(aa, ab);
    T apl = SFX(pmax)(ap, T_TRUE_MIN);
    T q = bp / apl;
    return ap * T_SQRT(T_FMA(q, q, (T)1));
}

/* Sec. 2 (cosine formulas of Eq. 7, 15, 16) with the remedy of Sec. 6:
 * invsqrt(x) = 1/sqrt(x). */
static inline T SFX(invsqrt)(T x)
{
    return (T)1 / T_SQRT(x);
}

/* Eq. 1 as vectorized in Fig. 7 and Fig. 9: e^{i arg z} for z = (re, im) with
 * |z| = az given.  cos(arg z) = fmin(|Re z| / |z|, 1) with the sign of Re z
 * (the 0/0 NaN of z = 0 becomes 1 through fmin); sin(arg z) =
 * Im z / max(|z|, TRUE_MIN). */
static inline void SFX(cis_arg)(T re, T im, T az, T *cr, T *ci)
{
    *cr = T_COPYSIGN(SFX(pmin)(T_FABS(re) / az, (T)1), re);
    *ci = im / SFX(pmax)(az, T_TRUE_MIN);
}

/* Sec. 2.1, Eq. 2 and Fig. 3: s = min{T_MAX, min_ij (h - exp2 part_ij)} over the
 * np parts (4 real, 8 complex), h = MAX_EXP - 3, exp2 0 = -inf. */
static inline T SFX(scale_exponent)(const T *part, int np)
{
    const T h = (T)(T_MAX_EXP - 3);
    T s = T_MAX;
    for (int k = 0; k < np; ++k)
        s = SFX(pmin)(s, h - T_LOGB(part[k]));
    return s;
}

/* Fig. 3, last line: a_hat = SCALEF(a, s) = a * 2^s.  With s = T_MAX (all parts
 * zero) the parts are zeros and are kept as they are (0 * 2^s = 0, Sec. 2.1). */
static inline T SFX(scalef)(T a, T s)
{
    if (s == T_MAX)
        return a;
    return T_SCALBN(a, (int)s);
}

/*
 * One real 2x2 SVD, Sec. 2 with the real-case simplifications of Eq. 10 and the
 * figures' R-comments.  A[i][j] = a_{i+1,j+1}.  Outputs: U, V (row-major 2x2),
 * the scaled singular values sigma'_max >= sigma'_min (Eq. 17), the scale
 * exponent s (Eq. 2) and the two pivot bits (bit 0: P_c swapped the columns,
 * bit 1: P_r* swapped the rows).
 */
static inline void SFX(svd2_real_t)(const T A[2][2], T U[2][2], T V[2][2],
                           T *smax, T *smin, T *s_out, int *piv, T tau, int *wide,
                           int sine);

static inline void SFX(svd2_real)(const T A[2][2], T U[2][2], T V[2][2],
                           T *smax, T *smin, T *s_out, int *piv)
{
    int wide;
    SFX(svd2_real_t)(A, U, V, smax, smin, s_out, piv, (T)0, &wide, 0);
}

/*
 * The same with the tangent step of Eq. 6 - Eq. 7 optionally taken in the next
 * wider precision T_WIDE (defined for float only: the FP32 form with the FP64
 * tangent step).  When |r''_22| < tau r11 -- evaluated in T; r''_22 / r11 is
 * within a factor of two of sigma_min / sigma_max, because r11 <= sigma_max <=
 * sqrt(2) r11 after the column pivoting and sigma_max sigma_min = r11 r22 --
 * the quotient -tan(alpha) = pmax(a'''_21 / a'''_11, 0) and the fma of Eq. 7
 * are evaluated again in T_WIDE on the exactly widened a''' (in the real case
 * these are the scaled entries themselves, signs changed, so they are exact
 * in T), and r''_22 = RN_T(cos(alpha) RN_T(fma_W(tan(alpha), a'''_12, a'''_22))),
 * with the T value of cos(alpha).  Every other step stays in T.  *wide = 1
 * when the step ran.  tau = 0 never runs it (|r''_22| < 0 is false): that is
 * the plain method.  sine != 0 assembles U by Eq. 31 instead of Eq. 29 (see
 * below); V is the same either way.
 */
static inline void SFX(svd2_real_t)(const T A[2][2], T U[2][2], T V[2][2],
                           T *smax, T *smin, T *s_out, int *piv, T tau, int *wide,
                           int sine)
{
    /* Phase 1, Sec. 2.1: scale A by 2^s (Eq. 2, Fig. 3). */
    const T parts[4] = { A[0][0], A[1][0], A[0][1], A[1][1] };
    const T s = SFX(scale_exponent)(parts, 4);
    T Ah[2][2], absAh[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            Ah[i][j] = SFX(scalef)(A[i][j], s);
            absAh[i][j] = T_FABS(Ah[i][j]);        /* Fig. 4, real case */
        }

    /* Phase 2, Sec. 2.2.  Column norms, Eq. 3 / Fig. 4. */
    T nrm[2];
    for (int j = 0; j < 2; ++j)
        nrm[j] = SFX(hypot_naive)(absAh[0][j], absAh[1][j]);

    /* Column pivoting P_c (Fig. 5): swap iff ||a_1|| < ||a_2||. */
    const int pc = nrm[0] < nrm[1];
    T A1[2][2], absA1[2][2], nrm1[2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            A1[i][j] = Ah[i][pc ? 1 - j : j];
            absA1[i][j] = absAh[i][pc ? 1 - j : j];
        }
    nrm1[0] = nrm[pc ? 1 : 0];
    nrm1[1] = nrm[pc ? 0 : 1];

    /* Row sorting P_r* (Fig. 6): swap iff |a'_11| < |a'_21|. */
    const int pr = absA1[0][0] < absA1[1][0];
    T A2[2][2], absA2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            A2[i][j] = A1[pr ? 1 - i : i][j];
            absA2[i][j] = absA1[pr ? 1 - i : i][j];
        }

    /* D* of Eq. 10 (Fig. 7, real case): d_ii = sign a''_i1, a'''_i1 = |a''_i1|,
     * a'''_i2 = d_ii a''_i2. */
    T d[2], A3[2][2];
    for (int i = 0; i < 2; ++i) {
        d[i] = T_COPYSIGN((T)1, A2[i][0]);
        A3[i][0] = absA2[i][0];
        A3[i][1] = d[i] * A2[i][1];
    }

    /* QR by the Givens rotation Q_alpha*, Eq. 6 and Eq. 7 (Fig. 8).  r11 is the
     * already known norm of the first column. */
    const T r11 = nrm1[0];
    const T mtana = SFX(pmax)(A3[1][0] / A3[0][0], (T)0);      /* -tan(alpha) */
    const T tana = -mtana;
    const T cosa = SFX(invsqrt)(T_FMA(tana, tana, (T)1));
    const T r12p = cosa * T_FMA(mtana, A3[1][1], A3[0][1]);  /* r'_12 */
    T r22pp = cosa * T_FMA(tana, A3[0][1], A3[1][1]);        /* r''_22: -(-tan a * a12) + a22 */
    *wide = 0;
#ifdef T_WIDE
    if (T_FABS(r22pp) < tau * r11) {
        const T_WIDE q = (T_WIDE)A3[1][0] / (T_WIDE)A3[0][0];
        const T_WIDE mtw = q > (T_WIDE)0 ? q : (T_WIDE)0;       /* pmax(q, 0) */
        const T_WIDE g = T_WIDE_FMA(-mtw, (T_WIDE)A3[0][1], (T_WIDE)A3[1][1]);
        r22pp = cosa * (T)g;
        *wide = 1;
    }
#else
    (void)tau;
#endif

    /* D~ of Eq. 8 and D^* of Eq. 9, real case (Eq. 10, Fig. 9). */
    const T dt = T_COPYSIGN((T)1, r12p);     /* d~_22 */
    const T r12 = T_FABS(r12p);
    const T r22p = r22pp * dt;               /* r'_22 = r''_22 d~_22 */
    const T dh = T_COPYSIGN((T)1, r22p);     /* d^_22 */
    const T r22 = T_FABS(r22p);

    /* Phase 3, Sec. 2.3: SVD of R, Eq. 13 - Eq. 17 (Fig. 10). */
    const T x = SFX(pmax)(r12 / r11, (T)0);
    const T y = SFX(pmax)(r22 / r11, (T)0);
    const T num = ((T)2 * SFX(pmin)(x, y)) * SFX(pmax)(x, y);
    const T den = T_FMA(x - y, x + y, (T)1);
    const T tan2p = -SFX(pmin)(SFX(pmax)(num / den, (T)0), T_SQRT_MAX);   /* Eq. 14 */
    const T tanp = tan2p / ((T)1 + T_SQRT(T_FMA(tan2p, tan2p, (T)1))); /* Eq. 15 */
    const T sec2p = T_FMA(tanp, tanp, (T)1);
    const T cosp = SFX(invsqrt)(sec2p);
    const T tanq = T_FMA(y, tanp, -x);                               /* Eq. 16 */
    const T sec2q = T_FMA(tanq, tanq, (T)1);
    const T cosq = SFX(invsqrt)(sec2q);
    const T cpq = cosp * cosq;
    *smax = (cpq * sec2q) * r11;                                     /* Eq. 17 */
    *smin = (cpq * sec2p) * r22;

    /* Phase 4: Eq. 29 with c = cos(alpha) cos(phi), t = -tan(alpha) tan(phi).
     * Real case: d11, d22, d^22 are +-1, so the complex products reduce to
     * sign changes. */
    const T c = cosa * cosp;
    const T t = -(tana * tanp);
    T Ur[2][2];                              /* P_r* U */
    Ur[0][0] = c * (d[0] * T_FMA(dh, t, (T)1));
    Ur[1][0] = -(c * (d[1] * T_FMA(dh, tanp, tana)));
    Ur[0][1] = c * (d[0] * T_FMA(dh, tana, tanp));
    Ur[1][1] = c * (d[1] * T_FMA(-tana, tanp, dh));
    if (sine) {
        /* Eq. 31: the same U from the sines and cosines, sin = cos tan
         * (Sec. 7): pp = cos a cos p, qq = sin a sin p, rr = cos a sin p,
         * tt = sin a cos p, each combined with d^_22 by one fma. */
        const T sina = cosa * tana, sinp = cosp * tanp;
        const T pp = cosa * cosp, qq = sina * sinp, rr = cosa * sinp, tt = sina * cosp;
        Ur[0][0] = d[0] * T_FMA(-dh, qq, pp);
        Ur[0][1] = d[0] * T_FMA(dh, tt, rr);
        Ur[1][0] = -(d[1] * T_FMA(dh, rr, tt));
        Ur[1][1] = d[1] * T_FMA(dh, pp, -qq);
    }
    for (int i = 0; i < 2; ++i)              /* U = P_r (P_r* U) */
        for (int j = 0; j < 2; ++j)
            U[i][j] = Ur[pr ? 1 - i : i][j];

    const T w = cosq * tanq;
    T Vc[2][2];                              /* D~ V_psi */
    Vc[0][0] = cosq;
    Vc[0][1] = w;
    Vc[1][0] = -(dt * w);
    Vc[1][1] = dt * cosq;
    for (int i = 0; i < 2; ++i)              /* V = P_c (D~ V_psi) */
        for (int j = 0; j < 2; ++j)
            V[i][j] = Vc[pc ? 1 - i : i][j];

    *s_out = s;
    *piv = pc | (pr << 1);
}

/*
 * One complex 2x2 SVD, Sec. 2 (Eq. 1 - Eq. 29) as vectorized in Fig. 3 - Fig. 10,
 * one lane at a time.  Ar/Ai hold the real and imaginary parts of a_{i+1,j+1}.
 * sine != 0 assembles U by Eq. 31 instead of Eq. 29 (V is the same).
 */
static inline void SFX(svd2_cplx_t)(const T Ar[2][2], const T Ai[2][2],
                           T Ur[2][2], T Ui[2][2], T Vr[2][2], T Vi[2][2],
                           T *smax, T *smin, T *s_out, int *piv, int sine);

static inline void SFX(svd2_cplx)(const T Ar[2][2], const T Ai[2][2],
                           T Ur[2][2], T Ui[2][2], T Vr[2][2], T Vi[2][2],
                           T *smax, T *smin, T *s_out, int *piv)
{
    SFX(svd2_cplx_t)(Ar, Ai, Ur, Ui, Vr, Vi, smax, smin, s_out, piv, 0);
}

static inline void SFX(svd2_cplx_t)(const T Ar[2][2], const T Ai[2][2],
                           T Ur[2][2], T Ui[2][2], T Vr[2][2], T Vi[2][2],
                           T *smax, T *smin, T *s_out, int *piv, int sine)
{
    /* Phase 1: Eq. 2 over the real and the imaginary parts (Fig. 3). */
    const T parts[8] = { Ar[0][0], Ai[0][0], Ar[1][0], Ai[1][0],
                         Ar[0][1], Ai[0][1], Ar[1][1], Ai[1][1] };
    const T s = SFX(scale_exponent)(parts, 8);
    T Ahr[2][2], Ahi[2][2], absAh[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            Ahr[i][j] = SFX(scalef)(Ar[i][j], s);
            Ahi[i][j] = SFX(scalef)(Ai[i][j], s);
            absAh[i][j] = SFX(hypot_naive)(Ahr[i][j], Ahi[i][j]);   /* Eq. 1, Fig. 4 */
        }

    /* Column norms (Eq. 3) and the column pivoting (Fig. 5). */
    T nrm[2];
    for (int j = 0; j < 2; ++j)
        nrm[j] = SFX(hypot_naive)(absAh[0][j], absAh[1][j]);
    const int pc = nrm[0] < nrm[1];
    T A1r[2][2], A1i[2][2], absA1[2][2], nrm1[2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const int jj = pc ? 1 - j : j;
            A1r[i][j] = Ahr[i][jj];
            A1i[i][j] = Ahi[i][jj];
            absA1[i][j] = absAh[i][jj];
        }
    nrm1[0] = nrm[pc ? 1 : 0];
    nrm1[1] = nrm[pc ? 0 : 1];

    /* Row sorting (Fig. 6). */
    const int pr = absA1[0][0] < absA1[1][0];
    T A2r[2][2], A2i[2][2], absA2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const int ii = pr ? 1 - i : i;
            A2r[i][j] = A1r[ii][j];
            A2i[i][j] = A1i[ii][j];
            absA2[i][j] = absA1[ii][j];
        }

    /* D* of Eq. 4 (Fig. 7): d_ii = e^{i arg a''_i1}; a'''_i1 = |a''_i1|;
     * a'''_i2 = conj(d_ii) a''_i2 by the fma complex product of Eq. 5. */
    T dr[2], di[2], A3r[2][2], A3i[2][2];
    for (int i = 0; i < 2; ++i) {
        SFX(cis_arg)(A2r[i][0], A2i[i][0], absA2[i][0], &dr[i], &di[i]);
        A3r[i][1] = T_FMA(dr[i], A2r[i][1], di[i] * A2i[i][1]);
        A3i[i][1] = T_FMA(dr[i], A2i[i][1], -(di[i] * A2r[i][1]));
        A3r[i][0] = absA2[i][0];
        A3i[i][0] = (T)0;
    }

    /* QR, Eq. 6 and Eq. 7 (Fig. 8). */
    const T r11 = nrm1[0];
    const T mtana = SFX(pmax)(A3r[1][0] / A3r[0][0], (T)0);
    const T tana = -mtana;
    const T cosa = SFX(invsqrt)(T_FMA(tana, tana, (T)1));
    const T r12pr = cosa * T_FMA(mtana, A3r[1][1], A3r[0][1]);
    const T r12pi = cosa * T_FMA(mtana, A3i[1][1], A3i[0][1]);
    const T r22ppr = cosa * T_FMA(tana, A3r[0][1], A3r[1][1]);
    const T r22ppi = cosa * T_FMA(tana, A3i[0][1], A3i[1][1]);

    /* D~ of Eq. 8 (Fig. 9): r12 = |r'_12|; d~*_22 = e^{i arg r'_12};
     * r'_22 = r''_22 d~_22 = r''_22 conj(d~*_22). */
    const T r12 = SFX(hypot_naive)(r12pr, r12pi);
    T dtsr, dtsi;
    SFX(cis_arg)(r12pr, r12pi, r12, &dtsr, &dtsi);
    const T r22pr = T_FMA(r22ppr, dtsr, r22ppi * dtsi);
    const T r22pi = T_FMA(r22ppi, dtsr, -(r22ppr * dtsi));

    /* D^* of Eq. 9 (Fig. 9): r22 = |r'_22|; d^_22 = e^{i arg r'_22}. */
    const T r22 = SFX(hypot_naive)(r22pr, r22pi);
    T dhr, dhi;
    SFX(cis_arg)(r22pr, r22pi, r22, &dhr, &dhi);

    /* Phase 3, Eq. 13 - Eq. 17 (Fig. 10); identical to the real case. */
    const T x = SFX(pmax)(r12 / r11, (T)0);
    const T y = SFX(pmax)(r22 / r11, (T)0);
    const T num = ((T)2 * SFX(pmin)(x, y)) * SFX(pmax)(x, y);
    const T den = T_FMA(x - y, x + y, (T)1);
    const T tan2p = -SFX(pmin)(SFX(pmax)(num / den, (T)0), T_SQRT_MAX);
    const T tanp = tan2p / ((T)1 + T_SQRT(T_FMA(tan2p, tan2p, (T)1)));
    const T sec2p = T_FMA(tanp, tanp, (T)1);
    const T cosp = SFX(invsqrt)(sec2p);
    const T tanq = T_FMA(y, tanp, -x);
    const T sec2q = T_FMA(tanq, tanq, (T)1);
    const T cosq = SFX(invsqrt)(sec2q);
    const T cpq = cosp * cosq;
    *smax = (cpq * sec2q) * r11;
    *smin = (cpq * sec2p) * r22;

    /* Phase 4: the expansion of Eq. 29 printed after it.  Each element of
     * P_r* U is c * (d_ii * w) with the inner value w, the complex product by
     * Eq. 5, and the real factor c; the (2,1) element is negated. */
    const T c = cosa * cosp;
    const T t = -(tana * tanp);
    T wr[2][2], wi[2][2];
    wr[0][0] = T_FMA(dhr, t, (T)1);      wi[0][0] = dhi * t;
    wr[1][0] = T_FMA(dhr, tanp, tana);   wi[1][0] = dhi * tanp;
    wr[0][1] = T_FMA(dhr, tana, tanp);   wi[0][1] = dhi * tana;
    wr[1][1] = T_FMA(-tana, tanp, dhr);  wi[1][1] = dhi;
    T Prr[2][2], Pri[2][2];               /* P_r* U */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const T pr_ = T_FMA(dr[i], wr[i][j], -(di[i] * wi[i][j]));
            const T pi_ = T_FMA(dr[i], wi[i][j], di[i] * wr[i][j]);
            const T sg = (i == 1 && j == 0) ? (T)-1 : (T)1;
            Prr[i][j] = sg * (c * pr_);
            Pri[i][j] = sg * (c * pi_);
        }
    if (sine) {
        /* Eq. 31: each element of P_r* U is d_ii z_ij (Eq. 5), the (2,1)
         * element negated, with z from the sines and cosines (sin = cos tan,
         * Sec. 7) and d^_22 = dhr + i dhi:
         * z11 = pp - d^ qq, z12 = rr + d^ tt, z21 = tt + d^ rr, z22 = d^ pp - qq,
         * pp = cos a cos p, qq = sin a sin p, rr = cos a sin p, tt = sin a cos p. */
        const T sina = cosa * tana, sinp = cosp * tanp;
        const T pp = cosa * cosp, qq = sina * sinp, rr = cosa * sinp, tt = sina * cosp;
        T zr[2][2], zi[2][2];
        zr[0][0] = T_FMA(-dhr, qq, pp);   zi[0][0] = -(dhi * qq);
        zr[0][1] = T_FMA(dhr, tt, rr);    zi[0][1] = dhi * tt;
        zr[1][0] = T_FMA(dhr, rr, tt);    zi[1][0] = dhi * rr;
        zr[1][1] = T_FMA(dhr, pp, -qq);   zi[1][1] = dhi * pp;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                const T pr_ = T_FMA(dr[i], zr[i][j], -(di[i] * zi[i][j]));
                const T pi_ = T_FMA(dr[i], zi[i][j], di[i] * zr[i][j]);
                const T sg = (i == 1 && j == 0) ? (T)-1 : (T)1;
                Prr[i][j] = sg * pr_;
                Pri[i][j] = sg * pi_;
            }
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            Ur[i][j] = Prr[pr ? 1 - i : i][j];
            Ui[i][j] = Pri[pr ? 1 - i : i][j];
        }

    /* V = P_c D~ V_psi (Eq. 29), d~_22 = conj(d~*_22). */
    const T w = cosq * tanq;
    T Vcr[2][2], Vci[2][2];
    Vcr[0][0] = cosq;          Vci[0][0] = (T)0;
    Vcr[0][1] = w;             Vci[0][1] = (T)0;
    Vcr[1][0] = -(dtsr * w);   Vci[1][0] = dtsi * w;
    Vcr[1][1] = dtsr * cosq;   Vci[1][1] = -(dtsi * cosq);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            Vr[i][j] = Vcr[pc ? 1 - i : i][j];
            Vi[i][j] = Vci[pc ? 1 - i : i][j];
        }

    *s_out = s;
    *piv = pc | (pr << 1);
}

/*
 * Reverse-mode derivative of A = U diag(s1, s2) V^T (real, s1 >= s2 >= 0) for a
 * loss with gradients gU, gV (element order u11, u21, u12, u22) and g1, g2.  The
 * paper has no backward; this is the square-SVD adjoint written out for order
 * two (derivation in the design notes):
 *   J = U^T gU, K = V^T gV, a = J12 - J21, b = K12 - K21,
 *   M = [[g1, (a-b)/(2(s1+s2)) - (a+b)/(2(s1-s2))],
 *        [-(a-b)/(2(s1+s2)) - (a+b)/(2(s1-s2)), g2]],
 *   gA = U M V^T.
 * 1/(s1 - s2) is safeguarded for nearly equal singular values: with the
 * relative gap g = (s1 - s2)/s1 it is replaced by g / (s1 (g^2 + dl^2)), which
 * is 1/(s1 - s2) for g >> dl and tends to 0 as g -> 0.  s1 + s2 = 0 (A = 0)
 * gives 0 for both rotation terms.
 */
static inline void SFX(adjoint)(const T u[4], const T v[4], T s1, T s2, const T gu[4],
                         const T gv[4], T g1, T g2, T dl, T ga[4])
{
    const T u11 = u[0], u21 = u[1], u12 = u[2], u22 = u[3];
    const T v11 = v[0], v21 = v[1], v12 = v[2], v22 = v[3];
    /* every two-term dot product as fma(x0, y0, x1 y1) */
    const T J12 = T_FMA(u11, gu[2], u21 * gu[3]);
    const T J21 = T_FMA(u12, gu[0], u22 * gu[1]);
    const T K12 = T_FMA(v11, gv[2], v21 * gv[3]);
    const T K21 = T_FMA(v12, gv[0], v22 * gv[1]);
    const T a = J12 - J21, b = K12 - K21;
    const T sum = s1 + s2;
    const T inv_sum = sum > (T)0 ? (T)1 / sum : (T)0;
    T inv_gap = (T)0;
    if (s1 > (T)0) {
        const T g = (s1 - s2) / s1;
        /* g = 0 (s1 = s2): the safeguard's value there, 0, also at dl = 0,
         * where the formula reads 0/0 */
        inv_gap = g == (T)0 ? (T)0 : g / (s1 * T_FMA(g, g, dl * dl));
    }
    const T p = (T)0.5 * (a - b) * inv_sum;
    const T q = (T)0.5 * (a + b) * inv_gap;
    const T m11 = g1, m12 = p - q, m21 = -p - q, m22 = g2;
    /* W = U M, then gA = W V^T */
    const T w11 = T_FMA(u11, m11, u12 * m21), w12 = T_FMA(u11, m12, u12 * m22);
    const T w21 = T_FMA(u21, m11, u22 * m21), w22 = T_FMA(u21, m12, u22 * m22);
    ga[0] = T_FMA(w11, v11, w12 * v12);   /* gA_11 */
    ga[1] = T_FMA(w21, v11, w22 * v12);   /* gA_21 */
    ga[2] = T_FMA(w11, v21, w12 * v22);   /* gA_12 */
    ga[3] = T_FMA(w21, v21, w22 * v22);   /* gA_22 */
}

/*
 * Reverse-mode derivative of the complex A = U diag(s1, s2) V^* (s1 >= s2 >= 0,
 * U and V unitary).  Elements in the record order x11, x21, x12, x22 (element
 * (r, c) at r + 2c) with separate real and imaginary parts; every gradient g is
 * dL/dRe + i dL/dIm (the convention under which dL = Re sum conj(g) dx).  The
 * paper has no backward; derived from the mathematics (see the design notes):
 * with dP = U^* dA V = Omega_U Sigma + dSigma - Sigma Omega_V (Omega_U = U^* dU,
 * Omega_V = V^* dV skew-Hermitian), J = U^* gU, K = V^* gV,
 *   a = J12 - conj(J21), b = K12 - conj(K21),
 *   p = (a - b) / (2 (s1 + s2)), q = (a + b) / (2 (s1 - s2)),
 *   M = [[g1 + i t1, p - q], [-conj(p) - conj(q), g2 + i t2]],
 *   t_i = (Im J_ii - Im K_ii) / (2 s_i)   (0 when s_i = 0),
 *   gA = U M V^*.
 * The diagonal terms t_i carry the phase gauge (U, V -> U D, V D for a unitary
 * diagonal D): for a loss that is invariant under it Im J_ii + Im K_ii = 0 and
 * t_i = Im J_ii / s_i.  1/(s1 - s2) is safeguarded as in the real adjoint, and
 * for real data the result is the real adjoint's.
 */
static inline void SFX(adjoint_cplx)(const T ur[4], const T ui[4], const T vr[4], const T vi[4],
                              T s1, T s2, const T gur[4], const T gui[4], const T gvr[4],
                              const T gvi[4], T g1, T g2, T dl, T gar[4], T gai[4])
{
    /* J_xy = sum_a conj(u_ax) gu_ay, element (a, x) at a + 2x; every four-term
     * sum as the fma chain x0 y0 + (x1 y1 + (x2 y2 + x3 y3)), innermost a product */
#define CRE(x, y, a0, b0, a1, b1) T_FMA(x##r[a0], y##r[b0], T_FMA(x##i[a0], y##i[b0], \
        T_FMA(x##r[a1], y##r[b1], x##i[a1] * y##i[b1])))
#define CIM(x, y, a0, b0, a1, b1) T_FMA(x##r[a0], y##i[b0], T_FMA(-x##i[a0], y##r[b0], \
        T_FMA(x##r[a1], y##i[b1], -(x##i[a1] * y##r[b1]))))
    const T Jr12 = CRE(u, gu, 0, 2, 1, 3), Ji12 = CIM(u, gu, 0, 2, 1, 3);
    const T Jr21 = CRE(u, gu, 2, 0, 3, 1), Ji21 = CIM(u, gu, 2, 0, 3, 1);
    const T Ji11 = CIM(u, gu, 0, 0, 1, 1), Ji22 = CIM(u, gu, 2, 2, 3, 3);
    const T Kr12 = CRE(v, gv, 0, 2, 1, 3), Ki12 = CIM(v, gv, 0, 2, 1, 3);
    const T Kr21 = CRE(v, gv, 2, 0, 3, 1), Ki21 = CIM(v, gv, 2, 0, 3, 1);
    const T Ki11 = CIM(v, gv, 0, 0, 1, 1), Ki22 = CIM(v, gv, 2, 2, 3, 3);
#undef CRE
#undef CIM
    /* a = J12 - conj(J21), b = K12 - conj(K21) */
    const T ar = Jr12 - Jr21, ai = Ji12 + Ji21;
    const T br = Kr12 - Kr21, bi = Ki12 + Ki21;
    const T sum = s1 + s2;
    const T inv_sum = sum > (T)0 ? (T)1 / sum : (T)0;
    T inv_gap = (T)0;
    if (s1 > (T)0) {
        const T g = (s1 - s2) / s1;
        /* g = 0 (s1 = s2): the safeguard's value there, 0, also at dl = 0,
         * where the formula reads 0/0 */
        inv_gap = g == (T)0 ? (T)0 : g / (s1 * T_FMA(g, g, dl * dl));
    }
    const T pr = (T)0.5 * (ar - br) * inv_sum, pi = (T)0.5 * (ai - bi) * inv_sum;
    const T qr = (T)0.5 * (ar + br) * inv_gap, qi = (T)0.5 * (ai + bi) * inv_gap;
    const T t1 = s1 > (T)0 ? (T)0.5 * (Ji11 - Ki11) / s1 : (T)0;
    const T t2 = s2 > (T)0 ? (T)0.5 * (Ji22 - Ki22) / s2 : (T)0;
    /* M in the record order m11, m21, m12, m22 */
    const T mr[4] = { g1, -pr - qr, pr - qr, g2 };
    const T mi[4] = { t1, pi + qi, pi - qi, t2 };
    /* W = U M: w_xy = u_x1 m_1y + u_x2 m_2y */
    T wr[4], wi[4];
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
            const int o = x + 2 * y, u1 = x, u2 = x + 2, m1 = 2 * y, m2 = 2 * y + 1;
            wr[o] = T_FMA(ur[u1], mr[m1], T_FMA(-ui[u1], mi[m1],
                          T_FMA(ur[u2], mr[m2], -(ui[u2] * mi[m2]))));
            wi[o] = T_FMA(ur[u1], mi[m1], T_FMA(ui[u1], mr[m1],
                          T_FMA(ur[u2], mi[m2], ui[u2] * mr[m2])));
        }
    /* gA = W V^*: ga_xy = w_x1 conj(v_y1) + w_x2 conj(v_y2) */
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
            const int o = x + 2 * y, w1 = x, w2 = x + 2, v1 = y, v2 = y + 2;
            gar[o] = T_FMA(wr[w1], vr[v1], T_FMA(wi[w1], vi[v1],
                           T_FMA(wr[w2], vr[v2], wi[w2] * vi[v2])));
            gai[o] = T_FMA(wi[w1], vr[v1], T_FMA(-wr[w1], vi[v1],
                           T_FMA(wi[w2], vr[v2], -(wr[w2] * vi[v2]))));
        }
}
