"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them (a wrong sign, a dropped term, a transposed operand, a
wrong index, an off-by-one constant).  The mistakes are planted in the oracle
only, on the CPU; nothing here touches the CUDA path."""
import os

import numpy as np
import pytest

import oracle
from paper_2005_07403_gb300 import inputs
from tests.helpers import EPS64, ZERO_S, bits_equal, hexf, read_rows

HERE = os.path.dirname(os.path.abspath(oracle.__file__))
SRC = open(os.path.join(HERE, "svd2_oracle.c")).read()
BODY = open(os.path.join(HERE, "svd2_oracle_body.h")).read()

MUTATIONS = {
    "r22_sign": ("T r22pp = cosa * T_FMA(tana, A3[0][1], A3[1][1]);",
                 "T r22pp = cosa * T_FMA(mtana, A3[0][1], A3[1][1]);"),
    # the FP64 tangent step of the FP32 form (Eq. 6 - Eq. 7 in double)
    "wide_quotient_in_float": ("const T_WIDE q = (T_WIDE)A3[1][0] / (T_WIDE)A3[0][0];",
                               "const T_WIDE q = (T_WIDE)(A3[1][0] / A3[0][0]);"),
    "wide_fma_sign": ("T_WIDE_FMA(-mtw, (T_WIDE)A3[0][1], (T_WIDE)A3[1][1]);",
                      "T_WIDE_FMA(mtw, (T_WIDE)A3[0][1], (T_WIDE)A3[1][1]);"),
    "wide_operands_swapped": ("T_WIDE_FMA(-mtw, (T_WIDE)A3[0][1], (T_WIDE)A3[1][1]);",
                              "T_WIDE_FMA(-mtw, (T_WIDE)A3[1][1], (T_WIDE)A3[0][1]);"),
    "wide_test_reversed": ("if (T_FABS(r22pp) < tau * r11) {", "if (T_FABS(r22pp) > tau * r11) {"),
    "wide_cos_dropped": ("r22pp = cosa * (T)g;", "r22pp = (T)g;"),
    # the sine-based assembly of Eq. 31
    "eq31_dhat_sign": ("zr[0][0] = T_FMA(-dhr, qq, pp);", "zr[0][0] = T_FMA(dhr, qq, pp);"),
    "eq31_terms_swapped": ("zr[0][1] = T_FMA(dhr, tt, rr);", "zr[0][1] = T_FMA(dhr, rr, tt);"),
    "eq31_real_u21_sign": ("Ur[1][0] = -(d[1] * T_FMA(dh, rr, tt));",
                           "Ur[1][0] = (d[1] * T_FMA(dh, rr, tt));"),
    "eq31_sine_without_cos": ("const T sina = cosa * tana, sinp = cosp * tanp;",
                              "const T sina = tana, sinp = cosp * tanp;"),
    "eq31_d22_conj": ("const T pi_ = T_FMA(dr[i], zi[i][j], di[i] * zr[i][j]);",
                      "const T pi_ = T_FMA(dr[i], zi[i][j], -(di[i] * zr[i][j]));"),
    "u21_sign": ("Ur[1][0] = -(c * (d[1] * T_FMA(dh, tanp, tana)));",
                 "Ur[1][0] = (c * (d[1] * T_FMA(dh, tanp, tana)));"),
    "tanpsi_transposed": ("const T tanq = T_FMA(y, tanp, -x);",
                          "const T tanq = T_FMA(x, tanp, -y);"),
    "col_pivot_reversed": ("const int pc = nrm[0] < nrm[1];",
                           "const int pc = nrm[0] > nrm[1];"),
    "hypot_dropped_square": ("return ap * T_SQRT(T_FMA(q, q, (T)1));",
                             "return ap * T_SQRT(q + (T)1);"),
    "v21_sign": ("Vc[1][0] = -(dt * w);", "Vc[1][0] = (dt * w);"),
    "conj_dropped": ("A3i[i][1] = T_FMA(dr[i], A2i[i][1], -(di[i] * A2r[i][1]));",
                     "A3i[i][1] = T_FMA(dr[i], A2i[i][1], (di[i] * A2r[i][1]));"),
    "h_off_by_one": ("const T h = (T)(T_MAX_EXP - 3);", "const T h = (T)(T_MAX_EXP - 2);"),
    "tan2phi_dropped_2": ("const T num = ((T)2 * SFX(pmin)(x, y)) * SFX(pmax)(x, y);",
                          "const T num = SFX(pmin)(x, y) * SFX(pmax)(x, y);"),
    "alpha_quotient_inverted": ("const T mtana = SFX(pmax)(A3[1][0] / A3[0][0], (T)0);",
                                "const T mtana = SFX(pmax)(A3[0][0] / A3[1][0], (T)0);"),
    "u_cmul_sign": ("const T pi_ = T_FMA(dr[i], wi[i][j], di[i] * wr[i][j]);",
                    "const T pi_ = T_FMA(dr[i], wi[i][j], -(di[i] * wr[i][j]));"),
    "real_dstar_dropped": ("A3[i][1] = d[i] * A2[i][1];", "A3[i][1] = A2[i][1];"),
    "row_sort_wrong_index": ("const int pr = absA1[0][0] < absA1[1][0];",
                             "const int pr = absA1[0][0] < absA1[0][1];"),
    "sigma_min_wrong_secant": ("*smin = (cpq * sec2p) * r22;", "*smin = (cpq * sec2q) * r22;"),
    "u12_swapped_tangents": ("wr[0][1] = T_FMA(dhr, tana, tanp);", "wr[0][1] = T_FMA(dhr, tanp, tana);"),
}


def pin_failures(o):
    """Run a compact version of the pins against oracle build ``o``; return the
    names of those that fail."""
    failed = []
    with np.errstate(all="ignore"):
        for rows, seed in ((4, 901), (8, 902)):
            A = inputs.normal_batch(3000, rows, seed)
            r = o.svd2(A)
            sxh, sxl, snh, snl = o.truth(A, r["s"])
            ex = np.abs((r["smax"] - sxh) - sxl) / sxh
            en = np.abs((r["smin"] - snh) - snl) / sxh
            if not (np.nanmax(ex) <= 4 * EPS64 and np.nanmax(en) <= 4 * EPS64
                    and np.isfinite(ex).all()):
                failed.append(f"sigma{rows}")
            m = o.metrics(A, r["U"], r["V"], r["smax"], r["smin"], r["s"])
            if not (m["rho"].max() <= 8 * EPS64):
                failed.append(f"rho{rows}")
            if not (max(m["delta"].max(), m["eta"].max()) <= 16 * EPS64):
                failed.append(f"orth{rows}")
            _, e = np.frexp(A)
            e = np.where(A != 0, e.astype(np.int64) - 1, -(2**62))
            emax = e.max(axis=0)
            if not np.array_equal(r["s"].astype(np.int64), 1021 - emax):
                failed.append(f"s{rows}")
        # the FP32 form with the FP64 tangent step: sigma_min of the matrices that
        # take it against the binary128 closed form (kappa <= 2^24), the trigger
        # against sigma_min / sigma_max, sigma_max throughout
        A32, _ = inputs.real_fp32_illcond(20000, seed=903)
        r = o.svd2_tan64(A32, -4)
        A64 = A32.astype(np.float64)
        sxh, sxl, snh, snl = o.truth(A64, r["s"])
        u = 2.0**-24
        ex = np.abs((r["smax"].astype(np.float64) - sxh) - sxl) / sxh / u
        en = np.abs((r["smin"].astype(np.float64) - snh) - snl) / snh / u
        ratio = (snh + snl) / (sxh + sxl)
        w = r["wide"].astype(bool)
        sel = w & (ratio >= 2.0**-24)
        if not (np.nanmax(ex) <= 8 and sel.any() and np.nanmax(en[sel]) <= 8
                and np.all(w[ratio < 2.0**-5 * 0.999]) and not np.any(w & (ratio > 2.0**-4 * 1.001))):
            failed.append("tan64")
        # the sine-based assembly of Eq. 31: accuracy of Sec. 8 and agreement
        # with the tangent form
        for rows, seed in ((4, 904), (8, 905)):
            A = inputs.normal_batch(3000, rows, seed)
            t = o.svd2(A)
            r = o.svd2(A, sine=True)
            m = o.metrics(A, r["U"], r["V"], r["smax"], r["smin"], r["s"])
            if not (m["rho"].max() <= 8 * EPS64
                    and max(m["delta"].max(), m["eta"].max()) <= 16 * EPS64
                    and np.abs(r["U"] - t["U"]).max() <= 3 * EPS64):
                failed.append(f"eq31_{rows}")
        for row in read_rows("hand_cases.txt"):
            fields = dict(tok.split("=") for tok in row[1:])
            A = np.array([[hexf(t)] for t in fields["A"].split(",")])
            r = o.svd2(A)
            U = np.array([hexf(t) for t in fields["U"].split(",")])
            if not bits_equal(r["U"][:, 0], U) or int(r["s"][0]) != int(fields["s"]):
                failed.append("hand_" + row[0])
    return failed


def test_unmutated_oracle_passes_compact_pins(tmp_path):
    o = oracle.build_variant(SRC, BODY, str(tmp_path))
    assert pin_failures(o) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    assert old in BODY, name
    o = oracle.build_variant(SRC, BODY.replace(old, new), str(tmp_path))
    assert pin_failures(o), f"mistake {name} went unnoticed"
