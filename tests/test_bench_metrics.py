"""bench.py's FP64 evaluation of the error metrics of Sec. 8 (Eq. 33 - Eq. 35)
against the oracle's binary128 evaluation, on the oracle's own FP32 results
(FP64 evaluation of float data is exact to far below the float errors)."""
import os
import sys
from types import SimpleNamespace

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2005_07403_gb300 import inputs  # noqa: E402


def test_error_metrics_match_oracle_binary128():
    A, _ = inputs.real_fp32_illcond(20000)
    o = oracle.svd2(A)
    r = SimpleNamespace(**{k: torch.from_numpy(o[k]) for k in ("U", "V", "smax", "smin", "s")})
    m = bench.error_metrics(torch, torch.from_numpy(A), r)
    d = lambda k: o[k].astype(np.float64)
    q = oracle.metrics(A.astype(np.float64), d("U"), d("V"), d("smax"), d("smin"), o["s"])
    for name in ("rho", "delta", "eta"):
        assert abs(m[name + "_max"] - q[name].max()) <= 1e-6 * q[name].max()
        p99 = np.sort(q[name])[int(np.ceil(0.99 * q[name].size)) - 1]
        assert abs(m[name + "_p99"] - p99) <= 1e-6 * p99
