"""Shared test helpers: fixture parsing and error measures.  No SVD arithmetic."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23
ZERO_S = 2**31 - 1


def hexf(tok, dtype=np.float64):
    return dtype(float.fromhex(tok))


def read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def bits_equal(a, b):
    """Bitwise equality of float arrays (distinguishes signed zeros)."""
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    assert a.dtype == b.dtype
    view = np.uint64 if a.dtype == np.float64 else np.uint32
    return np.array_equal(a.view(view), b.view(view))


def rel_err_hilo(x, hi, lo):
    """|x - (hi + lo)| / |hi + lo|, evaluated with the double-double truth."""
    x = np.asarray(x, np.float64)
    with np.errstate(all="ignore"):
        return np.abs((x - hi) - lo) / np.abs(hi)
