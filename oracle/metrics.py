"""Distribution metrics (float64).  Test infrastructure only."""
from __future__ import annotations

import numpy as np


def tv(p, q):
    """Total-variation distance 1/2 sum |p - q|."""
    return 0.5 * float(np.abs(np.asarray(p, np.float64) - np.asarray(q, np.float64)).sum())


def chi2(a, b):
    """Eq. 3: sum_i (a_i - b_i)^2 / (a_i + b_i), over the terms with
    a_i + b_i != 0 (a: evaluated distribution, b: ground truth)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    s = a + b
    m = s != 0
    return float(((a[m] - b[m]) ** 2 / s[m]).sum())


def norm_error(p):
    """|sum p - 1|."""
    return abs(float(np.asarray(p, np.float64).sum()) - 1.0)


def max_abs(p, q):
    return float(np.abs(np.asarray(p, np.float64) - np.asarray(q, np.float64)).max())


def clip_renormalise(p):
    """A reconstruction from finite-shot variants has negative entries; Eq. 3
    is stated for probability distributions, so the chi^2 reading here clips
    the negatives to 0 and rescales to total 1 first."""
    q = np.clip(np.asarray(p, np.float64), 0.0, None)
    return q / q.sum()
