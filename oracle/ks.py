"""Two-sample Kolmogorov-Smirnov distance (Eq. KS): max_x |F(x) - G(x)| over
the empirical CDFs, evaluated at every pooled sample point."""

import numpy as np


def ks_distance(a, b):
    a = np.sort(np.asarray(a, dtype=np.float64))
    b = np.sort(np.asarray(b, dtype=np.float64))
    pts = np.concatenate([a, b])
    fa = np.searchsorted(a, pts, side="right") / len(a)
    fb = np.searchsorted(b, pts, side="right") / len(b)
    return float(np.max(np.abs(fa - fb)))
