"""Growth-rate extraction from a field-energy history -- TEST INFRASTRUCTURE ONLY.

The paper extracts linear growth rates from the exponential stage of the field-energy
histories (results section).  It does not say how; the reading used here:
  * W0 = mean of W over t <= t_noise (the noise level);
  * a candidate window is `width` consecutive samples, all with W > start_factor * W0 and
    W < max(W) * end_factor (after the noise, before saturation; end_factor=None drops the
    upper bound for histories that end inside the exponential stage);
  * ln W is fitted by least squares over every candidate window; the largest slope wins;
  * the field energy grows as exp(2 Gamma t), so Gamma = slope / 2.
"""
from __future__ import annotations

import numpy as np


def growth_rate(t, W, width=60, t_noise=2.0, start_factor=10.0, end_factor=1.0 / 30.0):
    """Return (Gamma, t_start, t_end); Gamma is nan when no window qualifies."""
    t = np.asarray(t, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    noise = W[t <= t_noise]
    if noise.size == 0 or W.size < width:
        return float("nan"), float("nan"), float("nan")
    lo = start_factor * noise.mean()
    hi = np.inf if end_factor is None else W.max() * end_factor
    ok = (W > lo) & (W < hi)
    best = (float("nan"), float("nan"), float("nan"))
    best_slope = -np.inf
    for a in range(0, W.size - width + 1):
        if not ok[a:a + width].all():
            continue
        tt = t[a:a + width]
        yy = np.log(W[a:a + width])
        tm = tt.mean()
        slope = np.sum((tt - tm) * (yy - yy.mean())) / np.sum((tt - tm) ** 2)
        if slope > best_slope:
            best_slope = slope
            best = (0.5 * slope, float(tt[0]), float(tt[-1]))
    return best
