"""Periodic steady state of a discharge from its per-period mean particle counts.

The paper reports that its discharges needed about 1000 to 4000 rf periods to reach the periodic
state (section "Numerical parameters and initial values") and that the initial values do not
change that state. The criterion used here (the library's reading): the state is steady from the
first period k at which the mean superparticle count of each species over periods [k-W, k)
differs by less than `tol` (relative) from the mean over [k-2W, k-W), with W = 50. Block means
rather than single periods keep the sampling noise of small runs below the threshold.
"""
from __future__ import annotations

import numpy as np


def steady_period(means: np.ndarray, window: int = 50, tol: float = 1e-3):
    """means: (periods, species) mean counts per rf period. Returns the first period index k at
    which the criterion holds, or None."""
    m = np.asarray(means, dtype=np.float64)
    if m.ndim == 1:
        m = m[:, None]
    c = np.concatenate([np.zeros((1, m.shape[1])), np.cumsum(m, axis=0)])
    for k in range(2 * window, m.shape[0] + 1):
        a = (c[k] - c[k - window]) / window
        b = (c[k - window] - c[k - 2 * window]) / window
        if np.all(a > 0) and np.all(np.abs(a - b) / a < tol):
            return k
    return None
