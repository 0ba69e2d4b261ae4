"""Oracle: XFNO extrapolation (Sec. 2, three occupation thresholds).

The paper extrapolates FNO energies obtained at three truncation thresholds
towards the untruncated limit, but prints no formula (the fit data sit in its
unavailable Supplementary Information). The reading here: a least-squares straight
line E(f) through the points (f_k, E_k), where f_k is the fraction of the total
natural-orbital occupation that was kept, evaluated at f = 1. It is applied to
every total energy independently.

Parity: unpinned against the paper (no data); pinned algebraically (exact on
linear data; returns E when every point has f = 1).
"""
from __future__ import annotations

import numpy as np


def extrapolate(kept_fraction, energy):
    """Least-squares line E(f) through the points, evaluated at f = 1 (Sec. 2, read as stated above)."""
    f = np.asarray(kept_fraction, dtype=np.float64)
    e = np.asarray(energy, dtype=np.float64)
    if len(f) != len(e) or len(f) == 0:
        raise ValueError("need matching, non-empty point lists")
    if np.ptp(f) == 0.0:
        return float(np.mean(e))
    a = np.stack([np.ones_like(f), f], axis=1)
    coef = np.linalg.lstsq(a, e, rcond=None)[0]
    return float(coef[0] + coef[1])
