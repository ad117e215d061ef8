"""Error measures.  Test infrastructure: see ``oracle/__init__``."""
from __future__ import annotations

import numpy as np


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 over all entries (0 when both vanish)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    nd = np.linalg.norm(a - b)
    return 0.0 if nb == 0 and nd == 0 else nd / nb


def delta_l2_z(xi_appr, xi_exact):
    """Delta_L2(z) of Sec. 5.3: per X plane, ||xi_appr - xi_exact||_{L2(xy)} /
    ||xi_exact||_{L2(xy)} (NaN on planes where xi_exact vanishes)."""
    d = np.linalg.norm((np.asarray(xi_appr) - np.asarray(xi_exact)).reshape(len(xi_exact), -1), axis=1)
    n = np.linalg.norm(np.asarray(xi_exact).reshape(len(xi_exact), -1), axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(n > 0, d / n, np.nan)
