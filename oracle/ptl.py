"""Practical time-step limit (Sec. 2, Eqs. 3-5).

Keeping the sign of every neighbour difference (Eq. 3), to first order in dt (the unnumbered
inequality after Eq. 3), only constrains dt where du != 0, dF != 0 and du dF < 0, and there
dt <= -du/dF (Eq. 4).  The condition is evaluated only at k = argmax |F| over all components
(the F_max localisation stated below Eq. 4), over the 6 orthogonal neighbours (Eq. 5):

    dt_PTL = min over neighbours j of k with (u_k - u_j)(F_k - F_j) < 0 of -(u_k - u_j)/(F_k - F_j).

Readings fixed by the project: ties in |F| go to the smallest flat index (component first, then
r fastest); neighbours that do not satisfy the Eq. 4 case are skipped (Eq. 5 written literally
would admit negative ratios); with no qualifying neighbour dt_PTL = +inf.
"""
from __future__ import annotations

import math

import numpy as np


def ptl(op, u: np.ndarray, F: np.ndarray):
    """Returns (dt_PTL, k, |F_k|)."""
    k = int(np.argmax(np.abs(F)))
    best = math.inf
    for j in op.neighbors(k):
        du = u[k] - u[j]
        dF = F[k] - F[j]
        if du != 0.0 and dF != 0.0 and du * dF < 0.0:
            best = min(best, -du / dF)
    return best, k, float(abs(F[k]))
