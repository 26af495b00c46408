"""Practical time-step limit (Sec. 2, Eqs. 3-5).

Keeping the sign of every neighbour difference (Eq. 3), to first order in dt (the unnumbered
inequality after Eq. 3), only constrains dt where du != 0, dF != 0 and du dF < 0, and there
dt <= -du/dF (Eq. 4).  The condition is evaluated only at k = argmax |F| over all components
(the F_max localisation stated below Eq. 4), over the 6 orthogonal neighbours (Eq. 5):

    dt_PTL = min over neighbours j of k with (u_k - u_j)(F_k - F_j) < 0 of -(u_k - u_j)/(F_k - F_j).

Readings fixed by the project: ties in |F| go to the smallest flat index (component first, then
r fastest); neighbours that do not satisfy the Eq. 4 case are skipped (Eq. 5 written literally
would admit negative ratios); with no qualifying neighbour dt_PTL = +inf.

ptl_full drops the localisation: Sec. 2 notes that the Eq. 4 condition can be checked over every
cell in every direction and the minimum taken, which Eq. 5 avoids by assuming the minimum lies at
F_max.  Every unordered pair of face neighbours (i, j) of one component is taken once, as
(i, i + e_d) with d = 0 (r), 1 (theta), 2 (phi, periodic; on the periodic box r and theta wrap
too); -du/dF is symmetric in i and j.  Ties in the bound go to the smallest key 3 i + d.
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


def ptl_full(op, u: np.ndarray, F: np.ndarray):
    """Returns (dt, key): the smallest Eq. 4 bound over all pairs of face neighbours and the pair
    (i, i + e_d) as key = 3 i + d, or (inf, -1) when no pair qualifies."""
    offsets = getattr(op, "offsets", [0])
    best, best_key = math.inf, -1
    for shape, off in zip(op.shapes, offsets):
        n = int(np.prod(shape))
        U = u[off:off + n].reshape(shape)
        G = F[off:off + n].reshape(shape)
        idx = off + np.arange(n, dtype=np.int64).reshape(shape)
        # (cell, neighbour) arrays per direction; axes are (phi, theta, r)
        if getattr(op, "periodic", False):     # the box: r and theta wrap too
            pairs = [(U, np.roll(U, -1, axis=a), G, np.roll(G, -1, axis=a), idx, d)
                     for d, a in ((0, 2), (1, 1), (2, 0))]
        else:
            pairs = [
                (U[:, :, :-1], U[:, :, 1:], G[:, :, :-1], G[:, :, 1:], idx[:, :, :-1], 0),
                (U[:, :-1, :], U[:, 1:, :], G[:, :-1, :], G[:, 1:, :], idx[:, :-1, :], 1),
                (U, np.roll(U, -1, axis=0), G, np.roll(G, -1, axis=0), idx, 2),
            ]
        for ua, ub, fa, fb, ia, d in pairs:
            du = ua - ub
            dF = fa - fb
            ok = (du != 0.0) & (dF != 0.0) & (du * dF < 0.0)
            if not ok.any():
                continue
            bound = -du[ok] / dF[ok]
            keys = 3 * ia[ok] + d
            m = float(bound.min())
            kmin = int(keys[bound == m].min())
            if m < best or (m == best and kmin < best_key):
                best, best_key = m, kmin
    return best, best_key
