"""Field-aligned thermal conduction, Eq. 2 (right):

    F_tc(T) = C / n * div( kappa b b . grad T ),   kappa = T0^{5/2} (lagged, Sec. 2 below Eq. 2),
    C = (gamma - 1)/2 with gamma = 5/3, and m_p/k, kappa_0, f_c, f_m folded to 1.

Discretisation (the paper gives none; this is the reading the project fixes): a symmetric corner
("dual-cell") scheme.  At every interior corner c the field-aligned gradient is

    s_c = ahat_c . D_c,    D_c,x = sum over the 4 cell pairs straddling c along x of (u+ - u-),
    ahat_c = sqrt(W_c kappa_c) (h_r b_r, h_t b_t, h_p b_p)_c / 4,

with kappa_c the mean of the 8 surrounding cells' T0^{5/2}, b = B/|B| at the corner (the paper
prints |B|/B, read as the unit vector B/|B|), h the corner metric factors and W_c the corner's
dual volume.  The energy E = 1/2 sum_c s_c^2 gives the symmetric negative semi-definite
A = -grad^2 E, i.e.

    (A u)_cell = - sum over the 8 corners c of the cell of  sigma(p) . (ahat_c s_c),

where p in {0,1}^3 is the cell's position inside corner c and sigma(p) = 2p - 1.  Then
F = w A u with the cell weight w = C / (n V).  Corners on r_min, r_max and the poles are absent
(ahat = 0), which makes every boundary zero-flux and keeps M A symmetric (M = diag(1/w)).

The periodic box (TCOperator.box) is the same scheme on unit cells (h = 1, W = V = 1) with every
corner present and all three directions periodic: the geometry on which Fourier modes are
eigenvectors with the closed-form eigenvalues used to pin the schemes.
"""
from __future__ import annotations

import numpy as np

from .geometry import CUBE, Shell, shift

C_TC = (5.0 / 3.0 - 1.0) / 2.0


def sigma(p):
    """Sign vector (r, theta, phi) of a cell at position p = (pk, pj, pi) inside a corner."""
    pk, pj, pi = p
    return (2 * pi - 1, 2 * pj - 1, 2 * pk - 1)


class TCOperator:
    """Thermal conduction on one scalar field; state vectors are flat (r fastest)."""

    ncomp = 1

    def __init__(self, ahat: np.ndarray, w: np.ndarray, periodic: bool = False):
        """periodic: r and theta wrap as phi does (the box); the PTL then has six neighbours
        everywhere."""
        self.ahat = np.asarray(ahat, dtype=np.float64)      # (3, n_p, n_t, n_r)
        self.w3 = np.asarray(w, dtype=np.float64)            # (n_p, n_t, n_r)
        self.shape = self.w3.shape
        self.shapes = [self.shape]
        self.n = self.w3.size
        self.w = self.w3.reshape(-1)
        self.periodic = periodic

    @classmethod
    def box(cls, T0: np.ndarray, n: np.ndarray, B, C: float = C_TC):
        """Periodic box of unit cells: kappa_c the mean of the 8 cells' T0^{5/2} (wrapping),
        b = B/|B| at the corners (corner [k, j, i] between cells i..i+1, j..j+1, k..k+1),
        ahat = sqrt(kappa_c) b / 4 and w = C / n."""
        kappa = np.asarray(T0, dtype=np.float64) ** 2.5
        kc = sum(shift(kappa, *p) for p in CUBE) / 8.0
        br, bt, bp = (np.asarray(b, dtype=np.float64) for b in B)
        bmag = np.sqrt(br * br + bt * bt + bp * bp)
        root = np.sqrt(kc)
        ahat = np.stack([root * br / bmag, root * bt / bmag, root * bp / bmag]) / 4.0
        return cls(ahat, C / np.asarray(n, dtype=np.float64), periodic=True)

    @classmethod
    def spherical(cls, shell: Shell, T0: np.ndarray, n: np.ndarray, B, C: float = C_TC):
        """Build the operator from the lagged temperature T0 and density n (cells) and the
        magnetic field B = (B_r, B_t, B_p) at the corners."""
        kappa = np.asarray(T0, dtype=np.float64) ** 2.5
        kc = sum(shift(kappa, *p) for p in CUBE) / 8.0
        br, bt, bp = (np.asarray(b, dtype=np.float64) for b in B)
        bmag = np.sqrt(br * br + bt * bt + bp * bp)
        hr, ht, hp, W = shell.corner_metric()
        root = np.sqrt(W[None, :, :] * kc)
        ahat = np.stack([root * hr[None] * (br / bmag),
                         root * ht[None] * (bt / bmag),
                         root * hp[None] * (bp / bmag)]) / 4.0
        ahat[:, :, W == 0.0] = 0.0
        w = C / (np.asarray(n, dtype=np.float64) * shell.cell_volume())
        return cls(ahat, w)

    # -- operator application ------------------------------------------------------------------
    def corner_flux(self, u3: np.ndarray):
        """Q_c = ahat_c s_c (3 components) at every corner."""
        D = [0.0, 0.0, 0.0]
        for p in CUBE:
            v = shift(u3, *p)
            sg = sigma(p)
            for x in range(3):
                D[x] = D[x] + sg[x] * v
        s = self.ahat[0] * D[0] + self.ahat[1] * D[1] + self.ahat[2] * D[2]
        return [self.ahat[x] * s for x in range(3)]

    def apply_A(self, u: np.ndarray) -> np.ndarray:
        u3 = np.asarray(u, dtype=np.float64).reshape(self.shape)
        Q = self.corner_flux(u3)
        Au = np.zeros(self.shape)
        for p in CUBE:
            sg = sigma(p)
            back = (-p[0], -p[1], -p[2])       # corner index = cell index - p
            for x in range(3):
                Au -= sg[x] * shift(Q[x], *back)
        return Au.reshape(-1)

    def apply(self, u: np.ndarray) -> np.ndarray:
        return self.w * self.apply_A(u)

    # -- matrix rows -----------------------------------------------------------------------------
    def row_entries(self) -> dict:
        """A[cell, cell + o] for the 27 offsets o = (ok, oj, oi), as arrays indexed by cell.
        A = -sum_c g_c g_c^T with g_c(p) = sigma(p) . ahat_c."""
        g = {p: sum(sigma(p)[x] * self.ahat[x] for x in range(3)) for p in CUBE}
        rows = {}
        for p in CUBE:
            for p2 in CUBE:
                o = (p2[0] - p[0], p2[1] - p[1], p2[2] - p[2])
                contrib = -shift(g[p] * g[p2], -p[0], -p[1], -p[2])
                rows[o] = rows.get(o, 0.0) + contrib
        return rows

    def diag_A(self) -> np.ndarray:
        return self.row_entries()[(0, 0, 0)].reshape(-1)

    def gershgorin(self) -> np.ndarray:
        """|L_ii| + sum_{j != i} |L_ij| per cell, with L = diag(w) A."""
        rows = self.row_entries()
        tot = sum(np.abs(v) for v in rows.values())
        return (self.w3 * tot).reshape(-1)

    def dt_explicit(self) -> float:
        """dt_E = 2 / max_i Gershgorin_i, a bound below the forward-Euler stability limit."""
        return 2.0 / float(np.max(self.gershgorin()))

    def neighbors(self, idx: int):
        return grid_neighbors(self.shape, idx, 0, self.periodic)


def grid_neighbors(shape, idx: int, offset: int, periodic: bool = False):
    """The up-to-6 orthogonal neighbours of flat index idx (relative to `offset`) on a grid of
    `shape` = (n_p, n_t, n_r): phi wraps; r and theta wrap only on the periodic box."""
    n_p, n_t, n_r = shape
    loc = idx - offset
    k, rem = divmod(loc, n_t * n_r)
    j, i = divmod(rem, n_r)
    at = lambda kk, jj, ii: offset + (ii % n_r) + n_r * ((jj % n_t) + n_t * (kk % n_p))
    out = []
    if i > 0 or periodic:
        out.append(at(k, j, i - 1))
    if i < n_r - 1 or periodic:
        out.append(at(k, j, i + 1))
    if j > 0 or periodic:
        out.append(at(k, j - 1, i))
    if j < n_t - 1 or periodic:
        out.append(at(k, j + 1, i))
    out.append(at(k - 1, j, i))
    out.append(at(k + 1, j, i))
    return out
