"""Spherical shell geometry (Sec. 3.2 uses a highly non-uniform (r, theta, phi) grid; the paper
gives no discretisation, so the finite-volume reading below is the one this project fixes).

Fields are arrays of shape (n_phi, n_theta, n_r), index [k, j, i].  Cell (i, j, k) spans
[r_face[i], r_face[i+1]] x [t_face[j], t_face[j+1]] x [k dphi, (k+1) dphi].  Corner [k, j, i]
is the grid vertex (i+1/2, j+1/2, k+1/2) in cell-index units, i.e. (r_face[i+1], t_face[j+1],
(k+1) dphi); it touches the eight cells i..i+1, j..j+1, k..k+1 (k+1 taken modulo n_phi).
"""
from __future__ import annotations

import numpy as np


def centres(faces: np.ndarray) -> np.ndarray:
    return 0.5 * (faces[:-1] + faces[1:])


class Shell:
    """`dphi` defaults to 2 pi / n_phi; an explicit value describes a phi window of a larger grid
    (the window is then closed periodically, which only changes points near its phi ends)."""

    def __init__(self, r_face, t_face, n_phi: int, dphi: float | None = None):
        self.r_face = np.asarray(r_face, dtype=np.float64)
        self.t_face = np.asarray(t_face, dtype=np.float64)
        self.n_r = len(self.r_face) - 1
        self.n_t = len(self.t_face) - 1
        self.n_p = int(n_phi)
        if self.n_r < 2 or self.n_t < 2 or self.n_p < 3:
            raise ValueError("need n_r >= 2, n_theta >= 2, n_phi >= 3")
        self.r_c = centres(self.r_face)
        self.t_c = centres(self.t_face)
        self.dphi = 2.0 * np.pi / self.n_p if dphi is None else float(dphi)
        self.shape = (self.n_p, self.n_t, self.n_r)

    def cell_volume(self) -> np.ndarray:
        """V = (r+^3 - r-^3)/3 * (cos t- - cos t+) * dphi, broadcast to the field shape."""
        dr3 = (self.r_face[1:] ** 3 - self.r_face[:-1] ** 3) / 3.0
        dcos = np.cos(self.t_face[:-1]) - np.cos(self.t_face[1:])
        v2 = dcos[:, None] * dr3[None, :] * self.dphi
        return np.broadcast_to(v2[None, :, :], self.shape).copy()

    def corner_metric(self):
        """Metric factors h_r, h_theta, h_phi and dual (corner) volume W at every corner.

        For the corner at (r_face[i+1], t_face[j+1]):
            h_r = 1 / (r_c[i+1] - r_c[i])
            h_t = 1 / (r_face[i+1] (t_c[j+1] - t_c[j]))
            h_p = 1 / (r_face[i+1] sin(t_face[j+1]) dphi)
            W   = r_face[i+1]^2 (r_c[i+1] - r_c[i]) sin(t_face[j+1]) (t_c[j+1] - t_c[j]) dphi
        Only corners with i <= n_r - 2 and j <= n_theta - 2 are interior; the others are returned
        as zero and carry no flux (zero-flux boundaries at r_min, r_max and the poles).
        Returns four arrays of shape (n_theta, n_r) (independent of phi).
        """
        nr, nt = self.n_r, self.n_t
        hr = np.zeros((nt, nr)); ht = np.zeros((nt, nr)); hp = np.zeros((nt, nr)); W = np.zeros((nt, nr))
        drc = self.r_c[1:] - self.r_c[:-1]           # (nr-1,)
        dtc = self.t_c[1:] - self.t_c[:-1]           # (nt-1,)
        rf = self.r_face[1:nr]                        # interior r faces
        tf = self.t_face[1:nt]                        # interior theta faces
        hr[:nt - 1, :nr - 1] = (1.0 / drc)[None, :]
        ht[:nt - 1, :nr - 1] = 1.0 / (rf[None, :] * dtc[:, None])
        hp[:nt - 1, :nr - 1] = 1.0 / (rf[None, :] * np.sin(tf)[:, None] * self.dphi)
        W[:nt - 1, :nr - 1] = (rf ** 2 * drc)[None, :] * (np.sin(tf) * dtc)[:, None] * self.dphi
        return hr, ht, hp, W


def shift(a: np.ndarray, dk: int, dj: int, di: int) -> np.ndarray:
    """Periodic shift: shift(a, dk, dj, di)[k, j, i] == a[k+dk, j+dj, i+di] (indices wrap)."""
    return np.roll(a, (-dk, -dj, -di), axis=(0, 1, 2))


CUBE = [(pk, pj, pi) for pk in (0, 1) for pj in (0, 1) for pi in (0, 1)]
