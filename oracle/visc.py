"""Artificial kinematic viscosity, Eq. 2 (left):  F_visc(v) = (1/rho) div( nu rho grad v ).

Reading fixed by the project (the paper is silent on the vector-Laplacian coupling): each velocity
component is diffused as a scalar on its own staggered grid -- v_r on the interior r faces, v_theta
on the interior theta faces, v_phi on the phi faces (periodic) -- with the isotropic 7-point
finite-volume flux form

    F_i = 1/(rho_i V_i) * sum over faces f of c_f (u_nbr - u_i),   c_f = A_f nu_f rho_f / d_f,

nu_f, rho_f the arithmetic means of the two points sharing face f, zero flux at the ends of the r
and theta index ranges.  The curvature coupling terms of the spherical vector Laplacian are
omitted, as Eq. 2 is written.  The three components form one operator: their state vectors are
concatenated (v_r, v_theta, v_phi), each flattened with r fastest.
"""
from __future__ import annotations

import numpy as np

from .geometry import Shell, shift
from .tc import grid_neighbors

AXES = ((0, 0, 1), (0, 1, 0), (1, 0, 0))   # shift vectors for the r, theta, phi directions


def staggered_axes(shell: Shell, comp: int):
    """Point coordinates and control-volume bounds along r, theta, phi for component comp."""
    if comp == 0:
        pr, er = shell.r_face[1:shell.n_r], shell.r_c
    else:
        pr, er = shell.r_c, shell.r_face
    if comp == 1:
        pt, et = shell.t_face[1:shell.n_t], shell.t_c
    else:
        pt, et = shell.t_c, shell.t_face
    d = shell.dphi
    if comp == 2:
        pp = d * np.arange(shell.n_p)
    else:
        pp = d * (np.arange(shell.n_p) + 0.5)
    return (pr, er), (pt, et), pp


class ViscOperator:
    ncomp = 3

    def __init__(self, c_list, w_list, periodic: bool = False):
        """c_list[comp] = (c_r, c_t, c_p): coefficient of the face between a point and its +1
        neighbour along each axis (zero on the last r / theta point unless periodic);
        w_list[comp] = 1/(rho V).  periodic: r and theta wrap as phi does (the box)."""
        self.periodic = periodic
        self.c = [tuple(np.asarray(a, dtype=np.float64) for a in c) for c in c_list]
        self.w_list = [np.asarray(w, dtype=np.float64) for w in w_list]
        self.shapes = [w.shape for w in self.w_list]
        self.sizes = [w.size for w in self.w_list]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(int)
        self.n = int(self.offsets[-1])
        self.w = np.concatenate([w.reshape(-1) for w in self.w_list])

    @classmethod
    def spherical(cls, shell: Shell, rho_list, nu_list):
        c_list, w_list = [], []
        for comp in range(3):
            (pr, er), (pt, et), pp = staggered_axes(shell, comp)
            rho = np.asarray(rho_list[comp], dtype=np.float64)
            nu = np.asarray(nu_list[comp], dtype=np.float64)
            shp = (len(pp), len(pt), len(pr))
            assert rho.shape == shp and nu.shape == shp, (rho.shape, shp)
            d = shell.dphi
            dr3 = (er[1:] ** 3 - er[:-1] ** 3) / 3.0
            dr2 = (er[1:] ** 2 - er[:-1] ** 2) / 2.0
            dcos = np.cos(et[:-1]) - np.cos(et[1:])
            dth = et[1:] - et[:-1]
            V = np.broadcast_to((dcos[:, None] * dr3[None, :] * d)[None], shp)
            face = lambda a, ax: 0.5 * (a + shift(a, *AXES[ax]))
            nr, nt = shp[2], shp[1]
            # r faces between points i and i+1, at er[i+1]
            cr = np.zeros(shp)
            Ar = er[1:-1][None, :] ** 2 * dcos[:, None] * d            # (nt, nr-1)
            dr = (pr[1:] - pr[:-1])[None, :]
            cr[:, :, :nr - 1] = (Ar / dr)[None] * (face(nu, 0) * face(rho, 0))[:, :, :nr - 1]
            # theta faces between points j and j+1, at et[j+1]
            ct = np.zeros(shp)
            At = dr2[None, :] * np.sin(et[1:-1])[:, None] * d          # (nt-1, nr)
            dt = pr[None, :] * (pt[1:] - pt[:-1])[:, None]
            ct[:, :nt - 1, :] = (At / dt)[None] * (face(nu, 1) * face(rho, 1))[:, :nt - 1, :]
            # phi faces between points k and k+1 (periodic)
            Ap = dr2[None, :] * dth[:, None]                           # (nt, nr)
            dp = pr[None, :] * np.sin(pt)[:, None] * d
            cp = (Ap / dp)[None] * face(nu, 2) * face(rho, 2)
            c_list.append((cr, ct, cp))
            w_list.append(1.0 / (rho * V))
        return cls(c_list, w_list)

    @classmethod
    def box(cls, rho_list, nu_list):
        """Periodic box of unit cells: every component on the full (n_p, n_t, n_r) grid,
        c_f = nu_f rho_f (face means, wrapping; A_f = d_f = 1) and w = 1/rho."""
        c_list, w_list = [], []
        for comp in range(3):
            rho = np.asarray(rho_list[comp], dtype=np.float64)
            nu = np.asarray(nu_list[comp], dtype=np.float64)
            c = []
            for ax in range(3):
                c.append(0.5 * (nu + shift(nu, *AXES[ax])) * (0.5 * (rho + shift(rho, *AXES[ax]))))
            c_list.append(tuple(c))
            w_list.append(1.0 / rho)
        return cls(c_list, w_list, periodic=True)

    def split(self, u):
        u = np.asarray(u, dtype=np.float64)
        return [u[self.offsets[c]:self.offsets[c + 1]].reshape(self.shapes[c]) for c in range(3)]

    def apply_A(self, u):
        out = []
        for comp, uc in enumerate(self.split(u)):
            acc = np.zeros(self.shapes[comp])
            for ax in range(3):
                cplus = self.c[comp][ax]
                up = shift(uc, *AXES[ax])
                um = shift(uc, *[-a for a in AXES[ax]])
                cminus = shift(cplus, *[-a for a in AXES[ax]])
                acc += cplus * (up - uc) + cminus * (um - uc)
            out.append(acc.reshape(-1))
        return np.concatenate(out)

    def apply(self, u):
        return self.w * self.apply_A(u)

    def face_sum(self):
        out = []
        for comp in range(3):
            tot = 0.0
            for ax in range(3):
                cplus = self.c[comp][ax]
                tot = tot + cplus + shift(cplus, *[-a for a in AXES[ax]])
            out.append(np.asarray(tot).reshape(-1))
        return np.concatenate(out)

    def diag_A(self):
        return -self.face_sum()

    def gershgorin(self):
        return 2.0 * self.w * self.face_sum()

    def dt_explicit(self) -> float:
        return 2.0 / float(np.max(self.gershgorin()))

    def neighbors(self, idx: int):
        comp = int(np.searchsorted(self.offsets, idx, side="right") - 1)
        return grid_neighbors(self.shapes[comp], idx, int(self.offsets[comp]), self.periodic)
