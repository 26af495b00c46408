"""The PTL cycle loop with RKL2 / RKG2 stages and with Backward Euler + PC1 PCG, decomposed over
ranks by phi slabs: the plain form of the multi-processor algorithm that the paper's scaling runs
use (Sec. 3.2, Figs. 5-6: MAS on many CPU nodes or GPUs), written on the oracle's operators.  This
is test infrastructure like the rest of oracle/: it runs on CPU ranks (torch.distributed, gloo)
and its results are checked against the single-rank oracle.

Partitioning.  Rank p of P owns the phi planes [k0_p, k1_p) of every component (contiguous
slabs, the remainder spread over the first ranks); r and theta are never split, so a slab's
neighbours are the ranks holding the planes just below and above it (phi is periodic, so the
ranks form a ring).  Both stencils couple a point to points at most one plane away in phi: the
27-point conduction stencil through the corners k - 1/2 and k + 1/2, the 7-point viscosity
stencil through its +-phi faces.  A one-plane halo on each side -- whole planes, so it carries
the face, edge and corner neighbours of the slab alike -- therefore makes every owned point's F
exact; each rank evaluates the operator on its slab extended by the two halo planes, with the
coefficients of those planes, and keeps the owned planes.

Communication per cycle (Sec. 2 PTL, Sec. 3.1 schemes):
  * dt_E: a max-reduction of the local Gershgorin bounds (once per step);
  * the PTL: F on the owned planes, then a MAXLOC over ranks of (|F|, flat index) with the
    oracle's tie rule (the smallest flat index), the F halo exchanged so that the rank holding
    k sees all six neighbours, Eq. 5 evaluated there and a min-reduction hands dt_PTL to all;
  * STS: one halo exchange of the stage value per stage (the stencil's input), no reduction;
  * BE + PCG: one halo exchange per product S p, and sum-reductions for <r, z>, <p, q>, <r, r>
    (and <b, b> once per solve) -- the global communications Sec. 3.1 names as what limits
    the scaling of PCG.
Every reduction that decides something exactly (the max, the MAXLOC, the min) gives the same
value on every rank as the single-rank oracle; the STS arithmetic per point is the oracle's, so
a decomposed STS + PTL run equals the single-rank one exactly.  PCG sums its dot products in
another order, so its iterates agree to rounding.
"""
from __future__ import annotations

import math

import numpy as np

from .advance import CycleLog
from .pcg import PCGResult
from .sts import SCHEMES, TIE, sts_step
from .tc import TCOperator
from .visc import ViscOperator


def slab(n_phi: int, rank: int, world: int) -> tuple[int, int]:
    """Planes [k0, k1) owned by rank: n_phi // world each, the first n_phi % world ranks one more."""
    base, extra = divmod(n_phi, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


class SlabOperator:
    """One rank's part of a global oracle operator: the operator on its slab extended by a halo
    plane on each side, the exchange of halos with the neighbouring ranks and the reductions."""

    def __init__(self, op, rank: int, world: int, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.op, self.rank, self.world = op, rank, world
        self.n_phi = op.shapes[0][0]
        if self.n_phi < world:
            raise ValueError("every rank needs at least one phi plane")
        self.k0, self.k1 = slab(self.n_phi, rank, world)
        self.nloc = self.k1 - self.k0
        ext = [(self.k0 - 1 + m) % self.n_phi for m in range(self.nloc + 2)]
        if isinstance(op, TCOperator):
            self.local = TCOperator(op.ahat[:, ext], op.w3[ext], periodic=op.periodic)
        else:
            self.local = ViscOperator([tuple(a[ext] for a in c) for c in op.c], [w[ext] for w in op.w_list],
                                      periodic=op.periodic)
        self.shapes = op.shapes
        self.offsets = getattr(op, "offsets", [0, op.n])
        # flat global indices of the owned points, in local (component, plane, theta, r) order
        idx = []
        for c, shp in enumerate(self.shapes):
            plane = shp[1] * shp[2]
            idx.append(self.offsets[c] + np.arange(self.k0 * plane, self.k1 * plane))
        self.owned = np.concatenate(idx)
        self.w = op.w[self.owned]

    # -- layout ----------------------------------------------------------------------------------
    def split(self, flat_owned: np.ndarray):
        """Owned flat vector -> per-component arrays (nloc, n_t, n_r)."""
        out, at = [], 0
        for shp in self.shapes:
            n = self.nloc * shp[1] * shp[2]
            out.append(flat_owned[at:at + n].reshape(self.nloc, shp[1], shp[2]))
            at += n
        return out

    def take(self, global_vec: np.ndarray) -> np.ndarray:
        return np.array(global_vec[self.owned], dtype=np.float64)

    # -- communication ---------------------------------------------------------------------------
    def halo(self, flat_owned: np.ndarray):
        """The owned state extended by one plane below and one above (from the ring neighbours),
        per component, flattened in the local operator's layout."""
        import torch
        parts = self.split(flat_owned)
        lo_send = [np.ascontiguousarray(a[0]) for a in parts]      # my first plane -> rank below
        hi_send = [np.ascontiguousarray(a[-1]) for a in parts]     # my last plane -> rank above
        if self.world == 1:
            lo_recv, hi_recv = hi_send, lo_send
        else:
            below, above = (self.rank - 1) % self.world, (self.rank + 1) % self.world
            lo_recv = [np.empty_like(a) for a in hi_send]
            hi_recv = [np.empty_like(a) for a in lo_send]
            reqs = []
            for c in range(len(parts)):
                # tag 2c: a plane travelling up (it becomes the receiver's lower halo), 2c + 1: down
                reqs.append(self.dist.isend(torch.from_numpy(hi_send[c]), above, group=self.group, tag=2 * c))
                reqs.append(self.dist.isend(torch.from_numpy(lo_send[c]), below, group=self.group, tag=2 * c + 1))
                reqs.append(self.dist.irecv(torch.from_numpy(lo_recv[c]), below, group=self.group, tag=2 * c))
                reqs.append(self.dist.irecv(torch.from_numpy(hi_recv[c]), above, group=self.group, tag=2 * c + 1))
            for r in reqs:
                r.wait()
        ext = [np.concatenate([lo[None], a, hi[None]]) for lo, a, hi in zip(lo_recv, parts, hi_recv)]
        return np.concatenate([e.reshape(-1) for e in ext])

    def _owned_of_ext(self, ext_flat: np.ndarray) -> np.ndarray:
        out, at = [], 0
        for shp in self.shapes:
            n = (self.nloc + 2) * shp[1] * shp[2]
            out.append(ext_flat[at:at + n].reshape(self.nloc + 2, shp[1], shp[2])[1:-1].reshape(-1))
            at += n
        return np.concatenate(out)

    def allreduce(self, x: float, op: str) -> float:
        import torch
        if self.world == 1:
            return float(x)
        t = torch.tensor([x], dtype=torch.float64)
        self.dist.all_reduce(t, op={"sum": self.dist.ReduceOp.SUM, "max": self.dist.ReduceOp.MAX,
                                    "min": self.dist.ReduceOp.MIN}[op], group=self.group)
        return float(t.item())

    def dot(self, a: np.ndarray, b: np.ndarray) -> float:
        return self.allreduce(float(a @ b), "sum")

    # -- operator --------------------------------------------------------------------------------
    def apply(self, u_owned: np.ndarray) -> np.ndarray:
        return self._owned_of_ext(self.local.apply(self.halo(u_owned)))

    def apply_A(self, u_owned: np.ndarray) -> np.ndarray:
        return self._owned_of_ext(self.local.apply_A(self.halo(u_owned)))

    def diag_A(self) -> np.ndarray:
        return self._owned_of_ext(self.local.diag_A())

    def dt_explicit(self) -> float:
        return 2.0 / self.allreduce(float(np.max(self._owned_of_ext(self.local.gershgorin()))), "max")

    def ptl(self, u_owned: np.ndarray, F_owned: np.ndarray):
        """Eq. 5 at k = argmax |F| over all ranks (ties: the smallest flat index)."""
        import torch
        a = np.abs(F_owned)
        m = int(np.argmax(a))
        cand = torch.tensor([float(a[m]), float(self.owned[m])], dtype=torch.float64)
        if self.world > 1:
            everyone = [torch.empty(2, dtype=torch.float64) for _ in range(self.world)]
            self.dist.all_gather(everyone, cand, group=self.group)
        else:
            everyone = [cand]
        best_v = max(float(t[0]) for t in everyone)
        k = min(int(t[1]) for t in everyone if float(t[0]) == best_v)
        # the F halo, so that the rank holding k sees its phi neighbours
        u_ext, F_ext = self.halo(u_owned), self.halo(F_owned)
        dtp = math.inf
        pos = np.searchsorted(self.owned, k)
        if pos < self.owned.size and self.owned[pos] == k:
            loc = self._ext_index(k)
            uk, fk = u_ext[loc], F_ext[loc]
            for j in self.op.neighbors(k):
                lj = self._ext_index(j)
                du, dF = uk - u_ext[lj], fk - F_ext[lj]
                if du != 0.0 and dF != 0.0 and du * dF < 0.0:
                    dtp = min(dtp, -du / dF)
        return self.allreduce(dtp, "min"), k, best_v

    def _ext_index(self, g: int) -> int:
        """Position of global flat index g (an owned point or a halo neighbour) in the extended
        local layout."""
        c = int(np.searchsorted(self.offsets, g, side="right") - 1)
        shp = self.shapes[c]
        plane = shp[1] * shp[2]
        kk, rem = divmod(g - self.offsets[c], plane)
        m = (kk - (self.k0 - 1)) % self.n_phi
        base = sum((self.nloc + 2) * s[1] * s[2] for s in self.shapes[:c])
        return base + m * plane + rem

    def gather(self, u_owned: np.ndarray) -> np.ndarray:
        """The global vector, assembled on every rank."""
        import torch
        if self.world == 1:
            out = np.empty(self.op.n)
            out[self.owned] = u_owned
            return out
        n = max(slab(self.n_phi, r, self.world)[1] - slab(self.n_phi, r, self.world)[0] for r in range(self.world))
        per_plane = sum(s[1] * s[2] for s in self.shapes)
        buf = np.zeros(n * per_plane)
        buf[:u_owned.size] = u_owned
        parts = [torch.empty(buf.size, dtype=torch.float64) for _ in range(self.world)]
        self.dist.all_gather(parts, torch.from_numpy(buf), group=self.group)
        out = np.empty(self.op.n)
        for r in range(self.world):
            other = SlabIndex(self, r)
            out[other.owned] = parts[r].numpy()[:other.owned.size]
        return out


class SlabIndex:
    """The flat global indices owned by another rank (for assembling gathered vectors)."""

    def __init__(self, so: SlabOperator, rank: int):
        k0, k1 = slab(so.n_phi, rank, so.world)
        idx = []
        for c, shp in enumerate(so.shapes):
            plane = shp[1] * shp[2]
            idx.append(so.offsets[c] + np.arange(k0 * plane, k1 * plane))
        self.owned = np.concatenate(idx)


def _cycles(so: SlabOperator, u, dt, use_ptl, forced, max_cycles, floor, log):
    """The PTL cycle loop of oracle.advance on the slab: yields (dt_c, F(u)) and receives u."""
    t_rem, c = dt, 0
    dtE = so.dt_explicit()
    while True:
        if forced is not None:
            if c >= len(forced):
                return
            dt_c, dtp, k = float(forced[c]), math.nan, -1
            F = so.apply(u)
        else:
            if not t_rem > 1e-12 * dt:
                return
            if c >= max_cycles:
                raise RuntimeError(f"more than {max_cycles} cycles")
            F = so.apply(u)
            if use_ptl:
                dtp, k, _ = so.ptl(u, F)
                dtl = max(dtp, floor * dtE)
                q = t_rem / dtl * TIE
                n = 1.0 if q <= 1.0 else math.ceil(q)
                dt_c = t_rem / n
            else:
                dt_c, dtp, k = t_rem, math.nan, -1
        u = yield dt_c, F
        t_rem -= dt_c
        log.dt_c.append(dt_c)
        log.dt_ptl.append(dtp)
        log.k.append(k)
        c += 1


def sts_advance(so: SlabOperator, u_owned, dt: float, scheme: str = "rkl2", use_ptl: bool = True,
                forced=None, max_cycles: int = 100000, floor: float = 1.0):
    """oracle.advance.sts_advance on the slab: returns (owned u_new, CycleLog)."""
    stages, coeffs = SCHEMES[scheme]
    dtE = so.dt_explicit()
    u = np.array(u_owned, dtype=np.float64, copy=True)
    log = CycleLog()
    gen = _cycles(so, u, dt, use_ptl, forced, max_cycles, floor, log)
    try:
        dt_c, y0 = next(gen)
        while True:
            s = stages(dt_c / dtE)
            u = sts_step(so.apply, u, y0, dt_c, coeffs(s))
            log.s.append(s)
            dt_c, y0 = gen.send(u)
    except StopIteration:
        pass
    return u, log


def pcg(so: SlabOperator, apply_S, b, x0, Dinv, rtol: float, max_iter: int, fixed_iters: int = 0) -> PCGResult:
    """oracle.pcg.pcg with the dot products summed over ranks."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_S(x)
    bb = so.dot(b, b)
    tol2 = rtol * rtol * bb
    rr = so.dot(r, r)
    z = Dinv * r
    p = z.copy()
    rz = so.dot(r, z)
    it = 0
    limit = fixed_iters if fixed_iters > 0 else max_iter
    converged = fixed_iters == 0 and rr <= tol2
    while it < limit and not converged:
        q = apply_S(p)
        alpha = rz / so.dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rr = so.dot(r, r)
        if fixed_iters == 0 and rr <= tol2:
            converged = True
            break
        z = Dinv * r
        rz_new = so.dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    if fixed_iters > 0:
        converged = True
    res = b - apply_S(x)
    true_res = math.sqrt(so.dot(res, res) / bb) if bb > 0 else 0.0
    return PCGResult(x, it, converged, math.sqrt(rr / bb) if bb > 0 else 0.0, true_res)


def be_advance(so: SlabOperator, u_owned, dt: float, use_ptl: bool = True, rtol: float = 1e-10,
               max_iter: int = 100000, forced=None, max_cycles: int = 100000, fixed_iters: int = 0,
               floor: float = 1.0):
    """oracle.advance.be_advance on the slab: returns (owned u_new, CycleLog)."""
    u = np.array(u_owned, dtype=np.float64, copy=True)
    log = CycleLog()
    M = 1.0 / so.w
    dA = so.diag_A()
    gen = _cycles(so, u, dt, use_ptl, forced, max_cycles, floor, log)
    try:
        dt_c, _ = next(gen)
        while True:
            Dinv = 1.0 / (M - dt_c * dA)
            res = pcg(so, lambda v: M * v - dt_c * so.apply_A(v), M * u, u, Dinv, rtol, max_iter, fixed_iters)
            u = res.x
            log.iters.append(res.iters)
            log.true_res.append(res.true_rel_residual)
            dt_c, _ = gen.send(u)
    except StopIteration:
        pass
    return u, log
