"""The dynamic PTL cycle loop (Sec. 2, last paragraph; Sec. 1): the operator is advanced over the
full step dt in cycles, the PTL being re-evaluated from the current state before every cycle.

Reading fixed by the project (the paper gives no formula for the cycle length): with t_rem the
time still to cover and the limit floored at the explicit step, dt_L = max(dt_PTL, floor dt_E),
n = ceil(t_rem / dt_L) (n = 1 when dt_L >= t_rem), the next cycle has length dt_c = t_rem / n,
and the loop stops once t_rem <= 1e-12 dt.  As for the stage counts, a quotient t_rem / dt_L
within 1e-12 (relative) of an integer takes the smaller n, so that the cycle count is not
decided by the last bit of dt_E when dt is a whole multiple of it.  The floor (default 1, in units of dt_E) keeps the
loop from cycling more finely than the explicit stability limit, which Sec. 2 names as the costly
extreme the PTL is meant to improve on: taken literally, a cycle of length dt_PTL drives the
neighbour difference at k towards zero, so the next dt_PTL collapses and the loop need not end.
floor = 0 gives the literal rule.  Without the PTL the step is
one cycle of length dt.  A forced schedule (a list of cycle lengths) replaces the PTL decision;
it is used to compare runs whose PTL decisions are taken in different precisions.
ptl_mode="full" takes dt_PTL from the Eq. 4 condition over every pair of neighbours (ptl_full)
instead of the F_max localisation of Eq. 5; the cycle rule is the same.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .pcg import be_solve
from .ptl import ptl, ptl_full
from .sts import SCHEMES, TIE, sts_step


class MaxCyclesError(RuntimeError):
    pass


@dataclasses.dataclass
class CycleLog:
    dt_c: list = dataclasses.field(default_factory=list)
    s: list = dataclasses.field(default_factory=list)        # STS stages per cycle
    iters: list = dataclasses.field(default_factory=list)    # PCG iterations per cycle
    dt_ptl: list = dataclasses.field(default_factory=list)
    k: list = dataclasses.field(default_factory=list)
    true_res: list = dataclasses.field(default_factory=list)

    @property
    def cycles(self) -> int:
        return len(self.dt_c)


def _cycles(op, u, dt, use_ptl, forced, max_cycles, log, needs_F_always, floor, ptl_mode="fmax"):
    """Generator over cycles: yields (dt_c, F(u) or None) and receives the new state."""
    t_rem = dt
    c = 0
    dtE = op.dt_explicit() if (use_ptl and forced is None) else 0.0
    while True:
        if forced is not None:
            if c >= len(forced):
                return
            dt_c = float(forced[c])
            F = op.apply(u) if needs_F_always else None
            dtp, k = math.nan, -1
        else:
            if not t_rem > 1e-12 * dt:
                return
            if c >= max_cycles:
                raise MaxCyclesError(f"more than {max_cycles} cycles")
            F = op.apply(u) if (use_ptl or needs_F_always) else None
            if use_ptl:
                if ptl_mode == "full":
                    dtp, key = ptl_full(op, u, F)
                    k = key // 3 if key >= 0 else -1
                else:
                    dtp, k, _ = ptl(op, u, F)
                dtl = max(dtp, floor * dtE)
                q = t_rem / dtl * TIE
                n = 1.0 if q <= 1.0 else math.ceil(q)
                dt_c = t_rem / n
            else:
                dtp, k = math.nan, -1
                dt_c = t_rem
        u = yield dt_c, F
        t_rem -= dt_c
        log.dt_c.append(dt_c)
        log.dt_ptl.append(dtp)
        log.k.append(k)
        c += 1


def sts_advance(op, u, dt: float, scheme: str = "rkl2", use_ptl: bool = True, forced=None,
                max_cycles: int = 100000, floor: float = 1.0, ptl_mode: str = "fmax"):
    """Advance u over dt with RKL2 / RKG2 and PTL cycling.  Returns (u_new, CycleLog)."""
    stages, coeffs = SCHEMES[scheme]
    dtE = op.dt_explicit()
    u = np.array(u, dtype=np.float64, copy=True)
    log = CycleLog()
    gen = _cycles(op, u, dt, use_ptl, forced, max_cycles, log, True, floor, ptl_mode)
    try:
        dt_c, y0 = next(gen)
        while True:
            s = stages(dt_c / dtE)
            u = sts_step(op.apply, u, y0, dt_c, coeffs(s))
            log.s.append(s)
            dt_c, y0 = gen.send(u)
    except StopIteration:
        pass
    return u, log


def sts_advance_relag(build, u, dt: float, scheme: str = "rkl2", use_ptl: bool = True, forced=None,
                      max_cycles: int = 100000, floor: float = 1.0):
    """Non-linear conduction with the diffusivity re-lagged every cycle.  Sec. 3.1 notes that super
    time stepping can handle a non-linear operator, and Sec. 2 freezes kappa at a lagged
    temperature; reading fixed by the project: before every cycle the operator is rebuilt from
    the current state, build(T0) with T0 = max(u, 0) (kappa = T0^{5/2}; a state that undershoots
    zero gets no negative diffusivity), dt_E is re-evaluated from it, and the cycle -- its PTL
    decision and its s stages -- runs with that operator frozen.  The cycle rule is that of
    sts_advance.  Returns (u_new, CycleLog, dt_E of the last cycle's operator)."""
    stages, coeffs = SCHEMES[scheme]
    u = np.array(u, dtype=np.float64, copy=True)
    log = CycleLog()
    t_rem, c, dtE = dt, 0, math.nan
    while True:
        if forced is not None:
            if c >= len(forced):
                break
        elif not t_rem > 1e-12 * dt:
            break
        elif c >= max_cycles:
            raise MaxCyclesError(f"more than {max_cycles} cycles")
        op = build(np.maximum(u, 0.0))
        dtE = op.dt_explicit()
        F = op.apply(u)
        dtp, k = math.nan, -1
        if forced is not None:
            dt_c = float(forced[c])
        elif use_ptl:
            dtp, k, _ = ptl(op, u, F)
            dtl = max(dtp, floor * dtE)
            q = t_rem / dtl * TIE
            n = 1.0 if q <= 1.0 else math.ceil(q)
            dt_c = t_rem / n
        else:
            dt_c = t_rem
        s = stages(dt_c / dtE)
        u = sts_step(op.apply, u, F, dt_c, coeffs(s))
        log.dt_c.append(dt_c)
        log.s.append(s)
        log.dt_ptl.append(dtp)
        log.k.append(k)
        t_rem -= dt_c
        c += 1
    return u, log, dtE


def be_advance(op, u, dt: float, use_ptl: bool = True, rtol: float = 1e-10, max_iter: int = 100000,
               forced=None, max_cycles: int = 100000, fixed_iters: int = 0, floor: float = 1.0,
               ptl_mode: str = "fmax", precond: str = "jacobi", degree: int = 3):
    """Advance u over dt with Backward Euler + PCG (point-Jacobi, or the Chebyshev polynomial
    preconditioner of oracle.pcg) and PTL cycling."""
    u = np.array(u, dtype=np.float64, copy=True)
    log = CycleLog()
    gen = _cycles(op, u, dt, use_ptl, forced, max_cycles, log, False, floor, ptl_mode)
    try:
        dt_c, _ = next(gen)
        while True:
            res = be_solve(op, u, dt_c, rtol, max_iter, fixed_iters=fixed_iters, precond=precond, degree=degree)
            u = res.x
            log.iters.append(res.iters)
            log.true_res.append(res.true_rel_residual)
            dt_c, _ = gen.send(u)
    except StopIteration:
        pass
    return u, log
