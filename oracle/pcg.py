"""Backward Euler solved by point-Jacobi preconditioned conjugate gradients (Sec. 3.1, PC1).

BE over a cycle of length dt: (I - dt L) x = u^n with L = diag(w) A.  Multiplying by
M = diag(1/w) gives the symmetric positive definite system

    S x = b,   S = M - dt A,   b = M u^n,

solved by CG preconditioned with D = diag(S) = 1/w - dt diag(A).  The iteration is the textbook
PCG recurrence; the stopping test is ||r||_2 <= rtol ||b||_2 on the recursively updated residual,
written as r.r <= rtol^2 b.b, and the true residual ||b - S x|| / ||b|| is reported at exit.
`fixed_iters` > 0 runs exactly that many iterations with no stopping test.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    converged: bool
    rel_residual: float       # recursive residual norm / ||b||
    true_rel_residual: float  # ||b - S x|| / ||b||


def pcg(apply_S, b, x0, Dinv, rtol: float, max_iter: int, fixed_iters: int = 0) -> PCGResult:
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_S(x)
    bb = float(b @ b)
    tol2 = rtol * rtol * bb
    rr = float(r @ r)
    z = Dinv * r
    p = z.copy()
    rz = float(r @ z)
    it = 0
    limit = fixed_iters if fixed_iters > 0 else max_iter
    converged = fixed_iters == 0 and rr <= tol2
    while it < limit and not converged:
        q = apply_S(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rr = float(r @ r)
        if fixed_iters == 0 and rr <= tol2:
            converged = True
            break
        z = Dinv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    if fixed_iters > 0:
        converged = True
    true_res = float(np.linalg.norm(b - apply_S(x)) / np.sqrt(bb)) if bb > 0 else 0.0
    rel = float(np.sqrt(rr / bb)) if bb > 0 else 0.0
    return PCGResult(x, it, converged, rel, true_res)


def be_solve(op, u: np.ndarray, dt: float, rtol: float, max_iter: int, x0=None,
             fixed_iters: int = 0) -> PCGResult:
    """One Backward Euler step of size dt for operator op from state u."""
    M = 1.0 / op.w
    dA = op.diag_A()
    Dinv = 1.0 / (M - dt * dA)
    apply_S = lambda v: M * v - dt * op.apply_A(v)
    b = M * u
    x0 = u if x0 is None else x0
    return pcg(apply_S, b, x0, Dinv, rtol, max_iter, fixed_iters)
