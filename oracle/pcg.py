"""Backward Euler solved by point-Jacobi preconditioned conjugate gradients (Sec. 3.1, PC1).

BE over a cycle of length dt: (I - dt L) x = u^n with L = diag(w) A.  Multiplying by
M = diag(1/w) gives the symmetric positive definite system

    S x = b,   S = M - dt A,   b = M u^n,

solved by CG preconditioned with D = diag(S) = 1/w - dt diag(A).  The iteration is the textbook
PCG recurrence; the stopping test is ||r||_2 <= rtol ||b||_2 on the recursively updated residual,
written as r.r <= rtol^2 b.b, and the true residual ||b - S x|| / ||b|| is reported at exit.
`fixed_iters` > 0 runs exactly that many iterations with no stopping test.

A stronger preconditioner (Sec. 3.1 calls the one MAS uses PC2, an incomplete factorisation):
the project's GPU substitute is polynomial, z = p(D^-1 S) D^-1 r, the degree-m Chebyshev
acceleration of point-Jacobi on an interval [a, b] holding the spectrum of D^-1 S (the classical
Chebyshev semi-iteration, written out in `chebyshev`).  Its residual polynomial is
1 - lambda p(lambda) = T_m((theta - lambda)/delta) / T_m(theta/delta), theta = (a+b)/2,
delta = (b-a)/2.  The interval is b = 1.05 max_i (M_i + dt sum_j |A_ij|)/(M_i - dt A_ii) (the
Gershgorin bound of D^-1 S) and a = b/30.
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


def chebyshev(apply_S, Dinv, a: float, b: float, m: int):
    """z = p(D^-1 S) D^-1 r: m - 1 steps of the Chebyshev semi-iteration for S y = r from y_0 = 0
    with the point-Jacobi splitting, the spectrum of D^-1 S assumed in [a, b]."""
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta

    def apply(r):
        y_prev = np.zeros_like(r)
        y = Dinv * r / theta
        rho_prev = 1.0 / sigma
        for _ in range(1, m):
            rho = 1.0 / (2.0 * sigma - rho_prev)
            y, y_prev = y + rho * rho_prev * (y - y_prev) + (2.0 * rho / delta) * (Dinv * (r - apply_S(y))), y
            rho_prev = rho
        return y
    return apply


def pcg(apply_S, b, x0, Dinv, rtol: float, max_iter: int, fixed_iters: int = 0, precond=None) -> PCGResult:
    """precond(r) -> z; point-Jacobi (z = D^-1 r) when None."""
    prec = precond or (lambda r: Dinv * r)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_S(x)
    bb = float(b @ b)
    tol2 = rtol * rtol * bb
    rr = float(r @ r)
    z = prec(r)
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
        z = prec(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    if fixed_iters > 0:
        converged = True
    true_res = float(np.linalg.norm(b - apply_S(x)) / np.sqrt(bb)) if bb > 0 else 0.0
    rel = float(np.sqrt(rr / bb)) if bb > 0 else 0.0
    return PCGResult(x, it, converged, rel, true_res)


def chebyshev_bound(op, dt: float) -> float:
    """Gershgorin bound of the spectrum of D^-1 S: max_i (M_i + dt sum_j |A_ij|) / (M_i - dt A_ii)."""
    M = 1.0 / op.w
    rowabs = op.gershgorin() / op.w          # sum_j |A_ij| (gershgorin() is that of L = diag(w) A)
    return float(np.max((M + dt * rowabs) / (M - dt * op.diag_A())))


def be_solve(op, u: np.ndarray, dt: float, rtol: float, max_iter: int, x0=None,
             fixed_iters: int = 0, precond: str = "jacobi", degree: int = 3) -> PCGResult:
    """One Backward Euler step of size dt for operator op from state u."""
    M = 1.0 / op.w
    dA = op.diag_A()
    Dinv = 1.0 / (M - dt * dA)
    apply_S = lambda v: M * v - dt * op.apply_A(v)
    b = M * u
    x0 = u if x0 is None else x0
    prec = None
    if precond == "chebyshev":
        hi = 1.05 * chebyshev_bound(op, dt)
        prec = chebyshev(apply_S, Dinv, hi / 30.0, hi, degree)
    return pcg(apply_S, b, x0, Dinv, rtol, max_iter, fixed_iters, prec)
