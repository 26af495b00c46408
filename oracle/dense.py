"""Dense tiny-grid truth: the operator as an explicit matrix, built column by column by applying
it to unit vectors, and exact functions of it through the symmetric similarity transform
M^{1/2} L M^{-1/2} = M^{-1/2} A M^{-1/2} (M = diag(1/w), A = M L symmetric)."""
from __future__ import annotations

import numpy as np


def dense_matrix(apply, n: int) -> np.ndarray:
    Lm = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        Lm[:, j] = apply(e)
        e[j] = 0.0
    return Lm


def symmetric_eig(op):
    """Eigen-decomposition of the symmetrised operator: returns (lam, Q, sqrtM) with
    L = M^{-1/2} Q diag(lam) Q^T M^{1/2}."""
    A = dense_matrix(op.apply_A, op.n)
    A = 0.5 * (A + A.T)
    sm = np.sqrt(1.0 / op.w)
    Ls = A / sm[:, None] / sm[None, :]
    lam, Q = np.linalg.eigh(Ls)
    return lam, Q, sm


def apply_function(op, f, u: np.ndarray, eig=None) -> np.ndarray:
    """f(L) u through the eigen-decomposition; f acts elementwise on the eigenvalues."""
    lam, Q, sm = eig if eig is not None else symmetric_eig(op)
    return (Q @ (f(lam) * (Q.T @ (sm * u)))) / sm
