"""Pins of the oracle's Chebyshev polynomial preconditioner (oracle/pcg.py `chebyshev`), the GPU
substitute for a stronger preconditioner than point-Jacobi (Sec. 3.1, PC2), against facts that do
not come from the function itself:

* on every eigenpair (lambda, v) of D^-1 S of a tiny Backward Euler system, P (S v) = (1 - R(lambda)) v
  with the Chebyshev residual polynomial R(lambda) = T_m((theta - lambda)/delta) / T_m(theta/delta)
  (numpy's Chebyshev series, not the three-term recurrence);
* P is symmetric positive definite (the matrix built column by column), as PCG needs;
* the Gershgorin value bounds the largest eigenvalue of D^-1 S;
* PCG with it reaches the dense direct solution, in fewer iterations than point-Jacobi."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from gpu_common import tc_problem, visc_problem
from oracle.dense import dense_matrix
from oracle.pcg import be_solve, chebyshev, chebyshev_bound


def _system(kind, ratio=200.0):
    g, inp, op, u = tc_problem(5, 4, 6, noise=0.1) if kind == "tc" else visc_problem(5, 4, 6)
    dt = ratio * op.dt_explicit()
    M = 1.0 / op.w
    apply_S = lambda v: M * v - dt * op.apply_A(v)
    S = dense_matrix(apply_S, op.n)
    return op, u, dt, M, apply_S, S


@pytest.mark.parametrize("kind", ["tc", "visc"])
@pytest.mark.parametrize("m", [2, 3, 5])
def test_chebyshev_residual_polynomial_on_eigenpairs(kind, m):
    op, u, dt, M, apply_S, S = _system(kind)
    d = np.diag(S)
    Dinv = 1.0 / d
    # D^-1 S is similar to the symmetric D^-1/2 S D^-1/2
    lam, W = np.linalg.eigh(S / np.sqrt(np.outer(d, d)))
    V = W / np.sqrt(d)[:, None]
    hi = 1.05 * chebyshev_bound(op, dt)
    lo = hi / 30.0
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    P = chebyshev(apply_S, Dinv, lo, hi, m)
    Tm = lambda x: npcheb.chebval(x, [0] * m + [1])
    for k in range(0, lam.size, max(1, lam.size // 12)):
        v = V[:, k]
        R = Tm((theta - lam[k]) / delta) / Tm(theta / delta)
        np.testing.assert_allclose(P(S @ v), (1.0 - R) * v, rtol=0, atol=1e-10 * np.abs(v).max())


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_chebyshev_preconditioner_is_spd_and_bound_holds(kind):
    op, u, dt, M, apply_S, S = _system(kind)
    d = np.diag(S)
    lam = np.linalg.eigvalsh(S / np.sqrt(np.outer(d, d)))
    bound = chebyshev_bound(op, dt)
    assert lam.max() <= bound * (1 + 1e-12)
    P = dense_matrix(chebyshev(apply_S, 1.0 / d, 1.05 * bound / 30.0, 1.05 * bound, 4), op.n)
    assert np.abs(P - P.T).max() <= 1e-12 * np.abs(P).max()
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0.0


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_chebyshev_pcg_reaches_the_direct_solution(kind):
    op, u, dt, M, apply_S, S = _system(kind, ratio=1e3)
    x_ref = np.linalg.solve(S, M * u)
    cond = np.linalg.cond(S)
    jac = be_solve(op, u, dt, 1e-12, 10000)
    for m in (2, 4):
        res = be_solve(op, u, dt, 1e-12, 10000, precond="chebyshev", degree=m)
        assert res.converged and res.true_rel_residual <= 1.01e-12
        # the error a relative residual allows: cond(S) times it
        assert np.linalg.norm(res.x - x_ref) <= cond * res.true_rel_residual * np.linalg.norm(x_ref)
        assert res.iters < jac.iters
