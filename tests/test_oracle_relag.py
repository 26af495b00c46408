"""Pins of the oracle's non-linear conduction (the diffusivity re-lagged every cycle,
oracle.advance.sts_advance_relag), against facts that do not come from the function itself:

* the energy sum_i u_i / w_i is conserved exactly: w = C/(n V) does not depend on kappa, and every
  cycle's operator conserves it (zero-flux boundaries), so the re-lag must too;
* as the cycles shrink, the result converges to the solution of the non-linear ODE
  dT/dt = C/n div(kappa(T) b b . grad T) computed by brute force (forward Euler with kappa
  re-evaluated at every tiny step), at first order in the cycle length (the lag);
* one cycle is the frozen-kappa super step with kappa taken from the initial state;
* at the workload ratio (100 dt_E, 5 % noise) the re-lagged run stays finite and positive,
  where re-evaluating kappa at every stage does not."""
import numpy as np
import pytest

import synth
from oracle.advance import sts_advance, sts_advance_relag
from oracle.geometry import Shell
from oracle.tc import TCOperator


def _problem(shape=(12, 10, 8), noise=0.05, seed=5):
    g = synth.make_grid(*shape, 1.05)
    inp = synth.tc_inputs(g, seed, noise=noise)
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    build = lambda T0: TCOperator.spherical(sh, np.reshape(T0, g.shape), inp.n, inp.B)
    return build, inp.T.reshape(-1).copy()


def test_relag_conserves_energy():
    build, u = _problem()
    w = build(u).w                        # C / (n V): independent of kappa
    dt = 100.0 * build(u).dt_explicit()
    x, log, _ = sts_advance_relag(build, u, dt)
    assert log.cycles > 3
    assert np.sum(x / w) == pytest.approx(np.sum(u / w), rel=1e-13)


def test_relag_converges_to_the_nonlinear_ode():
    build, u = _problem(shape=(6, 6, 6), noise=0.1)
    dt = 5.0 * build(u).dt_explicit()
    # brute force: forward Euler on the non-linear ODE, kappa(T) re-evaluated every step
    ref = u.copy()
    n_ref = 4000
    for _ in range(n_ref):
        ref = ref + (dt / n_ref) * build(np.maximum(ref, 0.0)).apply(ref)
    errs = []
    for n in (5, 20, 80):
        x, log, _ = sts_advance_relag(build, u, dt, forced=[dt / n] * n)
        errs.append(np.linalg.norm(x - ref) / np.linalg.norm(ref - u))
    assert errs[0] > errs[1] > errs[2]
    # first order in the lag: four times shorter cycles, about four times smaller error
    assert errs[2] < 0.4 * errs[1] and errs[1] < 0.4 * errs[0]
    assert errs[2] < 2e-2


def test_one_relag_cycle_is_the_frozen_super_step():
    build, u = _problem()
    dt = 30.0 * build(u).dt_explicit()
    x, log, _ = sts_advance_relag(build, u, dt, use_ptl=False)
    y, log2 = sts_advance(build(u), u, dt, use_ptl=False)
    assert log.s == log2.s
    np.testing.assert_array_equal(x, y)


def test_relag_stays_bounded_where_per_stage_kappa_does_not():
    build, u = _problem()
    dt = 100.0 * build(u).dt_explicit()
    x, log, _ = sts_advance_relag(build, u, dt)
    assert np.isfinite(x).all() and x.min() > 0.0
