"""The library on the periodic box (PB_CARTESIAN_PERIODIC) against closed forms and the oracle.

On the box every Fourier mode is an eigenvector of both operators, so the GPU path is checked
against the mathematics directly: F = lambda u, one STS step R_s(dt lambda) u (RKL2 and RKG2,
Appendix A), one BE step u / (1 - dt lambda), the PTL 1/|lambda| (Eqs. 4-5).  The Fig. 1 set-up
-- the 1-D second-order heat equation at 500 explicit steps -- is the conduction box with the
field along phi and states constant in r and theta: one step from a delta plane carries every
mode, and its FFT along phi gives the amplification factor of each mode.  Random fields are
compared with the oracle's box operators."""
import math

import numpy as np
import pytest

from gpu_common import TOL, rel_l2, rel_max, to_dev, to_host
from oracle.advance import be_advance, sts_advance
from oracle.pcg import be_solve
from oracle.ptl import ptl, ptl_full
from oracle.sts import rkg2_stages, rkl2_stages
from oracle.tc import TCOperator
from oracle.visc import ViscOperator
from periodic import R_closed, mode, tc_symbol, visc_symbol

pytestmark = pytest.mark.gpu

STAGES = {"rkl2": rkl2_stages, "rkg2": rkg2_stages}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda")


def tc_box_problem(shape, prec, bhat=None, T0=1.0, n=1.0, C=1.0, seed=None):
    """Conduction on the box: constant T0, n and field direction bhat, or (seed) random fields."""
    import paper_2403_01004_gb300 as pb
    n_p, n_t, n_r = shape
    if seed is None:
        T = np.full(shape, T0)
        nn = np.full(shape, n)
        B = [np.full(shape, 1.7 * b) for b in bhat]
    else:
        rng = np.random.default_rng(seed)
        T = 1.0 + 0.2 * rng.random(shape)
        nn = 0.5 + rng.random(shape)
        B = [rng.standard_normal(shape) + (0.5 if a == 2 else 0.0) for a in range(3)]
    op = TCOperator.box(T, nn, B, C)
    ctx = pb.parabolic_setup_box(n_r, n_t, n_p, "tc", {"T0": _cuda(T), "n": _cuda(nn), "B": [_cuda(b) for b in B]},
                                 prec, C=C)
    return op, ctx


def visc_box_problem(shape, prec, seed=None):
    import paper_2403_01004_gb300 as pb
    n_p, n_t, n_r = shape
    if seed is None:
        rho = [np.full(shape, 0.8)] * 3
        nu = [np.full(shape, 0.05)] * 3
    else:
        rng = np.random.default_rng(seed)
        rho = [0.5 + rng.random(shape) for _ in range(3)]
        nu = [0.01 + 0.05 * rng.random(shape) for _ in range(3)]
    op = ViscOperator.box(rho, nu)
    ctx = pb.parabolic_setup_box(n_r, n_t, n_p, "visc", {"rho": [_cuda(a) for a in rho], "nu": [_cuda(a) for a in nu]},
                                 prec)
    return op, ctx


BHAT = np.array([0.36, 0.48, 0.8])
SHAPE = (10, 6, 8)          # (n_phi, n_theta, n_r)


def _mode_problem(kind, m):
    u, th = mode(SHAPE, m)
    if kind == "tc":
        op, ctx = tc_box_problem(SHAPE, "fp64", BHAT, T0=1.3, n=0.7, C=1.0 / 3.0)
        lam = (1.0 / 3.0 / 0.7) * tc_symbol(th, BHAT, kappa=1.3 ** 2.5)
        return op, ctx, u, lam
    op, ctx = visc_box_problem(SHAPE, "fp64")
    return op, ctx, np.concatenate([u, 2 * u, -u]), 0.05 * visc_symbol(th)


@pytest.mark.parametrize("kind", ["tc", "visc"])
@pytest.mark.parametrize("m", [(1, 0, 0), (2, 1, 3), (4, 3, 5)])
def test_box_apply_is_the_symbol(kind, m):
    import paper_2403_01004_gb300 as pb
    op, ctx, u, lam = _mode_problem(kind, m)
    ud = to_dev(u, ctx)
    F = to_dev(np.zeros_like(u), ctx)
    pb.parabolic_apply(ctx, ud, F)
    # tolerance on the scale of the operator (2 / dt_E bounds its spectrum): some modes, such as
    # the checkerboard in r and theta of the corner scheme, have lambda = 0
    np.testing.assert_allclose(to_host(F), lam * u, atol=1e-13 * 2.0 / op.dt_explicit())
    assert pb.parabolic_dt_explicit(ctx) == pytest.approx(op.dt_explicit(), rel=1e-14)


@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
@pytest.mark.parametrize("kind", ["tc", "visc"])
@pytest.mark.parametrize("m", [(1, 0, 0), (2, 1, 3)])
def test_box_sts_step_is_the_stability_polynomial(kind, scheme, m):
    """One unsplit step: R_s(dt lambda) u with s from dt / dt_E, to 1e-13."""
    import paper_2403_01004_gb300 as pb
    op, ctx, u, lam = _mode_problem(kind, m)
    dt = 37.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    st = pb.rkl2_advance(ctx, ud, dt, scheme=scheme, use_ptl=False)
    s = STAGES[scheme](37.0)
    assert st["work_cycle"] == [s]
    np.testing.assert_allclose(to_host(ud), R_closed(scheme, s, dt * lam) * u, atol=1e-13)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_box_be_step_and_ptl(kind):
    """One BE step u / (1 - dt lambda); the PTL of a mode (Eq. 5 and over every pair) 1/|lambda|."""
    import paper_2403_01004_gb300 as pb
    op, ctx, u, lam = _mode_problem(kind, (2, 1, 3))
    ud = to_dev(u, ctx)
    dtp, k, fmax = pb.ptl_compute(ctx, ud)
    assert dtp == pytest.approx(-1.0 / lam, rel=1e-12)
    assert pb.ptl_full_compute(ctx, ud)[0] == pytest.approx(-1.0 / lam, rel=1e-12)
    dt = 250.0 * op.dt_explicit()
    pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, rtol=1e-14, max_iter=2000)
    np.testing.assert_allclose(to_host(ud), u / (1.0 - dt * lam), atol=1e-12)


def test_box_corner_spike_has_six_neighbours():
    """A point spike in the box's corner cell: the wrapped neighbours count, 1/7 both ways."""
    import paper_2403_01004_gb300 as pb
    op, ctx = visc_box_problem((9, 5, 5), "fp64")
    v = np.zeros(op.n)
    v[0] = 1.0
    vd = to_dev(v, ctx)
    dtp, k, _ = pb.ptl_compute(ctx, vd)
    assert k == 0 and dtp == pytest.approx(1.0 / 7.0 / 0.05, rel=1e-13)
    dt, cell, d = pb.ptl_full_compute(ctx, vd)
    assert dt == pytest.approx(1.0 / 7.0 / 0.05, rel=1e-13) and cell == 0 and d == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_box_random_fields_match_the_oracle(kind, prec):
    """Random coefficients on a ragged box (tiles do not divide it): apply, the PTL (Eq. 5 and
    every pair), the STS + PTL schedule and state, and fixed-iteration BE."""
    import paper_2403_01004_gb300 as pb
    shape = (7, 11, 37)
    op, ctx = tc_box_problem(shape, prec, seed=3) if kind == "tc" else visc_box_problem(shape, prec, seed=3)
    rng = np.random.default_rng(11)
    u = 1.0 + 0.1 * rng.standard_normal(op.n)
    ud = to_dev(u, ctx)
    u = to_host(ud)
    F = to_dev(np.zeros(op.n), ctx)
    pb.parabolic_apply(ctx, ud, F)
    assert rel_max(to_host(F), op.apply(u)) <= {"fp64": 1e-12, "fp32": 1e-4}[prec]
    if prec == "fp64":
        dtp, k, _ = pb.ptl_compute(ctx, ud)
        dto, ko, _ = ptl(op, u, op.apply(u))
        assert k == ko and dtp == pytest.approx(dto, rel=1e-10)
        dt, cell, d = pb.ptl_full_compute(ctx, ud)
        dfo, keyo = ptl_full(op, u, op.apply(u))
        assert 3 * cell + d == keyo and dt == pytest.approx(dfo, rel=1e-10)
    dt = 60.0 * op.dt_explicit()
    _, log = sts_advance(op, u, dt, "rkl2", use_ptl=True)
    xd = to_dev(u, ctx)
    if prec == "fp64":
        st = pb.rkl2_advance(ctx, xd, dt, use_ptl=True)
        assert st["cycles"] == log.cycles and st["work_cycle"] == log.s and st["k_cycle"] == log.k
    else:
        pb.rkl2_advance(ctx, xd, dt, forced=log.dt_c)
    uo, _ = sts_advance(op, u, dt, "rkl2", forced=log.dt_c)
    assert rel_l2(to_host(xd), uo) <= TOL[prec], rel_l2(to_host(xd), uo)
    xd = to_dev(u, ctx)
    pb.be_pcg_advance(ctx, xd, dt, use_ptl=False, fixed_iters=15)
    res = be_solve(op, u, dt, 0.0, 0, fixed_iters=15)
    assert rel_l2(to_host(xd), res.x) <= TOL[prec], rel_l2(to_host(xd), res.x)


FIG1_NP = 256


def fig1_amplification(pb, scheme: str, n_phi: int = FIG1_NP, ratio: float = 500.0):
    """Fig. 1 (middle / right) on the GPU: conduction box 3 x 3 x n_phi with the field along phi
    (the 1-D second-order heat equation along phi for states constant in r and theta, dt_E = 1/2),
    one step of `ratio` dt_E from a delta plane; returns (z_m, measured amplification, stages)."""
    op, ctx = tc_box_problem((n_phi, 3, 3), "fp64", np.array([0.0, 0.0, 1.0]))
    dt_e = pb.parabolic_dt_explicit(ctx)
    u = np.zeros((n_phi, 3, 3))
    u[0] = 1.0
    ud = to_dev(u.reshape(-1), ctx)
    if scheme == "be":
        st = pb.be_pcg_advance(ctx, ud, ratio * dt_e, use_ptl=False, rtol=1e-14, max_iter=20000)
        s = None
    else:
        st = pb.rkl2_advance(ctx, ud, ratio * dt_e, scheme=scheme, use_ptl=False)
        s = st["work_cycle"][0]
    line = to_host(ud).reshape(n_phi, 3, 3)[:, 1, 1]
    amp = np.fft.fft(line).real
    m = np.arange(n_phi)
    z = ratio * dt_e * (-4.0 * np.sin(np.pi * m / n_phi) ** 2)
    ctx.close()
    return z, amp, s, dt_e


@pytest.mark.parametrize("scheme", ["rkl2", "rkg2", "be"])
def test_fig1_amplification_factors_on_the_gpu(scheme):
    import paper_2403_01004_gb300 as pb
    z, amp, s, dt_e = fig1_amplification(pb, scheme)
    assert dt_e == pytest.approx(0.5, rel=1e-14)
    assert z.min() == pytest.approx(-1000.0, rel=1e-12)
    if scheme == "be":
        np.testing.assert_allclose(amp, 1.0 / (1.0 - z), atol=1e-12)
        return
    assert s == STAGES[scheme](500.0) and (scheme == "rkl2" or s % 2 == 1)
    np.testing.assert_allclose(amp, R_closed(scheme, s, z), atol=1e-12)
    high = np.abs(z) > 500.0
    if scheme == "rkg2":
        # Sec. 3.1: RKG2 saturates lower and varies less across the high modes than RKL2
        zl, al, sl, _ = fig1_amplification(pb, "rkl2")
        assert np.abs(amp[high]).max() < np.abs(al[high]).max()
        assert np.ptp(amp[high]) < np.ptp(al[high])
