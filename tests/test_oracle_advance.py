"""Pins of the oracle's time integration: STS and BE on eigenmodes (closed-form amplification),
the PTL (Eq. 5) on an eigenmode and on a spike, the unlocalised PTL (Eq. 4 over all pairs)
against brute force and closed forms, the dynamic cycle loop on an eigenmode, the
Fig. 1 set-up, conservation on the sphere, and dense eigen-decomposition / Cholesky truth."""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.special import eval_gegenbauer, eval_legendre

import synth
from oracle.advance import be_advance, sts_advance
from oracle.dense import apply_function, dense_matrix, symmetric_eig
from oracle.geometry import Shell
from oracle.pcg import be_solve
from oracle.ptl import ptl, ptl_full
from oracle.sts import rkg2_stages, rkl2_stages
from oracle.tc import TCOperator
from oracle.visc import ViscOperator
from periodic import R_closed, mode, tc_box, tc_symbol, visc_box, visc_symbol


STAGES = {"rkl2": rkl2_stages, "rkg2": rkg2_stages}


@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
@pytest.mark.parametrize("m", [(1, 0, 0), (2, 1, 3), (5, 3, 2)])
def test_sts_step_on_eigenmode(scheme, m):
    shape = (8, 6, 10)
    b = np.array([0.6, -0.48, 0.64])
    op = tc_box(shape, b, kappa=1.7)
    u, th = mode(shape, m)
    lam = tc_symbol(th, b, kappa=1.7)
    dt = 37.0 * op.dt_explicit()
    un, log = sts_advance(op, u, dt, scheme, use_ptl=False)
    s = STAGES[scheme](dt / op.dt_explicit())
    assert log.s == [s]
    np.testing.assert_allclose(un, R_closed(scheme, s, dt * lam) * u, atol=1e-13)


@pytest.mark.parametrize("m", [(1, 0, 0), (2, 1, 3), (5, 3, 4)])
def test_be_step_on_eigenmode(m):
    shape = (8, 6, 10)
    op = visc_box(shape)
    u1, th = mode(shape, m)
    u = np.concatenate([u1, 2 * u1, -u1])
    lam = visc_symbol(th)
    dt = 250.0 * op.dt_explicit()
    un, log = be_advance(op, u, dt, use_ptl=False, rtol=1e-14, max_iter=500)
    np.testing.assert_allclose(un, u / (1.0 - dt * lam), atol=1e-12)


def test_ptl_on_eigenmode_is_inverse_eigenvalue():
    """F = lambda u, so every qualifying neighbour gives -du/dF = -1/lambda."""
    shape = (8, 6, 10)
    b = np.array([0.36, 0.48, 0.8])
    op = tc_box(shape, b)
    u, th = mode(shape, (2, 1, 1))
    lam = tc_symbol(th, b)
    dtp, k, fmax = ptl(op, u, op.apply(u))
    assert dtp == pytest.approx(-1.0 / lam, rel=1e-12)
    assert fmax == pytest.approx(abs(lam) * np.abs(u).max(), rel=1e-12)


def test_ptl_on_spikes():
    """Unit spike: a 1-D spike (the plane i = 4, constant in theta and phi) under the 3-point
    Laplacian (bhat along r) gives dt_PTL = h^2/3 = (2/3) dt_E; a point spike under the 3-D
    7-point Laplacian gives 1/7 = (6/7) dt_E."""
    op = tc_box((5, 5, 9), (1.0, 0.0, 0.0))
    u = np.zeros(op.shape); u[:, :, 4] = 1.0; u = u.reshape(-1)
    dtp, k, _ = ptl(op, u, op.apply(u))
    assert k == 4
    assert dtp == pytest.approx(1.0 / 3.0, rel=1e-14)
    assert dtp == pytest.approx(2.0 / 3.0 * op.dt_explicit(), rel=1e-14)
    vop = visc_box((5, 5, 9))
    v = np.zeros(vop.n); v[vop.offsets[1] + 4 + 9 * (2 + 5 * 2)] = 1.0
    dtp, k, _ = ptl(vop, v, vop.apply(v))
    assert k == vop.offsets[1] + 4 + 9 * (2 + 5 * 2)
    assert dtp == pytest.approx(1.0 / 7.0, rel=1e-14)


def test_ptl_no_candidate_is_infinite_and_ties_pick_first():
    op = visc_box((4, 4, 4))
    u = np.zeros(op.n)
    dtp, k, fmax = ptl(op, u, op.apply(u))
    assert dtp == math.inf and k == 0 and fmax == 0.0


def _brute_full(shapes, u, F, periodic=False):
    """Eq. 4 over all face-neighbour pairs by explicit loops: for every cell (k, j, i) of every
    component and each direction, the neighbour one cell up (phi periodic; r and theta periodic
    only on the box)."""
    best, key, off = math.inf, -1, 0
    for (n_p, n_t, n_r) in shapes:
        for k in range(n_p):
            for j in range(n_t):
                for i in range(n_r):
                    a = off + (k * n_t + j) * n_r + i
                    nbrs = []
                    if i + 1 < n_r:
                        nbrs.append((a + 1, 0))
                    elif periodic:
                        nbrs.append((off + (k * n_t + j) * n_r, 0))
                    if j + 1 < n_t:
                        nbrs.append((a + n_r, 1))
                    elif periodic:
                        nbrs.append((off + k * n_t * n_r + i, 1))
                    nbrs.append((off + (((k + 1) % n_p) * n_t + j) * n_r + i, 2))
                    for b, d in nbrs:
                        du, dF = u[a] - u[b], F[a] - F[b]
                        if du != 0.0 and dF != 0.0 and du * dF < 0.0:
                            r = -du / dF
                            if r < best or (r == best and 3 * a + d < key):
                                best, key = r, 3 * a + d
        off += n_p * n_t * n_r
    return best, key


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_ptl_full_matches_brute_force(kind):
    """Random states and random F (every sign case), then small-integer values (many exact ties,
    zero differences): same bound and same pair as the explicit loops."""
    rng = np.random.default_rng(7)
    box = tc_box((3, 4, 5), (0.6, 0.0, 0.8)) if kind == "tc" else visc_box((3, 4, 5))
    wl = synth.make_grid(5, 4, 3, 1.05)
    if kind == "tc":
        inp = synth.tc_inputs(wl, 5)
        sph = TCOperator.spherical(Shell(wl.r_face, wl.t_face, wl.n_phi), inp.T, inp.n, inp.B)
    else:
        vi = synth.visc_inputs(wl, 5)
        sph = ViscOperator.spherical(Shell(wl.r_face, wl.t_face, wl.n_phi), vi.rho, vi.nu)
    for op in (box, sph):
        for _ in range(3):
            u = rng.standard_normal(op.n)
            F = rng.standard_normal(op.n)
            assert ptl_full(op, u, F) == _brute_full(op.shapes, u, F, op.periodic)
            u = rng.integers(-2, 3, op.n).astype(float)
            F = rng.integers(-3, 4, op.n).astype(float)
            assert ptl_full(op, u, F) == _brute_full(op.shapes, u, F, op.periodic)


def test_box_builders_reduce_to_the_closed_form_symbols():
    """Constant inputs on the periodic box: conduction F = (C/n) kappa (bhat . D)^2-symbol times u,
    kappa = T0^{5/2}; viscosity F = (1/rho) nu rho (7-point symbol) u."""
    shape = (6, 5, 8)
    T0, n, C = 1.3, 0.7, 1.0 / 3.0
    b = np.array([0.36, 0.48, 0.8])
    op = TCOperator.box(np.full(shape, T0), np.full(shape, n), [np.full(shape, 2.5 * x) for x in b], C)
    u, th = mode(shape, (1, 2, 3))
    lam = (C / n) * tc_symbol(th, b, kappa=T0 ** 2.5)
    np.testing.assert_allclose(op.apply(u), lam * u, atol=1e-12 * abs(lam))
    vop = ViscOperator.box([np.full(shape, 0.8)] * 3, [np.full(shape, 0.05)] * 3)
    v = np.concatenate([u, 2 * u, -u])
    np.testing.assert_allclose(vop.apply(v), 0.05 * visc_symbol(th) * v, atol=1e-13)


def test_box_ptl_has_six_neighbours_everywhere():
    """A point spike at the box's corner cell (0, 0, 0): the wrapped neighbours qualify like any
    others, 1/7 under the 7-point Laplacian, for Eq. 5 and for every pair."""
    vop = visc_box((5, 5, 9))
    v = np.zeros(vop.n); v[0] = 1.0
    F = vop.apply(v)
    assert len(set(vop.neighbors(0))) == 6
    assert ptl(vop, v, F)[0] == pytest.approx(1.0 / 7.0, rel=1e-14)
    dt, key = ptl_full(vop, v, F)
    assert dt == pytest.approx(1.0 / 7.0, rel=1e-14) and key == 0


def test_ptl_full_closed_forms():
    """Eigenmode: every qualifying pair gives -1/lambda.  Point spike under the 7-point
    Laplacian: only the six spike pairs qualify, each 1/7; the smallest key is the -phi pair."""
    shape = (8, 6, 10)
    b = np.array([0.36, 0.48, 0.8])
    op = tc_box(shape, b)
    u, th = mode(shape, (2, 1, 1))
    lam = tc_symbol(th, b)
    dt, key = ptl_full(op, u, op.apply(u))
    assert dt == pytest.approx(-1.0 / lam, rel=1e-12)
    vop = visc_box((5, 5, 9))
    s = vop.offsets[1] + 4 + 9 * (2 + 5 * 2)
    v = np.zeros(vop.n); v[s] = 1.0
    dt, key = ptl_full(vop, v, vop.apply(v))
    assert dt == pytest.approx(1.0 / 7.0, rel=1e-14)
    assert key == 3 * (s - 45) + 2
    assert ptl_full(vop, np.zeros(vop.n), np.zeros(vop.n)) == (math.inf, -1)


def test_ptl_full_differs_from_fmax_localisation():
    """Planes along r under the 3-point Laplacian (bhat along r, h = 1): a spike of height 10
    holds max |F| = 20, where Eq. 5 gives h^2/3; a checkerboard patch of height 0.1 elsewhere
    has |F| <= 0.4, but each pair inside it gives -du/dF = 2/8 = 1/4, the full-grid minimum."""
    op = tc_box((3, 3, 24), (1.0, 0.0, 0.0))
    u = np.zeros(op.shape)
    u[:, :, 4] = 10.0
    for i in range(12, 18):
        u[:, :, i] = 0.1 * (-1.0) ** i
    u = u.reshape(-1)
    F = op.apply(u)
    dtp, k, fmax = ptl(op, u, F)
    assert k % 24 == 4 and fmax == pytest.approx(20.0, rel=1e-14)
    assert dtp == pytest.approx(1.0 / 3.0, rel=1e-14)
    dt, key = ptl_full(op, u, F)
    assert dt == pytest.approx(0.25, rel=1e-14)
    assert 11 <= (key // 3) % 24 <= 17 and key % 3 == 0
    assert dt == pytest.approx(0.5 * op.dt_explicit(), rel=1e-14)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_ptl_full_never_above_fmax_localisation(kind):
    """The localised bound is a minimum over a subset of the pairs."""
    wl = synth.make_grid(12, 10, 8, 1.05)
    for seed in range(3):
        if kind == "tc":
            inp = synth.tc_inputs(wl, 100 + seed, noise=0.05)
            op = TCOperator.spherical(Shell(wl.r_face, wl.t_face, wl.n_phi), inp.T, inp.n, inp.B)
            u = inp.T.reshape(-1)
        else:
            vi = synth.visc_inputs(wl, 100 + seed)
            op = ViscOperator.spherical(Shell(wl.r_face, wl.t_face, wl.n_phi), vi.rho, vi.nu)
            u = np.concatenate([c.reshape(-1) for c in vi.v])
        F = op.apply(u)
        assert ptl_full(op, u, F)[0] <= ptl(op, u, F)[0]


@pytest.mark.parametrize("ptl_mode", ["fmax", "full"])
@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
def test_cycle_loop_on_eigenmode(scheme, ptl_mode):
    """On an eigenmode the PTL stays 1/|lambda| after every cycle (the mode only scales), so the
    loop takes n = ceil(dt |lambda|) equal cycles and returns R_s(dt_c lambda)^n u; the same for
    the unlocalised PTL, every qualifying pair giving 1/|lambda|."""
    shape = (8, 6, 10)
    b = np.array([0.36, 0.48, 0.8])
    op = tc_box(shape, b)
    u, th = mode(shape, (1, 1, 0))
    lam = tc_symbol(th, b)
    assert 1.0 / abs(lam) > op.dt_explicit()          # above the floor
    # ~10 cycles: over many more, rounding-level components of faster-decaying-under-R modes
    # grow relative to the mode and the PTL drifts (a property of the schemes, not of the loop)
    dt = 9.3 / abs(lam)
    un, log = sts_advance(op, u, dt, scheme, use_ptl=True, ptl_mode=ptl_mode)
    n = math.ceil(dt * abs(lam))
    assert log.cycles == n
    dt_c = dt / n
    s = STAGES[scheme](dt_c / op.dt_explicit())
    assert set(log.s) == {s}
    np.testing.assert_allclose(log.dt_c, dt_c, rtol=1e-10)
    np.testing.assert_allclose(un, R_closed(scheme, s, dt_c * lam) ** n * u, atol=1e-12)
    # BE takes the same schedule and gives (1 - dt_c lambda)^-n
    ub, logb = be_advance(op, u, dt, use_ptl=True, rtol=1e-14, ptl_mode=ptl_mode)
    assert logb.cycles == n
    np.testing.assert_allclose(ub, u / (1.0 - dt_c * lam) ** n, atol=1e-11)


def test_cycle_floor_at_explicit_limit():
    """Where the PTL is below dt_E (the spike) the cycle length is floored at dt_E; with the
    floor removed the literal rule cycles at dt_PTL."""
    op = tc_box((5, 5, 9), (1.0, 0.0, 0.0))
    u = np.zeros(op.shape); u[:, :, 4] = 1.0; u = u.reshape(-1)
    dtE = op.dt_explicit()
    _, log = sts_advance(op, u, 3.0 * dtE, "rkl2", use_ptl=True)
    assert log.dt_c[0] == pytest.approx(dtE, rel=1e-14)
    _, log0 = sts_advance(op, u, 3.0 * dtE, "rkl2", use_ptl=True, floor=0.0, max_cycles=1000)
    assert log0.dt_c[0] == pytest.approx(dtE * 3.0 / 5.0, rel=1e-14)   # ceil(3 / (2/3)) = 5


def test_fig1_amplification_factors():
    """Fig. 1 (middle, right): 1-D uniform heat equation, second-order central differences,
    dt = 500 dt_E.  Mode amplification of RKL2, RKG2 and BE from the oracle against
    R_s(z), 1/(1-z), with z = -1000 sin^2(theta/2); RKG2's high-mode amplification saturates
    lower and varies less than RKL2's; BE damps more weakly than exp(z) at high modes."""
    N = 64
    op = tc_box((3, 3, N), (1.0, 0.0, 0.0))
    dtE = op.dt_explicit()
    dt = 500.0 * dtE
    amps = {}
    ms = np.arange(1, N // 2 + 1)
    for scheme in ("rkl2", "rkg2", "be"):
        g = []
        for m in ms:
            u, th = mode(op.shape, (m, 0, 0), phase=0.0)
            if scheme == "be":
                un, _ = be_advance(op, u, dt, use_ptl=False, rtol=1e-14, max_iter=1000)
            else:
                un, _ = sts_advance(op, u, dt, scheme, use_ptl=False)
            g.append(un @ u / (u @ u))
        amps[scheme] = np.array(g)
    z = -1000.0 * np.sin(np.pi * ms / N) ** 2
    np.testing.assert_allclose(amps["rkl2"], R_closed("rkl2", rkl2_stages(500.0), z), atol=1e-12)
    np.testing.assert_allclose(amps["rkg2"], R_closed("rkg2", rkg2_stages(500.0), z), atol=1e-12)
    np.testing.assert_allclose(amps["be"], 1.0 / (1.0 - z), rtol=1e-10)
    hi = ms > N // 4
    assert np.abs(amps["rkg2"][hi]).max() < np.abs(amps["rkl2"][hi]).max()
    assert np.std(amps["rkg2"][hi]) < np.std(amps["rkl2"][hi])
    assert np.all(amps["be"][hi] > np.exp(z[hi]))


def _sphere_tc(shape=(6, 5, 8), seed=11):
    n_r, n_t, n_p = shape
    g = synth.make_grid(n_r, n_t, n_p, 1.2)
    inp = synth.tc_inputs(g, seed, noise=0.2, m=synth.random_unit_vector(np.random.default_rng(seed)))
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    return TCOperator.spherical(sh, inp.T, inp.n, inp.B), inp.T.reshape(-1)


def _sphere_visc(shape=(6, 5, 8), seed=11):
    n_r, n_t, n_p = shape
    g = synth.make_grid(n_r, n_t, n_p, 1.2)
    vi = synth.visc_inputs(g, seed)
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    return ViscOperator.spherical(sh, vi.rho, vi.nu), np.concatenate([a.reshape(-1) for a in vi.v])


@pytest.mark.parametrize("kind", ["tc", "visc"])
@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
def test_sts_matches_dense_polynomial_and_conserves(kind, scheme):
    op, u = _sphere_tc() if kind == "tc" else _sphere_visc()
    dtE = op.dt_explicit()
    dt = 60.0 * dtE
    un, log = sts_advance(op, u, dt, scheme, use_ptl=False)
    s = log.s[0]
    exact = apply_function(op, lambda lam: R_closed(scheme, s, dt * lam), u)
    np.testing.assert_allclose(un, exact, atol=1e-12 * np.abs(u).max())
    M = 1.0 / op.w
    assert (M * un).sum() == pytest.approx((M * u).sum(), rel=1e-13)
    # with PTL cycling too
    up, logp = sts_advance(op, u, dt, scheme, use_ptl=True)
    assert (M * up).sum() == pytest.approx((M * u).sum(), rel=1e-13)
    assert sum(logp.dt_c) == pytest.approx(dt, rel=1e-12)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_be_pcg_matches_cholesky(kind):
    op, u = _sphere_tc() if kind == "tc" else _sphere_visc()
    dt = 300.0 * op.dt_explicit()
    A = dense_matrix(op.apply_A, op.n)
    S = np.diag(1.0 / op.w) - dt * A
    x_exact = scipy.linalg.cho_solve(scipy.linalg.cho_factor(S), u / op.w)
    res = be_solve(op, u, dt, rtol=1e-14, max_iter=2000)
    assert res.converged and res.true_rel_residual < 1e-13
    np.testing.assert_allclose(res.x, x_exact, rtol=1e-10, atol=1e-11 * np.abs(x_exact).max())
    # and equals exp-free BE through the eigen-decomposition
    np.testing.assert_allclose(res.x, apply_function(op, lambda lam: 1.0 / (1.0 - dt * lam), u),
                               atol=1e-10 * np.abs(u).max())


def test_be_positivity_isotropic():
    """S = M - dt A is an M-matrix for the isotropic operator: BE keeps u >= 0 for any dt."""
    op, _ = _sphere_visc()
    u = np.random.default_rng(5).uniform(0.0, 1.0, op.n)
    for ratio in (1.0, 100.0, 1e4):
        res = be_solve(op, u, ratio * op.dt_explicit(), rtol=1e-14, max_iter=5000)
        assert res.x.min() >= -1e-12


def test_pcg_fixed_iterations_reduce_residual_monotonically_in_energy():
    op, u = _sphere_tc()
    dt = 300.0 * op.dt_explicit()
    errs = []
    A = dense_matrix(op.apply_A, op.n)
    S = np.diag(1.0 / op.w) - dt * A
    x_exact = np.linalg.solve(S, u / op.w)
    for n in range(1, 12):
        x = be_solve(op, u, dt, 0.0, 0, fixed_iters=n).x
        e = x - x_exact
        errs.append(e @ S @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))
