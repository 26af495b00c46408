"""Pins of the oracle's operators (Eq. 2) and their spherical geometry.

* Fourier symbols on periodic boxes (closed forms of the corner scheme and the 7-point scheme).
* Convergence to analytic divergences on the sphere (pins every metric factor and volume).
* Closed-form shell volume.
* Symmetry and semi-definiteness of M L, zero row sums (conservation), diagonal and
  Gershgorin rows against the dense matrix assembled column by column from `apply`.
* Positivity of the isotropic operator; non-monotonicity of the anisotropic corner scheme."""
import numpy as np
import pytest

import synth
from oracle.dense import dense_matrix
from oracle.geometry import Shell
from oracle.tc import TCOperator
from oracle.visc import ViscOperator
from periodic import mode, tc_box, tc_symbol, visc_box, visc_symbol


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (0, 0, 1), (2, 1, 3), (5, 3, 2), (4, 4, 4)])
def test_tc_fourier_symbol(m):
    shape = (8, 6, 10)
    rng = np.random.default_rng(1)
    b = rng.normal(size=3); b /= np.linalg.norm(b)
    op = tc_box(shape, b, kappa=2.5)
    u, th = mode(shape, m)
    lam = tc_symbol(th, b, kappa=2.5)
    np.testing.assert_allclose(op.apply(u), lam * u, atol=1e-13 * max(1.0, abs(lam)))


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (0, 0, 1), (2, 1, 3), (5, 3, 4)])
def test_visc_fourier_symbol(m):
    shape = (8, 6, 10)
    op = visc_box(shape)
    u, th = mode(shape, m)
    uu = np.concatenate([u, 0.5 * u, -u])
    lam = visc_symbol(th)
    np.testing.assert_allclose(op.apply(uu), lam * uu, atol=1e-13)


def test_tc_1d_gershgorin_is_explicit_limit():
    """With bhat along r and kappa = h = 1 the scheme is the 3-point Laplacian; its Gershgorin
    bound gives dt_E = h^2/2, the forward-Euler limit of the 1-D heat equation."""
    op = tc_box((3, 3, 16), (1.0, 0.0, 0.0))
    assert op.dt_explicit() == pytest.approx(0.5, rel=1e-15)
    op = visc_box((3, 3, 16))
    assert op.dt_explicit() == pytest.approx(1.0 / 6.0, rel=1e-15)


def test_shell_volume_closed_form():
    g = synth.make_grid(17, 13, 11, 1.07)
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    assert sh.cell_volume().sum() == pytest.approx(4.0 / 3.0 * np.pi * (10.0 ** 3 - 1.0), rel=1e-13)


def _tc_field_op(n, B, r_span=(1.0, 2.0)):
    """Conduction with kappa = n = 1 and C = 1 so that F = div(b b . grad u)."""
    n_r, n_t, n_p = n
    g = synth.Grid(np.linspace(*r_span, n_r + 1), synth.theta_faces(n_t), n_p)
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    ones = np.ones(sh.shape)
    Bc = [np.full(sh.shape, float(b)) for b in B]
    return sh, TCOperator.spherical(sh, ones, ones, Bc, C=1.0)


def _interior_error(sh, op, u, exact, margin):
    F = op.apply(u.reshape(-1)).reshape(sh.shape)
    sl = (slice(None), slice(margin[1], sh.n_t - margin[1]), slice(margin[0], sh.n_r - margin[0]))
    return np.max(np.abs(F[sl] - exact[sl]))


CASES = {
    # b along r, u = r^2:  (1/r^2) d/dr (r^2 2r) = 6
    "radial": ((1, 0, 0), lambda r, t, p: r ** 2, lambda r, t, p: 6.0 + 0 * r),
    # b along theta, u = cos t:  (1/(r^2 sin t)) d/dt (sin t (-sin t)) = -2 cos t / r^2
    "polar": ((0, 1, 0), lambda r, t, p: np.cos(t) + 0 * r, lambda r, t, p: -2 * np.cos(t) / r ** 2),
    # b along phi, u = cos p:  (1/(r^2 sin^2 t)) d2/dp2 cos p = -cos p / (r^2 sin^2 t)
    "azimuthal": ((0, 0, 1), lambda r, t, p: np.cos(p) + 0 * r,
                  lambda r, t, p: -np.cos(p) / (r ** 2 * np.sin(t) ** 2)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_tc_converges_to_divergence_on_sphere(case):
    B, fu, fex = CASES[case]
    errs = []
    for n in (16, 32, 64):
        sh, op = _tc_field_op((n, n, 2 * n), B)
        rr = sh.r_c[None, None, :]; tt = sh.t_c[None, :, None]
        pp = (sh.dphi * (np.arange(sh.n_p) + 0.5))[:, None, None]
        u = np.broadcast_to(fu(rr, tt, pp), sh.shape).copy()
        ex = np.broadcast_to(fex(rr, tt, pp), sh.shape)
        errs.append(_interior_error(sh, op, u, ex, (n // 4, n // 4)))
    # second order: the error falls towards 1/4 per halving of the spacing
    assert errs[0] / errs[1] > 2.8 and errs[1] / errs[2] > 3.2, errs


@pytest.mark.parametrize("comp", [0, 1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_visc_converges_to_laplacian_on_sphere(case, comp):
    """With nu = rho = 1 each component's operator is the scalar Laplacian on its own grid."""
    _, fu, fex = CASES[case]
    errs = []
    for n in (16, 32, 64):
        g = synth.Grid(np.linspace(1.0, 2.0, n + 1), synth.theta_faces(n), 2 * n)
        sh = Shell(g.r_face, g.t_face, g.n_phi)
        shapes = [synth.staggered_shape(g, c) for c in range(3)]
        op = ViscOperator.spherical(sh, [np.ones(s) for s in shapes], [np.ones(s) for s in shapes])
        pr, pt, pp = synth.staggered_points(g, comp)
        rr = pr[None, None, :]; tt = pt[None, :, None]; ppp = pp[:, None, None]
        u = [np.zeros(s) for s in shapes]
        u[comp] = np.broadcast_to(fu(rr, tt, ppp), shapes[comp]).copy()
        F = op.split(op.apply(np.concatenate([a.reshape(-1) for a in u])))[comp]
        ex = np.broadcast_to(fex(rr, tt, ppp), shapes[comp])
        m = n // 4
        errs.append(np.max(np.abs(F - ex)[:, m:-m, m:-m]))
    if max(errs) < 1e-10:      # exact on this grid (u = r^2 on the r-face grid)
        return
    assert errs[0] / errs[1] > 2.8 and errs[1] / errs[2] > 3.2, errs


def _small_tc(seed=3, shape=(5, 4, 6), tilt=True):
    n_r, n_t, n_p = shape
    g = synth.make_grid(n_r, n_t, n_p, 1.3)
    m = synth.random_unit_vector(np.random.default_rng(seed)) if tilt else None
    inp = synth.tc_inputs(g, seed, noise=0.3, m=m)
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    return sh, inp, TCOperator.spherical(sh, inp.T, inp.n, inp.B)


def _small_visc(seed=3, shape=(5, 4, 6)):
    n_r, n_t, n_p = shape
    g = synth.make_grid(n_r, n_t, n_p, 1.3)
    vi = synth.visc_inputs(g, seed)
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    return sh, vi, ViscOperator.spherical(sh, vi.rho, vi.nu)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_weighted_operator_symmetric_nsd_conservative(kind):
    _, _, op = _small_tc() if kind == "tc" else _small_visc()
    A = dense_matrix(op.apply_A, op.n)
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-14 * scale
    assert np.abs(A.sum(axis=1)).max() <= 1e-14 * scale * 27
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() <= 1e-12 * scale
    # F = w A u
    L = dense_matrix(op.apply, op.n)
    np.testing.assert_allclose(L, op.w[:, None] * A, rtol=1e-14, atol=1e-14 * np.abs(L).max())


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_diag_and_gershgorin_match_dense(kind):
    _, _, op = _small_tc() if kind == "tc" else _small_visc()
    A = dense_matrix(op.apply_A, op.n)
    np.testing.assert_allclose(op.diag_A(), np.diag(A), rtol=1e-13)
    L = op.w[:, None] * A
    np.testing.assert_allclose(op.gershgorin(), np.abs(L).sum(axis=1), rtol=1e-13)
    rho = np.max(np.abs(np.linalg.eigvals(L)))
    assert op.dt_explicit() <= 2.0 / rho * (1 + 1e-12)


def test_tc_boundaries_are_zero_flux():
    """No corner on r_min, r_max or the poles: a field that differs only across a boundary
    layer still conserves sum(M u) exactly and F vanishes for constant fields."""
    sh, inp, op = _small_tc(shape=(6, 5, 7))
    assert np.abs(op.apply(np.full(op.n, 3.7))).max() <= 1e-12 * np.abs(op.w).max()
    assert np.all(op.ahat[:, :, -1, :] == 0) and np.all(op.ahat[:, :, :, -1] == 0)


def test_visc_positivity_forward_stable():
    """The isotropic 7-point operator is an M-matrix: I + dt L >= 0 for dt <= dt_E."""
    _, _, op = _small_visc(shape=(6, 5, 7))
    L = dense_matrix(op.apply, op.n)
    E = np.eye(op.n) + op.dt_explicit() * L
    assert E.min() >= -1e-14
    off = L - np.diag(np.diag(L))
    assert off.min() >= 0.0


def test_tc_corner_scheme_not_monotone():
    """Known property of the symmetric corner scheme: some off-diagonal entries of L are
    negative, so positivity is not guaranteed for the anisotropic operator."""
    _, _, op = _small_tc(shape=(6, 5, 7))
    L = dense_matrix(op.apply, op.n)
    off = L - np.diag(np.diag(L))
    assert off.min() < 0.0
