"""Cartesian periodic unit boxes (h = 1, W = V = 1, w = 1) for the closed-form eigenmode pins.

On such a box the oracle operators reduce to constant-coefficient stencils whose Fourier symbols
are known in closed form.  These helpers only build coefficient arrays for the oracle classes."""
import numpy as np
from scipy.special import eval_gegenbauer, eval_legendre

from oracle.tc import TCOperator
from oracle.visc import ViscOperator


def tc_box(shape, bhat, kappa=1.0):
    """Anisotropic conduction with constant kappa and unit direction bhat = (b_r, b_t, b_p)."""
    bhat = np.asarray(bhat, dtype=np.float64)
    ahat = np.empty((3,) + tuple(shape))
    for x in range(3):
        ahat[x] = np.sqrt(kappa) * bhat[x] / 4.0
    return TCOperator(ahat, np.ones(shape), periodic=True)


def visc_box(shape):
    ones = np.ones(shape)
    return ViscOperator([(ones, ones, ones)] * 3, [ones] * 3, periodic=True)


def mode(shape, m, phase=0.3):
    """cos(theta . x + phase) with theta_a = 2 pi m_a / N_a, on an array of shape (n_p, n_t, n_r);
    m = (m_r, m_t, m_p)."""
    n_p, n_t, n_r = shape
    k, j, i = np.meshgrid(np.arange(n_p), np.arange(n_t), np.arange(n_r), indexing="ij")
    th = (2 * np.pi * m[0] / n_r, 2 * np.pi * m[1] / n_t, 2 * np.pi * m[2] / n_p)
    return np.cos(th[0] * i + th[1] * j + th[2] * k + phase).reshape(-1), th


def tc_symbol(th, bhat, kappa=1.0):
    """Eigenvalue of the corner scheme for mode angles th = (th_r, th_t, th_p):
    lambda = -kappa (bhat . g)^2, g_r = 2 sin(th_r/2) cos(th_t/2) cos(th_p/2) (cyclic)."""
    s = [np.sin(t / 2) for t in th]
    c = [np.cos(t / 2) for t in th]
    g = np.array([2 * s[0] * c[1] * c[2], 2 * c[0] * s[1] * c[2], 2 * c[0] * c[1] * s[2]])
    return -kappa * float(np.dot(bhat, g)) ** 2


def visc_symbol(th):
    return -sum(4 * np.sin(t / 2) ** 2 for t in th)


def R_closed(scheme, s, z):
    """Amplification factor of s-stage RKL2 (shifted Legendre form) or RKG2 (Gegenbauer C^(3/2)
    form, Appendix A) at z = dt lambda, written from the closed forms of the stability
    polynomials: R = a_s + b_s P(1 + w z)."""
    if scheme == "rkl2":
        b = (s * s + s - 2.0) / (2.0 * s * (s + 1.0))
        return (1 - b) + b * eval_legendre(s, 1.0 + 4.0 / (s * s + s - 2.0) * z)
    b = 4.0 * (s - 1.0) * (s + 4.0) / (3.0 * s * (s + 1.0) * (s + 2.0) * (s + 3.0))
    a = 1.0 - b * (s + 1.0) * (s + 2.0) / 2.0
    return a + b * eval_gegenbauer(s, 1.5, 1.0 + 6.0 / ((s + 4.0) * (s - 1.0)) * z)
