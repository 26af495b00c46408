"""Pins of the oracle's super-time-stepping coefficients and stage counts (Appendix A; Sec. 3.1).

Every check compares the oracle against something it does not compute itself: values printed in
the paper, hand-worked stage counts, the Legendre / Gegenbauer polynomials of scipy, and the
order and stability conditions of the method."""
import math
from fractions import Fraction
import os

import numpy as np
import pytest
from numpy.polynomial import Polynomial
from scipy.special import eval_gegenbauer, eval_legendre

from oracle.sts import (rkg2_coefficients, rkg2_stages, rkl2_coefficients, rkl2_stages,
                        sts_step)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_rkg2_printed_starting_values():
    """Appendix A prints b0, b1, b2, mut1 = w, mu2 = 1/2, nu2 = -1/10, mut2 = mu2 w, gamma2 = 0."""
    from oracle.sts import rkg2_b
    for s in (3, 5, 9, 25):
        co = rkg2_coefficients(s)
        w = 6.0 / ((s + 4) * (s - 1))
        got = {"b0": rkg2_b(0), "b1": rkg2_b(1), "b2": rkg2_b(2), "mut1": co.mut[1],
               "mu2": co.mu[2], "nu2": co.nu[2], "mut2": co.mut[2], "gamma2": co.gt[2]}
        for name, val in _read_golden("rkg2_appendix_a.txt"):
            if val.endswith("*w"):
                expect = float(Fraction(val[:-2])) * w
            else:
                expect = float(Fraction(val))
            assert got[name] == pytest.approx(expect, rel=1e-15, abs=1e-15), (s, name)


def test_stage_counts_golden():
    fn = {"rkl2": rkl2_stages, "rkg2": rkg2_stages}
    for scheme, r, s in _read_golden("stage_counts.txt"):
        assert fn[scheme](float(r)) == int(s), (scheme, r)


def test_stage_count_inequalities_sweep():
    """s is the smallest admissible count: the stability bound holds at s and fails at s-1."""
    for r in np.concatenate([np.linspace(0.01, 50, 997), np.logspace(0, 6, 500)]):
        s = rkl2_stages(r)
        assert (s * s + s - 2) / 4.0 >= r * (1 - 1e-12)
        assert s == 2 or ((s - 1) ** 2 + (s - 1) - 2) / 4.0 < r
        g = rkg2_stages(r)
        assert g % 2 == 1 and g >= 3
        assert (g + 4) * (g - 1) / 6.0 >= r * (1 - 1e-12)
        # the paper's ceil formula, then odd
        ref = max(2, math.ceil(0.5 * math.sqrt(25 + 24 * r) - 1.5))
        ref += (ref % 2 == 0)
        assert g == ref or abs(0.5 * math.sqrt(25 + 24 * r) - 1.5 - round(0.5 * math.sqrt(25 + 24 * r) - 1.5)) < 1e-9


def test_stage_count_ties_take_the_smaller_count():
    """A ratio equal to a boundary up to rounding gives the boundary's count on both sides."""
    for r, s in ((1.0, 2), (1.0 + 2.2e-16, 2), (10.0 * (1 + 4e-16), 6), (1.0 + 1e-9, 3)):
        assert rkl2_stages(r) == s, r
    assert rkg2_stages(1000.0 * (1 + 3e-16)) == 77


def _stability_scalar(co, z):
    """R_s(z) from the oracle's stage loop applied to the scalar problem u' = z u (dt = 1)."""
    u0 = np.array([1.0])
    return sts_step(lambda u: z * u, u0, z * u0, 1.0, co)[0]


def _rkl2_closed(s, z):
    b = (s * s + s - 2.0) / (2.0 * s * (s + 1.0))
    w1 = 4.0 / (s * s + s - 2.0)
    return (1.0 - b) + b * eval_legendre(s, 1.0 + w1 * z)


def _rkg2_closed(s, z):
    b = 4.0 * (s - 1.0) * (s + 4.0) / (3.0 * s * (s + 1.0) * (s + 2.0) * (s + 3.0))
    w = 6.0 / ((s + 4.0) * (s - 1.0))
    a = 1.0 - b * eval_gegenbauer(s, 1.5, 1.0)
    return a + b * eval_gegenbauer(s, 1.5, 1.0 + w * z)


@pytest.mark.parametrize("s", [2, 3, 4, 7, 20, 63])
def test_rkl2_recurrence_is_legendre_polynomial(s):
    co = rkl2_coefficients(s)
    zmin = -(s * s + s - 2.0) / 2.0
    for z in np.linspace(zmin, 0.0, 41):
        assert _stability_scalar(co, z) == pytest.approx(_rkl2_closed(s, z), abs=1e-11)


@pytest.mark.parametrize("s", [3, 5, 9, 25, 77])
def test_rkg2_recurrence_is_gegenbauer_polynomial(s):
    co = rkg2_coefficients(s)
    zmin = -(s + 4.0) * (s - 1.0) / 3.0
    for z in np.linspace(zmin, 0.0, 41):
        assert _stability_scalar(co, z) == pytest.approx(_rkg2_closed(s, z), abs=1e-11)


def _polynomial(co):
    """The stability polynomial built with exact polynomial arithmetic through the stage loop."""
    z = Polynomial([0.0, 1.0])
    one = Polynomial([1.0])
    return sts_step(lambda u: z * u, one, z, 1.0, co)


@pytest.mark.parametrize("make", [rkl2_coefficients, rkg2_coefficients])
@pytest.mark.parametrize("s", [2, 3, 5, 8, 13])
def test_second_order_and_degree(make, s):
    """R_s(z) = 1 + z + z^2/2 + O(z^3) (second order) and deg R_s = s."""
    P = _polynomial(make(s))
    c = P.coef
    assert len(P.trim().coef) == s + 1
    assert c[0] == pytest.approx(1.0, abs=1e-13)
    assert c[1] == pytest.approx(1.0, abs=1e-12)
    assert c[2] == pytest.approx(0.5, abs=1e-11)


@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
def test_stable_on_admissible_interval(scheme):
    """|R_s(z)| <= 1 for z in [-2 r, 0] whenever s = s(r) (z = dt lambda, lambda >= -2/dt_E)."""
    stages, make = (rkl2_stages, rkl2_coefficients) if scheme == "rkl2" else (rkg2_stages, rkg2_coefficients)
    for r in [0.7, 3.0, 10.0, 100.0, 1000.0]:
        s = stages(r)
        co = make(s)
        for z in np.linspace(-2.0 * r, 0.0, 301):
            assert abs(_stability_scalar(co, z)) <= 1.0 + 1e-10, (scheme, r, z)


def test_rkg2_even_stage_count_keeps_top_mode():
    """Appendix A: with even s the amplification at the highest mode (x = 1 + w z = -1) is 1;
    with odd s it is 2 a_s - 1 < 1 in magnitude."""
    for s in (4, 6, 10, 24):
        co = rkg2_coefficients(s)
        z = -(s + 4.0) * (s - 1.0) / 3.0
        assert _stability_scalar(co, z) == pytest.approx(1.0, abs=1e-10)
    for s in (3, 5, 11, 25):
        co = rkg2_coefficients(s)
        z = -(s + 4.0) * (s - 1.0) / 3.0
        assert abs(_stability_scalar(co, z)) < 0.5


def test_fig1_left_speedup():
    """Fig. 1 (left): speedup over explicit Euler, dt/(s dt_E) = r/s, grows like sqrt(r) and
    RKG2 is close to RKL2 (RKL2 s ~ 2 sqrt(r), RKG2 s ~ sqrt(6 r))."""
    rs = np.logspace(1, 4, 30)
    sp_l = np.array([r / rkl2_stages(r) for r in rs])
    sp_g = np.array([r / rkg2_stages(r) for r in rs])
    assert np.all(np.diff(sp_l) > 0) and np.all(np.diff(sp_g) > -0.2)
    ratio = sp_l[-5:] / sp_g[-5:]
    assert np.all((ratio > 1.1) & (ratio < 1.3))
    assert sp_l[-1] == pytest.approx(np.sqrt(rs[-1]) / 2, rel=0.02)
