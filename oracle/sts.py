"""Super-time-stepping: the s-stage three-term recurrence shared by RKL2 and RKG2.

Stage loop (Appendix A, left column; RKL2 uses the same loop with its own coefficients):
    u_0 = u^n,  y_0 = F(u_0),  u_1 = u_0 + mut_1 dt y_0,
    u_k = mu_k u_{k-1} + nu_k u_{k-2} + (1 - mu_k - nu_k) u_0 + mut_k dt F(u_{k-1}) + gt_k dt y_0,
    u^{n+1} = u_s.

RKG2 with alpha = 3/2 (Appendix A, right column and the lines below it):
    b_0 = 1, b_1 = 1/3, b_k = 4 (k-1)(k+4) / (3 k (k+1)(k+2)(k+3)) for k >= 2,
    w = 6 / ((s+4)(s-1)),  mut_1 = w,
    mu_k = (2 + 1/k) b_k / b_{k-1},  nu_k = -(1 + 1/k) b_k / b_{k-2},  mut_k = mu_k w,
    gt_k = (k (k+1)/2 b_{k-1} - 1) mut_k,
    s = ceil( sqrt(25 + 24 dt/dt_E)/2 - 3/2 ), then made odd by adding one stage if even.

RKL2 (Sec. 3.1 cites it; the coefficients are those of the published Legendre method of Meyer,
Balsara & Aslam, restated here from its stability polynomial R_s(z) = a_s + b_s P_s(1 + w1 z)):
    b_0 = b_1 = 1/3, b_j = (j^2 + j - 2) / (2 j (j+1)) for j >= 2,  a_j = 1 - b_j,
    w1 = 4 / (s^2 + s - 2),  mut_1 = b_1 w1,
    mu_j = (2j - 1)/j b_j / b_{j-1},  nu_j = -(j - 1)/j b_j / b_{j-2},  mut_j = mu_j w1,
    gt_j = -a_{j-1} mut_j,
    s = the smallest integer >= 2 with (s^2 + s - 2)/4 >= dt/dt_E.

Both stage-count rules are evaluated as integer inequalities ((s^2+s-2) >= 4r and
(s+4)(s-1) >= 6r, the squared forms of the square-root formulas) so that exact-integer ratios do
not round up, and with r taken as r (1 - 1e-12): a ratio within rounding of a stage-count
boundary (a cycle length equal to dt_E, say) takes the smaller count instead of a count decided
by the last bit of dt_E.  s >= 2 is needed for w (undefined at s = 1); RKG2 is then raised to odd
s >= 3.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MAX_STAGES = 1 << 20
TIE = 1.0 - 1e-12      # ratios within 1e-12 of a boundary take the smaller stage count


@dataclasses.dataclass
class STSCoefficients:
    s: int
    mu: np.ndarray    # index 0..s (entries 0, 1 unused)
    nu: np.ndarray
    mut: np.ndarray   # mut[1] used by stage 1
    gt: np.ndarray


def rkl2_stages(r: float) -> int:
    if not (r >= 0.0) or math.isinf(r):
        raise ValueError("dt/dt_E must be finite and >= 0")
    r = r * TIE
    s = max(2, int(math.ceil((math.sqrt(9.0 + 16.0 * r) - 1.0) / 2.0)))
    while s > 2 and (s - 1) * (s - 1) + (s - 1) - 2 >= 4.0 * r:
        s -= 1
    while s * s + s - 2 < 4.0 * r:
        s += 1
    if s > MAX_STAGES:
        raise ValueError("stage count too large")
    return s


def rkg2_stages(r: float) -> int:
    if not (r >= 0.0) or math.isinf(r):
        raise ValueError("dt/dt_E must be finite and >= 0")
    r = r * TIE
    s = max(2, int(math.ceil(0.5 * math.sqrt(25.0 + 24.0 * r) - 1.5)))
    while s > 2 and (s - 1 + 4) * (s - 1 - 1) >= 6.0 * r:
        s -= 1
    while (s + 4) * (s - 1) < 6.0 * r:
        s += 1
    if s % 2 == 0:
        s += 1
    if s > MAX_STAGES:
        raise ValueError("stage count too large")
    return s


def rkl2_coefficients(s: int) -> STSCoefficients:
    if s < 2:
        raise ValueError("RKL2 needs s >= 2")
    b = np.empty(s + 1)
    b[0] = b[1] = 1.0 / 3.0
    for j in range(2, s + 1):
        b[j] = (j * j + j - 2.0) / (2.0 * j * (j + 1.0))
    a = 1.0 - b
    w1 = 4.0 / (s * s + s - 2.0)
    mu = np.zeros(s + 1); nu = np.zeros(s + 1); mut = np.zeros(s + 1); gt = np.zeros(s + 1)
    mut[1] = b[1] * w1
    for j in range(2, s + 1):
        mu[j] = (2.0 * j - 1.0) / j * b[j] / b[j - 1]
        nu[j] = -(j - 1.0) / j * b[j] / b[j - 2]
        mut[j] = mu[j] * w1
        gt[j] = -a[j - 1] * mut[j]
    return STSCoefficients(s, mu, nu, mut, gt)


def rkg2_b(k: int) -> float:
    if k == 0:
        return 1.0
    if k == 1:
        return 1.0 / 3.0
    return 4.0 * (k - 1.0) * (k + 4.0) / (3.0 * k * (k + 1.0) * (k + 2.0) * (k + 3.0))


def rkg2_coefficients(s: int) -> STSCoefficients:
    if s < 2:
        raise ValueError("RKG2 needs s >= 2")
    b = np.array([rkg2_b(k) for k in range(s + 1)])
    w = 6.0 / ((s + 4.0) * (s - 1.0))
    mu = np.zeros(s + 1); nu = np.zeros(s + 1); mut = np.zeros(s + 1); gt = np.zeros(s + 1)
    mut[1] = w
    for k in range(2, s + 1):
        mu[k] = (2.0 + 1.0 / k) * b[k] / b[k - 1]
        nu[k] = -(1.0 / k + 1.0) * b[k] / b[k - 2]
        mut[k] = mu[k] * w
        gt[k] = (k * (k + 1.0) / 2.0 * b[k - 1] - 1.0) * mut[k]
    return STSCoefficients(s, mu, nu, mut, gt)


SCHEMES = {
    "rkl2": (rkl2_stages, rkl2_coefficients),
    "rkg2": (rkg2_stages, rkg2_coefficients),
}


def sts_step(apply_F, u0, y0, dt: float, co: STSCoefficients):
    """One s-stage super step of size dt from u0, with y0 = F(u0) given."""
    u_km2 = u0
    u_km1 = u0 + co.mut[1] * dt * y0
    for k in range(2, co.s + 1):
        Fk = apply_F(u_km1)
        u_k = (co.mu[k] * u_km1 + co.nu[k] * u_km2 + (1.0 - co.mu[k] - co.nu[k]) * u0
               + co.mut[k] * dt * Fk + co.gt[k] * dt * y0)
        u_km2, u_km1 = u_km1, u_k
    return u_km1
