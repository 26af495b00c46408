// Host-side float64 super-time-stepping coefficients and stage counts, shared by the one-problem
// driver and the batched launch.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace pb {

// ---- super-time-stepping coefficients (float64, host) ----------------------------------------
// RKL2 (the Legendre method cited in Sec. 3.1): s = smallest integer >= 2 with
// (s^2 + s - 2)/4 >= r; b_0 = b_1 = 1/3, b_j = (j^2 + j - 2)/(2 j (j+1)), a_j = 1 - b_j,
// w1 = 4/(s^2 + s - 2), mut_1 = b_1 w1, mu_j = (2j-1)/j b_j/b_{j-1}, nu_j = -(j-1)/j b_j/b_{j-2},
// mut_j = mu_j w1, gt_j = -a_{j-1} mut_j.
// RKG2 (Appendix A, alpha = 3/2): s = ceil(sqrt(25 + 24 r)/2 - 3/2) made odd; b_0 = 1,
// b_1 = 1/3, b_k = 4(k-1)(k+4)/(3k(k+1)(k+2)(k+3)), w = 6/((s+4)(s-1)), mut_1 = w,
// mu_k = (2 + 1/k) b_k/b_{k-1}, nu_k = -(1 + 1/k) b_k/b_{k-2}, mut_k = mu_k w,
// gt_k = (k(k+1)/2 b_{k-1} - 1) mut_k.
// Both stage counts are evaluated as the integer inequalities (s^2+s-2) >= 4r and
// (s+4)(s-1) >= 6r so that exact-integer ratios do not round up.
inline constexpr long long kMaxStages = 1 << 20;

struct Sts {
    int s = 0;
    std::vector<double> mu, nu, mut, gt;
};

// Ratios within 1e-12 (relative) of a stage-count boundary take the smaller count, so that a
// cycle length equal to a boundary up to rounding (e.g. dt_c = dt_E) does not decide s by the
// last bit of dt_E.
inline constexpr double kStageTie = 1.0 - 1e-12;

inline long long stages_rkl2(double r) {
    r *= kStageTie;
    long long s = std::max(2LL, (long long)std::ceil((std::sqrt(9.0 + 16.0 * r) - 1.0) / 2.0));
    while (s > 2 && (double)((s - 1) * (s - 1) + (s - 1) - 2) >= 4.0 * r) --s;
    while ((double)(s * s + s - 2) < 4.0 * r) ++s;
    return s;
}

inline long long stages_rkg2(double r) {
    r *= kStageTie;
    long long s = std::max(2LL, (long long)std::ceil(0.5 * std::sqrt(25.0 + 24.0 * r) - 1.5));
    while (s > 2 && (double)((s + 3) * (s - 2)) >= 6.0 * r) --s;
    while ((double)((s + 4) * (s - 1)) < 6.0 * r) ++s;
    if (s % 2 == 0) ++s;
    return s;
}

inline void coeffs_rkl2(int s, Sts& o) {
    std::vector<double> b(s + 1);
    b[0] = b[1] = 1.0 / 3.0;
    for (int j = 2; j <= s; ++j) b[j] = ((double)j * j + j - 2.0) / (2.0 * j * (j + 1.0));
    const double w1 = 4.0 / ((double)s * s + s - 2.0);
    o.s = s;
    o.mu.assign(s + 1, 0.0); o.nu.assign(s + 1, 0.0); o.mut.assign(s + 1, 0.0); o.gt.assign(s + 1, 0.0);
    o.mut[1] = b[1] * w1;
    for (int j = 2; j <= s; ++j) {
        o.mu[j] = (2.0 * j - 1.0) / j * b[j] / b[j - 1];
        o.nu[j] = -(j - 1.0) / j * b[j] / b[j - 2];
        o.mut[j] = o.mu[j] * w1;
        o.gt[j] = -(1.0 - b[j - 1]) * o.mut[j];
    }
}

inline void coeffs_rkg2(int s, Sts& o) {
    std::vector<double> b(s + 1);
    for (int k = 0; k <= s; ++k)
        b[k] = k == 0 ? 1.0 : k == 1 ? 1.0 / 3.0
             : 4.0 * (k - 1.0) * (k + 4.0) / (3.0 * k * (k + 1.0) * (k + 2.0) * (k + 3.0));
    const double w = 6.0 / ((s + 4.0) * (s - 1.0));
    o.s = s;
    o.mu.assign(s + 1, 0.0); o.nu.assign(s + 1, 0.0); o.mut.assign(s + 1, 0.0); o.gt.assign(s + 1, 0.0);
    o.mut[1] = w;
    for (int k = 2; k <= s; ++k) {
        o.mu[k] = (2.0 + 1.0 / k) * b[k] / b[k - 1];
        o.nu[k] = -(1.0 / k + 1.0) * b[k] / b[k - 2];
        o.mut[k] = o.mu[k] * w;
        o.gt[k] = (k * (k + 1.0) / 2.0 * b[k - 1] - 1.0) * o.mut[k];
    }
}

inline void make_sts(int scheme, double r, Sts& o) {
    if (!(r >= 0.0) || std::isinf(r)) throw Error{PB_EINVAL, "dt/dt_E must be finite and >= 0"};
    const long long s = scheme == PB_RKG2 ? stages_rkg2(r) : stages_rkl2(r);
    if (s > kMaxStages) throw Error{PB_EINVAL, "stage count above 2^20"};
    if (scheme == PB_RKG2) coeffs_rkg2((int)s, o);
    else coeffs_rkl2((int)s, o);
}

}  // namespace pb
