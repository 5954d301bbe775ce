// Host special functions for the off-line part (FP64).
//
// J0, J1, Y0, Y1 and integer-order J_n, written for this library:
//   * x < 20: Bessel's integral J_n(x) = (1/2pi) int_0^{2pi} cos(x sin t - n t) dt
//     summed by the trapezoid rule with K > n + x + 48 points, which is exact to
//     rounding because the rule's error is a sum of J_{n + jK}(x) terms (the same
//     aliasing identity as the circular quadrature of Sec. 5); Y0 and Y1 from the
//     Neumann series Y0 = (2/pi)(log(x/2) + gamma) J0 - (4/pi) sum_k (-1)^k J_2k / k
//     and its derivative;
//   * x >= 20: Hankel's asymptotic expansion, truncated at its smallest term
//     (error below exp(-2x));
//   * J_M(x) for M >= x (circle sizing, Sec. 5): Miller's backward recurrence
//     normalised by J1(x).
#pragma once
#include <vector>

namespace sbd {

double bessel_j0(double x);
double bessel_j1(double x);
double bessel_y0(double x);
double bessel_y1(double x);
// Y0(x) - (2/pi) log(x/2) J0(x): the part of Y0 that is smooth at 0 (no cancellation).
double bessel_y0_regular(double x);
// J_n(x) for 0 <= n, small x (< 64) by the trapezoid rule.
double bessel_jn_small(int n, double x);
// J_M(x) for M in [m_lo, m_hi] (m_lo >= x - 1 allowed), into out[M - m_lo].
void bessel_jn_range(double x, int m_lo, int m_hi, std::vector<double>& out);
// k-th positive root of J0 (k >= 1), of J1, and of Y0.
double j0_root(int k);
double j1_root(int k);
double y0_root(int k);
// k-th positive root of x J1(x) = H J0(x), H > 0 (the Dini roots of the Robin condition).
double dini_root(int k, double H);
// The first root of Y0 that is >= x.
double y0_first_root_at_least(double x);

}  // namespace sbd
