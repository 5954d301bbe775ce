// Host Bessel functions (see bessel.h for the methods).
#include "bessel.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace sbd {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;

// J_n(x) for all n in [0, nmax] by the trapezoid rule on Bessel's integral.
void jn_all_trapezoid(double x, int nmax, std::vector<double>& out) {
    int K = static_cast<int>(std::ceil(x)) + nmax + 48;
    K += K & 1;
    out.assign(nmax + 1, 0.0);
    const double dt = 2.0 * kPi / K;
    for (int j = 0; j < K; ++j) {
        const double t = j * dt;
        const double phase = x * std::sin(t);
        // cos(phase - n t) for n = 0..nmax via the rotation e^{-i t}
        const double cr = std::cos(t), sr = -std::sin(t);
        double re = std::cos(phase), im = std::sin(phase);
        for (int n = 0; n <= nmax; ++n) {
            out[n] += re;
            const double nre = re * cr - im * sr;
            const double nim = re * sr + im * cr;
            re = nre;
            im = nim;
        }
    }
    for (double& v : out) v /= K;
}

// Hankel asymptotic expansion for order nu in {0, 1}: returns (J, Y).
// P = sum_k (-1)^k a_2k / x^2k, Q = sum_k (-1)^k a_{2k+1} / x^{2k+1},
// a_k = prod_{j=1..k} (4 nu^2 - (2j-1)^2) / (k! 8^k); truncated before the terms grow.
void hankel_asymptotic(int nu, double x, double& J, double& Y) {
    const double mu = 4.0 * nu * nu;
    double P = 1.0, Q = 0.0, t = 1.0, prev = 1e300;
    for (int k = 1; k < 400; ++k) {
        t *= (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k * x);
        const double mag = std::fabs(t);
        if (mag >= prev) break;
        prev = mag;
        if (k & 1) Q += (((k - 1) / 2) & 1) ? -t : t;
        else P += ((k / 2) & 1) ? -t : t;
        if (mag < 1e-18) break;
    }
    // chi = x - (nu/2 + 1/4) pi, expanded so that x enters cos/sin exactly
    const double cx = std::cos(x), sx = std::sin(x), r2 = 0.70710678118654752440;
    double cc, sc;
    if (nu == 0) { cc = (cx + sx) * r2; sc = (sx - cx) * r2; }
    else         { cc = (sx - cx) * r2; sc = -(sx + cx) * r2; }
    const double s = std::sqrt(2.0 / (kPi * x));
    J = s * (P * cc - Q * sc);
    Y = s * (P * sc + Q * cc);
}

void small_jy(double x, double& j0, double& j1, double& y0, double& y1) {
    const int nmax = static_cast<int>(std::ceil(x)) + 48;
    std::vector<double> J;
    jn_all_trapezoid(x, nmax + 1, J);
    j0 = J[0];
    j1 = J[1];
    const double L = std::log(0.5 * x) + kEulerGamma;
    double s0 = 0.0, s1 = 0.0;
    for (int k = 1; 2 * k + 1 <= nmax + 1; ++k) {
        const double sg = (k & 1) ? -1.0 : 1.0;   // (-1)^k
        s0 += sg * J[2 * k] / k;
        s1 += sg * (J[2 * k - 1] - J[2 * k + 1]) / k;
    }
    y0 = (2.0 / kPi) * L * J[0] - (4.0 / kPi) * s0;
    // Y1 = -Y0' with J0' = -J1 and J_n' = (J_{n-1} - J_{n+1}) / 2
    y1 = -(2.0 / (kPi * x)) * J[0] + (2.0 / kPi) * L * J[1] + (2.0 / kPi) * s1;
}

// Piecewise Chebyshev tables of J0 and J1 on [0, 20): 80 pieces of width 1/4,
// 16 coefficients each, interpolated at Chebyshev points from the trapezoid values.
constexpr int kPieces = 80, kDeg = 16;
constexpr double kWidth = 0.25;
struct JTables {
    double c0[kPieces][kDeg];
    double c1[kPieces][kDeg];
    JTables() {
        std::vector<double> J;
        for (int q = 0; q < kPieces; ++q) {
            double f0[kDeg], f1[kDeg];
            for (int k = 0; k < kDeg; ++k) {
                const double t = std::cos(kPi * (k + 0.5) / kDeg);
                const double x = (q + 0.5 * (t + 1.0)) * kWidth;
                jn_all_trapezoid(x, 1, J);
                f0[k] = J[0];
                f1[k] = J[1];
            }
            for (int j = 0; j < kDeg; ++j) {
                double s0 = 0.0, s1 = 0.0;
                for (int k = 0; k < kDeg; ++k) {
                    const double c = std::cos(kPi * j * (k + 0.5) / kDeg);
                    s0 += f0[k] * c;
                    s1 += f1[k] * c;
                }
                c0[q][j] = s0 * (j == 0 ? 1.0 : 2.0) / kDeg;
                c1[q][j] = s1 * (j == 0 ? 1.0 : 2.0) / kDeg;
            }
        }
    }
};

const JTables& tables() {
    static const JTables t;   // thread-safe one-time initialisation
    return t;
}

double cheb_eval(const double* c, double x) {
    const int q = std::min(kPieces - 1, static_cast<int>(x / kWidth));
    const double t = 2.0 * (x / kWidth - q) - 1.0;
    double b1 = 0.0, b2 = 0.0;
    for (int j = kDeg - 1; j >= 1; --j) {
        const double b0 = 2.0 * t * b1 - b2 + c[q * kDeg + j];
        b2 = b1;
        b1 = b0;
    }
    return t * b1 - b2 + c[q * kDeg];
}

}  // namespace

double bessel_jn_small(int n, double x) {
    std::vector<double> J;
    jn_all_trapezoid(x, n, J);
    return J[n];
}

// Power series of J0, J1 for x < 2, where the terms decrease from the first one.
double series_j(int nu, double x) {
    const double q = -0.25 * x * x;
    double term = nu == 0 ? 1.0 : 0.5 * x, sum = term;
    for (int k = 1; k < 40; ++k) {
        term *= q / (k * (k + nu));
        sum += term;
        if (std::fabs(term) < 1e-18 * std::fabs(sum)) break;
    }
    return sum;
}

double bessel_j0(double x) {
    x = std::fabs(x);
    if (x < 2.0) return series_j(0, x);
    if (x < 20.0) return cheb_eval(&tables().c0[0][0], x);
    double J, Y;
    hankel_asymptotic(0, x, J, Y);
    return J;
}

double bessel_j1(double x) {
    const double sg = x < 0 ? -1.0 : 1.0;
    x = std::fabs(x);
    if (x < 2.0) return sg * series_j(1, x);
    if (x < 20.0) return sg * cheb_eval(&tables().c1[0][0], x);
    double J, Y;
    hankel_asymptotic(1, x, J, Y);
    return sg * J;
}

double bessel_y0_regular(double x) {
    if (x < 20.0) {
        const int nmax = static_cast<int>(std::ceil(x)) + 48;
        std::vector<double> J;
        jn_all_trapezoid(x, nmax, J);
        double s0 = 0.0;
        for (int k = 1; 2 * k <= nmax; ++k) s0 += ((k & 1) ? -1.0 : 1.0) * J[2 * k] / k;
        return (2.0 / kPi) * kEulerGamma * J[0] - (4.0 / kPi) * s0;
    }
    return bessel_y0(x) - (2.0 / kPi) * std::log(0.5 * x) * bessel_j0(x);
}

double bessel_y0(double x) {
    if (!(x > 0)) throw std::domain_error("Y0 needs x > 0");
    if (x < 20.0) {
        double j0, j1, y0, y1;
        small_jy(x, j0, j1, y0, y1);
        return y0;
    }
    double J, Y;
    hankel_asymptotic(0, x, J, Y);
    return Y;
}

double bessel_y1(double x) {
    if (!(x > 0)) throw std::domain_error("Y1 needs x > 0");
    if (x < 20.0) {
        double j0, j1, y0, y1;
        small_jy(x, j0, j1, y0, y1);
        return y1;
    }
    double J, Y;
    hankel_asymptotic(1, x, J, Y);
    return Y;
}

void bessel_jn_range(double x, int m_lo, int m_hi, std::vector<double>& out) {
    out.assign(m_hi - m_lo + 1, 0.0);
    // Miller: recur downward from an order N where J_N(x) is negligible, keep the
    // orders [m_lo, m_hi], and normalise with 1 = J0^2 + 2 sum_{n>=1} J_n^2 (all
    // terms positive, so no cancellation at any x); the sign comes from the
    // larger of the directly evaluated J0(x), J1(x).
    const int N = std::max(m_hi, static_cast<int>(x)) + 60 + static_cast<int>(30.0 * std::cbrt(x + 1.0));
    double jp1 = 0.0, j = 1e-100, S = 0.0;
    std::vector<double> keep(m_hi - m_lo + 1, 0.0);
    std::vector<int> keep_rescales(m_hi - m_lo + 1, 0);
    int rescales = 0;
    double j_at0 = 0.0, j_at1 = 0.0;
    for (int n = N; n >= 0; --n) {
        if (n >= m_lo && n <= m_hi) {
            keep[n - m_lo] = j;
            keep_rescales[n - m_lo] = rescales;
        }
        S += (n == 0 ? 1.0 : 2.0) * j * j;
        if (n == 1) j_at1 = j;
        if (n == 0) { j_at0 = j; break; }
        const double jm1 = (2.0 * n / x) * j - jp1;
        jp1 = j;
        j = jm1;
        if (std::fabs(j) > 1e100) {
            j *= 1e-100;
            jp1 *= 1e-100;
            S *= 1e-200;
            ++rescales;
        }
    }
    double scale = 1.0 / std::sqrt(S);
    const double J0 = bessel_j0(x), J1 = bessel_j1(x);
    const double ref = std::fabs(J0) > std::fabs(J1) ? J0 : J1;
    const double mine = std::fabs(J0) > std::fabs(J1) ? j_at0 : j_at1;
    if ((ref < 0) != (mine < 0)) scale = -scale;
    for (int m = m_lo; m <= m_hi; ++m) {
        double v = keep[m - m_lo] * scale;
        for (int e = keep_rescales[m - m_lo]; e < rescales; ++e) v *= 1e-100;
        out[m - m_lo] = v;
    }
}

double j0_root(int k) {
    // McMahon's expansion as the starting point, then Newton on J0 (J0' = -J1)
    const double beta = (k - 0.25) * kPi;
    const double b8 = 8.0 * beta;
    double x = beta + 1.0 / b8 - 124.0 / (3.0 * b8 * b8 * b8);
    for (int it = 0; it < 50; ++it) {
        const double f = bessel_j0(x);
        const double d = -bessel_j1(x);
        const double dx = f / d;
        x -= dx;
        if (std::fabs(dx) < 1e-16 * x) break;
    }
    return x;
}

double j1_root(int k) {
    // McMahon's expansion (order 1) as the starting point, then Newton on J1 (J1' = J0 - J1 / x)
    const double beta = (k + 0.25) * kPi;
    double x = beta - 3.0 / (8.0 * beta);
    for (int it = 0; it < 50; ++it) {
        const double f = bessel_j1(x);
        const double d = bessel_j0(x) - f / x;
        const double dx = f / d;
        x -= dx;
        if (std::fabs(dx) < 1e-16 * x) break;
    }
    return x;
}

double dini_root(int k, double H) {
    // the k-th positive root of x J1(x) = H J0(x) (H > 0) lies between the (k-1)-th root of J1
    // (0 for k = 1) and the k-th root of J0, where f(x) = x J1(x) - H J0(x) changes sign (the
    // signs at the ends alternate with k): bisection to a narrow bracket, then Newton
    // (f' = x J0(x) + H J1(x)) kept inside it
    double lo = k > 1 ? j1_root(k - 1) : 0.0, hi = j0_root(k);
    auto f = [&](double x) { return x * bessel_j1(x) - H * bessel_j0(x); };
    const double flo = f(lo);
    auto same_as_lo = [&](double v) { return (v < 0.0) == (flo < 0.0); };
    for (int it = 0; it < 40 && hi - lo > 1e-6 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (same_as_lo(f(mid))) lo = mid;
        else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 50; ++it) {
        const double d = x * bessel_j0(x) + H * bessel_j1(x);
        double nx = x - f(x) / d;
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (same_as_lo(f(nx))) lo = nx;
        else hi = nx;
        const bool done = std::fabs(nx - x) < 1e-16 * nx;
        x = nx;
        if (done) break;
    }
    return x;
}

double y0_root(int k) {
    const double beta = (k - 0.75) * kPi;
    const double b8 = 8.0 * beta;
    double x = beta + 1.0 / b8 - 124.0 / (3.0 * b8 * b8 * b8);
    for (int it = 0; it < 50; ++it) {
        const double f = bessel_y0(x);
        const double d = -bessel_y1(x);
        const double dx = f / d;
        x -= dx;
        if (std::fabs(dx) < 1e-16 * x) break;
    }
    return x;
}

double y0_first_root_at_least(double x) {
    int k = std::max(1, static_cast<int>(x / kPi) - 2);
    for (;; ++k) {
        const double r = y0_root(k);
        if (r >= x) return r;
    }
}

}  // namespace sbd
