// Off-line part on the host, FP64 (see offline.h).
//
// SBD fit (Sec. 3.1-3.2): the Gram matrix A^P of the quadratic form Q^P on the
// annulus A(a) uses the explicit formulas of Sec. 3.2 (off-diagonal sign taken
// so that A is the Gram matrix of the integral definition: denominator
// rho_i^2 - rho_j^2); the right-hand side int grad g . grad e_p is in closed
// form (Laplace: -2 pi C_p J0(rho_p a) since J0(rho_p) = 0; Y0: Lommel's
// integral).  A is factored once by a blocked Cholesky at a size above the
// expected P; the Gram matrix of any smaller P is its leading block, so every
// trial P of the search (Sec. 1, dichotomy) reuses the same factor.
#include "offline.h"

#include <deque>
#include <map>
#include <mutex>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>

#include "bessel.h"
#include "sbd.h"

namespace sbd {

// Q-point Gauss-Legendre nodes and weights on [0, a].
void gauss_legendre_0a(int Q, double a, std::vector<double>& s, std::vector<double>& w);

namespace {

constexpr double kPi = 3.14159265358979323846;

std::atomic<int> g_fit_device{0};
std::atomic<int> g_last_where{0};
std::atomic<double> g_last_seconds{0.0};

inline size_t tri(size_t i) { return i * (i + 1) / 2; }   // packed lower row start

// Sample set of [a, 1] for the L_inf stopping test: 512 points a + d (i/511)^2,
// d = min(1 - a, 30 a), and U = 256 + 4 ceil(extra/pi) uniform points.
void fit_samples(double a, double extra, std::vector<double>& s) {
    s.clear();
    const double d = std::min(1.0 - a, 30.0 * a);
    for (int i = 0; i < 512; ++i) {
        const double t = i / 511.0;
        s.push_back(a + d * t * t);
    }
    const int U = 256 + 4 * static_cast<int>(std::ceil(extra / kPi));
    for (int j = 0; j < U; ++j) s.push_back(a + (1.0 - a) * j / (U - 1.0));
}

// Blocked right-looking Cholesky of a packed lower matrix, in place.  Returns the
// number of leading rows factored (P on success; fewer when a pivot is not positive).
int cholesky_packed(std::vector<double>& A, int P) {
    const int nb = 64;
    for (int k0 = 0; k0 < P; k0 += nb) {
        const int kb = std::min(nb, P - k0);
        for (int j = k0; j < k0 + kb; ++j) {
            double d = A[tri(j) + j];
            for (int t = k0; t < j; ++t) d -= A[tri(j) + t] * A[tri(j) + t];
            if (!(d > 0.0)) return j;
            d = std::sqrt(d);
            A[tri(j) + j] = d;
            for (int i = j + 1; i < k0 + kb; ++i) {
                double s = A[tri(i) + j];
                for (int t = k0; t < j; ++t) s -= A[tri(i) + t] * A[tri(j) + t];
                A[tri(i) + j] = s / d;
            }
        }
#pragma omp parallel for schedule(static)
        for (int i = k0 + kb; i < P; ++i) {
            double* ai = &A[tri(i)];
            for (int j = k0; j < k0 + kb; ++j) {
                const double* aj = &A[tri(j)];
                double s = ai[j];
                for (int t = k0; t < j; ++t) s -= ai[t] * aj[t];
                ai[j] = s / aj[j];
            }
        }
#pragma omp parallel for schedule(dynamic, 8)
        for (int i = k0 + kb; i < P; ++i) {
            double* ai = &A[tri(i)];
            for (int j = k0 + kb; j <= i; ++j) {
                const double* aj = &A[tri(j)];
                double s = 0.0;
#pragma omp simd reduction(+ : s)
                for (int t = k0; t < k0 + kb; ++t) s += ai[t] * aj[t];
                ai[j] -= s;
            }
        }
    }
    return P;
}

// Solve (L L^T) x = b with the leading P x P block of a packed factor.
void chol_solve(const std::vector<double>& L, int P, const double* b, std::vector<double>& x) {
    x.assign(b, b + P);
    for (int i = 0; i < P; ++i) {
        const double* li = &L[tri(i)];
        double s = x[i];
        for (int t = 0; t < i; ++t) s -= li[t] * x[t];
        x[i] = s / li[i];
    }
    for (int i = P - 1; i >= 0; --i) {
        const double* li = &L[tri(i)];
        x[i] /= li[i];
        const double xi = x[i];
        for (int t = 0; t < i; ++t) x[t] -= li[t] * xi;
    }
}

struct FitWork {
    int kind;
    double a, kp, extra;
    // general radial kernel (kind 2): h(s) = G(R s) - K(s) - c with K(s) = sum_t kmu_t J0(kom_t s)
    const RadialKernel* rk = nullptr;
    double R = 0.0, c = 0.0;
    std::vector<double> kom, kmu;
    // low-wavenumber Helmholtz: Dini basis (roots of x J1 = H J0), g(s) = Y0(kp s)
    bool robin = false;
    double H = 0.0;
    int Pf = 0, Pok = 0;                 // factored size, usable leading size
    std::vector<double> rho, C, b, L;
    std::vector<double> s, gs;           // samples and g(s)
    std::vector<double> Jmat;            // [sample][p] = J0(rho_p s)
    // Low-rank form of the Gram matrix: A = I - F F^T exactly (to rounding), because the
    // e_p are orthonormal on the unit disk (A(0) = I) and the disk of radius a contributes
    // B_ij = 2 pi C_i C_j rho_i rho_j int_0^a s J1(rho_i s) J1(rho_j s) ds, which a Q-point
    // Gauss-Legendre rule on [0, a] integrates exactly: F_ik = sqrt(2 pi w_k s_k) C_i rho_i
    // J1(rho_i s_k).  A^-1 b = b + F (I - F^T F)^-1 F^T b (Woodbury) costs O(P Q^2) instead
    // of the O(P^3) Cholesky of A.  Near the Gram conditioning floor (Sec. 4.1) the
    // cancellation in I - F^T F costs accuracy, so it is used only for tolerances above it.
    bool lowrank = false;
    int Q = 0;
    std::vector<double> F;               // [p][k], p < Pf, k < Q
};


void build_fit_lowrank(FitWork& w, int Pf);
void radial_rhs(FitWork& w, int Pf);

// rho_p and C_p of the basis: J0 roots with C_p = 1 / (sqrt(pi) rho |J1(rho)|) (Sec. 2.1), or the
// Dini roots with 1 / C_p^2 = 2 pi (rho^2 int_0^1 s J1(rho s)^2 ds + H J0(rho)^2) (Sec. 2.3), the
// integral in closed form (J1'(rho)^2 + (1 - 1 / rho^2) J1(rho)^2) / 2.
void basis_term(const FitWork& w, int p, double& rho, double& C) {
    if (!w.robin) {
        rho = j0_root(p + 1);
        C = 1.0 / (std::sqrt(kPi) * rho * std::fabs(bessel_j1(rho)));
        return;
    }
    rho = dini_root(p + 1, w.H);
    const double j0 = bessel_j0(rho), j1 = bessel_j1(rho), d1 = j0 - j1 / rho;
    const double integ = 0.5 * (d1 * d1 + (1.0 - 1.0 / (rho * rho)) * j1 * j1);
    C = 1.0 / std::sqrt(2.0 * kPi * (rho * rho * integ + w.H * j0 * j0));
}

// h(s) and h'(s) of a general kernel's fit (kind 2)
double radial_h(const FitWork& w, double s) {
    double v = w.rk->value(w.R * s, w.rk->ctx) - w.c;
    for (size_t t = 0; t < w.kom.size(); ++t) v -= w.kmu[t] * bessel_j0(w.kom[t] * s);
    return v;
}
double radial_dh(const FitWork& w, double s) {
    if (w.robin) return -w.kp * bessel_y1(w.kp * s);      // d/ds Y0(kp s)
    double v = w.R * w.rk->deriv(w.R * s, w.rk->ctx);
    for (size_t t = 0; t < w.kom.size(); ++t) v += w.kmu[t] * w.kom[t] * bessel_j1(w.kom[t] * s);
    return v;
}

void build_fit(FitWork& w, int Pf) {
    if (w.lowrank) {
        build_fit_lowrank(w, Pf);
        return;
    }
    w.Pf = Pf;
    w.rho.resize(Pf);
    w.C.resize(Pf);
    w.b.resize(Pf);
    std::vector<double> j0a(Pf), j1a(Pf);
#pragma omp parallel for schedule(dynamic, 64)
    for (int p = 0; p < Pf; ++p) {
        double r, Cp;
        basis_term(w, p, r, Cp);
        w.rho[p] = r;
        w.C[p] = Cp;
        j0a[p] = bessel_j0(r * w.a);
        j1a[p] = bessel_j1(r * w.a);
        if (w.kind == 2 || w.robin) {
            // by quadrature below
        } else if (w.kind == 0) {
            w.b[p] = -2.0 * kPi * w.C[p] * j0a[p];
        } else {
            const double kp = w.kp, a = w.a;
            const double F = a * (r * bessel_y1(kp * a) * j0a[p] - kp * bessel_y0(kp * a) * j1a[p]) /
                             (kp * kp - r * r);
            w.b[p] = -2.0 * kPi * w.C[p] * r * kp * F;
        }
    }
    if (w.kind == 2 || w.robin) radial_rhs(w, Pf);
    // Gram matrix A_ij = int_{A(a)} grad e_i . grad e_j (Sec. 3.2), packed lower.  The closed
    // form is I minus the disk of radius a, as the basis is orthonormal on the unit disk; for the
    // Dini basis that holds in a_H (the gradient term plus H times the boundary term at r = 1).
    w.L.assign(tri(Pf), 0.0);
    const double a = w.a;
#pragma omp parallel for schedule(dynamic, 32)
    for (int i = 0; i < Pf; ++i) {
        const double ri = w.rho[i];
        double* row = &w.L[tri(i)];
        for (int j = 0; j < i; ++j) {
            const double rj = w.rho[j];
            row[j] = 2.0 * kPi * w.C[i] * w.C[j] * ri * rj * a / (ri * ri - rj * rj) *
                     (ri * j0a[i] * j1a[j] - rj * j0a[j] * j1a[i]);
        }
        // diagonal: 2 pi C_i^2 (F_i(1) - F_i(a)), F_i(1) = rho_i^2 J1(rho_i)^2 / 2
        const double x = ri * a;
        const double Fa = x * x * 0.5 * (j0a[i] * j0a[i] + j1a[i] * j1a[i]) - x * j0a[i] * j1a[i];
        row[i] = 1.0 - 2.0 * kPi * w.C[i] * w.C[i] * Fa;
    }
    const auto t0 = std::chrono::steady_clock::now();
    const int mode = fit_device_mode();
    bool done = false;
    if ((mode == 2 || (mode == 0 && Pf >= 3000)) && fit_gpu_available()) {
        std::string err;
        int pok = 0;
        if (gram_cholesky_gpu(w.rho, w.C, j0a, j1a, a, Pf, w.L, &pok, err) == 0) {
            w.Pok = pok;
            done = true;
            g_last_where = 2;
        }
    }
    if (!done) {
        w.Pok = cholesky_packed(w.L, Pf);
        g_last_where = 1;
    }
    g_last_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // J0(rho_p s) for every sample and p < Pf
    const int ns = static_cast<int>(w.s.size());
    w.Jmat.assign(static_cast<size_t>(ns) * Pf, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < ns; ++i) {
        double* Ji = &w.Jmat[static_cast<size_t>(i) * Pf];
        for (int p = 0; p < Pf; ++p) Ji[p] = bessel_j0(w.rho[p] * w.s[i]);
    }
}

// J0(rho_p s) for every sample and p < Pf (shared by both forms)
void fill_jmat(FitWork& w) {
    const int ns = static_cast<int>(w.s.size());
    w.Jmat.assign(static_cast<size_t>(ns) * w.Pf, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < ns; ++i) {
        double* Ji = &w.Jmat[static_cast<size_t>(i) * w.Pf];
        for (int p = 0; p < w.Pf; ++p) Ji[p] = bessel_j0(w.rho[p] * w.s[i]);
    }
}

void build_fit_lowrank(FitWork& w, int Pf) {
    w.Pf = Pf;
    w.rho.resize(Pf);
    w.C.resize(Pf);
    w.b.resize(Pf);
#pragma omp parallel for schedule(dynamic, 64)
    for (int p = 0; p < Pf; ++p) {
        double r, Cp;
        basis_term(w, p, r, Cp);
        w.rho[p] = r;
        w.C[p] = Cp;
        const double j0a = bessel_j0(r * w.a), j1a = bessel_j1(r * w.a);
        if (w.kind == 2 || w.robin) {
            // by quadrature below
        } else if (w.kind == 0) {
            w.b[p] = -2.0 * kPi * w.C[p] * j0a;
        } else {
            const double kp = w.kp, a = w.a;
            const double Fv = a * (r * bessel_y1(kp * a) * j0a - kp * bessel_y0(kp * a) * j1a) / (kp * kp - r * r);
            w.b[p] = -2.0 * kPi * w.C[p] * r * kp * Fv;
        }
    }
    if (w.kind == 2 || w.robin) radial_rhs(w, Pf);
    // the integrand s J1(rho_i s) J1(rho_j s) on [0, a] oscillates at most 2 rho_max a / (2 pi)
    // times: Q = rho_max a + 40 nodes (and at least 64) integrate it to rounding
    w.Q = std::max(64, static_cast<int>(std::ceil(w.rho[Pf - 1] * w.a)) + 40);
    std::vector<double> sq, wq;
    gauss_legendre_0a(w.Q, w.a, sq, wq);
    w.F.assign(static_cast<size_t>(Pf) * w.Q, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
    for (int p = 0; p < Pf; ++p) {
        double* Fp = &w.F[static_cast<size_t>(p) * w.Q];
        for (int k = 0; k < w.Q; ++k)
            Fp[k] = std::sqrt(2.0 * kPi * wq[k] * sq[k]) * w.C[p] * w.rho[p] * bessel_j1(w.rho[p] * sq[k]);
    }
    w.Pok = Pf;
    fill_jmat(w);
}

// alpha = A_P^-1 b_P with A_P = I - F_P F_P^T; false when I - F_P^T F_P is not positive
// definite (beyond the conditioning floor).
bool lowrank_solve(const FitWork& w, int P, std::vector<double>& alpha) {
    const int Q = w.Q;
    std::vector<double> M(static_cast<size_t>(Q) * Q, 0.0), y(Q, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < Q; ++k) {
        for (int l = 0; l <= k; ++l) {
            double g = 0.0;
            for (int p = 0; p < P; ++p) g += w.F[static_cast<size_t>(p) * Q + k] * w.F[static_cast<size_t>(p) * Q + l];
            M[static_cast<size_t>(k) * Q + l] = (k == l ? 1.0 : 0.0) - g;
        }
    }
    for (int k = 0; k < Q; ++k) {
        double t = 0.0;
        for (int p = 0; p < P; ++p) t += w.F[static_cast<size_t>(p) * Q + k] * w.b[p];
        y[k] = t;
    }
    // dense Cholesky of the Q x Q matrix (lower triangle)
    for (int j = 0; j < Q; ++j) {
        double d = M[static_cast<size_t>(j) * Q + j];
        for (int t = 0; t < j; ++t) d -= M[static_cast<size_t>(j) * Q + t] * M[static_cast<size_t>(j) * Q + t];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        M[static_cast<size_t>(j) * Q + j] = d;
        for (int i = j + 1; i < Q; ++i) {
            double v = M[static_cast<size_t>(i) * Q + j];
            for (int t = 0; t < j; ++t) v -= M[static_cast<size_t>(i) * Q + t] * M[static_cast<size_t>(j) * Q + t];
            M[static_cast<size_t>(i) * Q + j] = v / d;
        }
    }
    for (int i = 0; i < Q; ++i) {                       // forward
        double v = y[i];
        for (int t = 0; t < i; ++t) v -= M[static_cast<size_t>(i) * Q + t] * y[t];
        y[i] = v / M[static_cast<size_t>(i) * Q + i];
    }
    for (int i = Q - 1; i >= 0; --i) {                  // backward
        double v = y[i];
        for (int t = i + 1; t < Q; ++t) v -= M[static_cast<size_t>(t) * Q + i] * y[t];
        y[i] = v / M[static_cast<size_t>(i) * Q + i];
    }
    alpha.assign(P, 0.0);
#pragma omp parallel for schedule(static)
    for (int p = 0; p < P; ++p) {
        double v = w.b[p];
        for (int k = 0; k < Q; ++k) v += w.F[static_cast<size_t>(p) * Q + k] * y[k];
        alpha[p] = v;
    }
    return true;
}

double fit_error(const FitWork& w, int P, std::vector<double>& alpha) {
    if (w.lowrank) {
        if (!lowrank_solve(w, P, alpha)) return 1e300;
    } else {
        chol_solve(w.L, P, w.b.data(), alpha);
    }
    const int ns = static_cast<int>(w.s.size());
    double err = 0.0;
#pragma omp parallel for reduction(max : err)
    for (int i = 0; i < ns; ++i) {
        const double* Ji = &w.Jmat[static_cast<size_t>(i) * w.Pf];
        double v = 0.0;
        for (int p = 0; p < P; ++p) v += alpha[p] * w.C[p] * Ji[p];
        err = std::max(err, std::fabs(w.gs[i] - v));
    }
    return err;
}

// 2 sum_{j=1..4} |J_{jM}(r)|, with the j >= 2 terms kept only where they can matter (r < 20).
int circle_size(double r, double weight, double tol) {
    int M0 = std::max(2, 2 * static_cast<int>(std::ceil(0.5 * r)));
    if (weight == 0.0) return M0;
    int span = 64 + static_cast<int>(24.0 * std::cbrt(r + 1.0));
    for (;;) {
        std::vector<double> J;
        bessel_jn_range(r, M0, M0 + span, J);
        for (int M = M0; M <= M0 + span; M += 2) {
            double bound = std::fabs(J[M - M0]);
            if (r < 20.0)
                for (int j = 2; j <= 4; ++j) bound += std::fabs(bessel_jn_small(j * M, r));
            if (2.0 * bound * weight <= tol) return M;
        }
        M0 += span + 1;
        M0 += M0 & 1;
        span *= 2;
    }
}

}  // namespace

bool robin_applies(double k) { return k < 0.5 * y0_root(1); }

int good_fft_size(int n) {
    n = std::max(n, 2);
    for (int c = n + (n & 1);; c += 2) {
        int v = c;
        for (int f : {2, 3, 5})
            while (v % f == 0) v /= f;
        if (v == 1) return c;
    }
}

// Cache of normalised fits.  The P search and the least-squares coefficients depend
// only on the kernel kind, k' (Helmholtz), a = delta_min / scale_R, eps and fixed_P
// (Sec. 3-4: the fit is of g on [a, 1]); a is keyed to a relative resolution of
// 1e-12, far below what moves the fit error at the eps / 3 target.  Process-wide,
// under a lock, at most kFitCacheEntries entries (oldest evicted first).
namespace {
constexpr size_t kFitCacheEntries = 64;
struct FitNorm {
    int P;
    std::vector<double> rho, C, alpha;
    double e;
};
struct FitCache {
    std::mutex mu;
    std::map<FitKey, FitNorm> map;
    std::deque<FitKey> order;
    long long hits = 0, misses = 0;
};
FitCache& fit_cache() {
    static FitCache c;
    return c;
}
}  // namespace

FitKey fit_key(int kind, double kp, double a, double eps, int fixed_P) {
    return FitKey{kind, kp, std::llround(std::log(a) * 1e12), eps, fixed_P};
}

bool fit_cache_get(const FitKey& k, int& P, std::vector<double>& rho, std::vector<double>& C,
                   std::vector<double>& alpha, double& e) {
    FitCache& c = fit_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    auto it = c.map.find(k);
    if (it == c.map.end()) {
        ++c.misses;
        return false;
    }
    ++c.hits;
    P = it->second.P;
    rho = it->second.rho;
    C = it->second.C;
    alpha = it->second.alpha;
    e = it->second.e;
    return true;
}

void fit_cache_put(const FitKey& k, int P, const std::vector<double>& rho, const std::vector<double>& C,
                   const std::vector<double>& alpha, double e) {
    FitCache& c = fit_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    if (c.map.count(k)) return;
    while (c.map.size() >= kFitCacheEntries && !c.order.empty()) {
        c.map.erase(c.order.front());
        c.order.pop_front();
    }
    c.map.emplace(k, FitNorm{P, rho, C, alpha, e});
    c.order.push_back(k);
}

void fit_cache_stats(long long& hits, long long& misses, long long& entries) {
    FitCache& c = fit_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    hits = c.hits;
    misses = c.misses;
    entries = static_cast<long long>(c.map.size());
}

void fit_cache_clear() {
    FitCache& c = fit_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    c.map.clear();
    c.order.clear();
    c.hits = c.misses = 0;
}

namespace {
int offline_fit_impl(int kind, double kappa, const RadialKernel* rk, double delta_min, double delta_max,
                     double eps, int fixed_P, SbdFit& out, std::string& err);
}

int offline_fit(int kind, double kappa, double delta_min, double delta_max, double eps,
                int fixed_P, SbdFit& out, std::string& err) {
    if (kind != 0 && kind != 1) {
        err = "unknown kernel kind";
        return SBD_EINVAL;
    }
    return offline_fit_impl(kind, kappa, nullptr, delta_min, delta_max, eps, fixed_P, out, err);
}

int offline_fit_radial(const RadialKernel& k, double delta_min, double delta_max, double eps, int fixed_P,
                       SbdFit& out, std::string& err) {
    if (!k.value || !k.deriv || (k.n_enforce > 0 && !k.laplacian) || k.n_enforce < 0 || k.n_enforce > 8) {
        err = "radial kernel: value and deriv callbacks, laplacian when n_enforce > 0, n_enforce in [0, 8]";
        return SBD_EINVAL;
    }
    return offline_fit_impl(2, 0.0, &k, delta_min, delta_max, eps, fixed_P, out, err);
}

namespace {
// Sec. 4.3 (the reading of the oracle's R14): lambda_j = Delta_s^j g(1) = R^(2j) (Delta^j G)(R),
// omega' = sqrt of the mean |lambda_{j+1} / lambda_j|, omega_t = the roots of J1 nearest omega',
// and mu solving sum_t (-1)^j omega_t^(2j) mu_t = lambda_j (j = 1..n) by Gaussian elimination
// with partial pivoting; K(s) = sum_t mu_t J0(omega_t s) / J0(omega_t).
int dirichlet_correction(const RadialKernel& k, double R, std::vector<double>& om, std::vector<double>& mu,
                         std::string& err) {
    const int n = k.n_enforce;
    om.clear();
    mu.clear();
    if (n == 0) return SBD_OK;
    std::vector<double> lam(n + 1);
    for (int j = 1; j <= n + 1; ++j) lam[j - 1] = std::pow(R, 2.0 * j) * k.laplacian(j, R, k.ctx);
    double sum = 0.0;
    int cnt = 0;
    for (int j = 0; j < n; ++j)
        if (lam[j] != 0.0) {
            sum += std::fabs(lam[j + 1] / lam[j]);
            ++cnt;
        }
    const double wp = cnt ? std::sqrt(sum / cnt) : 1.0;
    // roots of J1 around wp: the candidates k0 - n .. k0 + n, the n nearest in order
    const int k0 = std::max(1, static_cast<int>(wp / kPi));
    std::vector<double> cand;
    for (int q = std::max(1, k0 - n - 1); q <= k0 + n + 1; ++q) cand.push_back(j1_root(q));
    std::stable_sort(cand.begin(), cand.end(),
                     [&](double x, double y) { return std::fabs(x - wp) < std::fabs(y - wp); });
    om.assign(cand.begin(), cand.begin() + n);
    std::sort(om.begin(), om.end());
    std::vector<double> M(static_cast<size_t>(n) * n), rhs(lam.begin(), lam.begin() + n);
    for (int j = 1; j <= n; ++j)
        for (int t = 0; t < n; ++t) M[(j - 1) * n + t] = ((j & 1) ? -1.0 : 1.0) * std::pow(om[t], 2.0 * j);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[r * n + c]) > std::fabs(M[piv * n + c])) piv = r;
        if (M[piv * n + c] == 0.0) {
            err = "radial kernel: singular Dirichlet correction system";
            return SBD_EFIT;
        }
        for (int t = 0; t < n; ++t) std::swap(M[c * n + t], M[piv * n + t]);
        std::swap(rhs[c], rhs[piv]);
        for (int r = c + 1; r < n; ++r) {
            const double f = M[r * n + c] / M[c * n + c];
            for (int t = c; t < n; ++t) M[r * n + t] -= f * M[c * n + t];
            rhs[r] -= f * rhs[c];
        }
    }
    mu.assign(n, 0.0);
    for (int c = n - 1; c >= 0; --c) {
        double v = rhs[c];
        for (int t = c + 1; t < n; ++t) v -= M[c * n + t] * mu[t];
        mu[c] = v / M[c * n + c];
    }
    return SBD_OK;
}

int offline_fit_impl(int kind, double kappa, const RadialKernel* rk, double delta_min, double delta_max,
                     double eps, int fixed_P, SbdFit& out, std::string& err) {
    if (!(delta_max > 0.0) || !(delta_min > 0.0) || !(delta_min < delta_max)) {
        err = "need 0 < delta_min < delta_max";
        return SBD_EINVAL;
    }
    if (!(eps >= 1e-10 && eps <= 0.1)) {
        err = "eps must lie in [1e-10, 0.1]";
        return SBD_EINVAL;
    }
    if (kind != 0 && kind != 1 && !(kind == 2 && rk)) {
        err = "unknown kernel kind";
        return SBD_EINVAL;
    }
    if (kind == 1 && !(kappa > 0.0)) {
        err = "Helmholtz kernel needs kappa > 0";
        return SBD_EINVAL;
    }
    SbdFit f;
    f.kind = kind;
    f.kappa = kappa;
    f.eps = eps;
    f.delta_min = delta_min;
    f.delta_max = delta_max;
    FitWork w;
    w.kind = kind;
    if (kind == 0) {
        // -log(r)/(2 pi) = -(1/2pi) [log delta_max + log(r / delta_max)]  (Sec. 4.1)
        f.scale_R = delta_max;
        f.gscale = -1.0 / (2.0 * kPi);
        f.w0 = -std::log(delta_max) / (2.0 * kPi);
        w.extra = 0.0;
        w.kp = 0.0;
    } else if (kind == 1 && robin_applies(kappa * delta_max)) {
        // low wavenumber: Y0(kappa r) = Y0(k s), k = kappa delta_max, s = r / delta_max, in the Dini
        // basis of the Robin condition it meets at s = 1, H = k Y1(k) / Y0(k)  (Sec. 2.3, Sec. 4.2)
        const double k = kappa * delta_max;
        f.robin = true;
        f.robin_H = k * bessel_y1(k) / bessel_y0(k);
        f.kprime = k;
        f.scale_R = delta_max;
        f.gscale = -0.25;
        f.w0 = 0.0;
        w.robin = true;
        w.H = f.robin_H;
        w.extra = 2.0 * k;
        w.kp = k;
    } else if (kind == 1) {
        // (i/4) H0(kappa r) = (i/4) J0 - (1/4) Y0; Y0(kappa r) = Y0(k' r / R), R = k'/kappa  (Sec. 4.2)
        f.kprime = y0_first_root_at_least(kappa * delta_max);
        f.scale_R = f.kprime / kappa;
        f.gscale = -0.25;
        f.w0 = 0.0;
        w.extra = 2.0 * f.kprime;
        w.kp = f.kprime;
    } else {
        // general radial kernel (Sec. 4.3): h = g - K - c fitted in kernel units, c at xi = 0
        f.radial = *rk;
        f.scale_R = delta_max;
        f.gscale = 1.0;
        int rc = dirichlet_correction(*rk, delta_max, f.enf_omega, f.enf_mu, err);
        if (rc) return rc;
        w.rk = &f.radial;
        w.R = delta_max;
        w.kom = f.enf_omega;
        w.kmu.resize(f.enf_mu.size());
        double k1 = 0.0;
        for (size_t t = 0; t < f.enf_mu.size(); ++t) {
            w.kmu[t] = f.enf_mu[t] / bessel_j0(f.enf_omega[t]);
            k1 += f.enf_mu[t];                      // K(1)
        }
        w.c = rk->value(delta_max, rk->ctx) - k1;
        if (!std::isfinite(w.c)) {
            err = "radial kernel: G(delta_max) or its iterates are not finite";
            return SBD_EINVAL;
        }
        f.w0 = w.c;
        w.extra = f.enf_omega.empty() ? 0.0 : 2.0 * f.enf_omega.back();
        w.kp = 0.0;
    }
    f.a = delta_min / f.scale_R;
    w.a = f.a;
    const double tol_g = (eps / 3.0) / std::fabs(f.gscale);
    // the low-rank Gram solve for the P search, unless the target is near the
    // conditioning floor (there the factor of the full Gram matrix is more accurate)
    w.lowrank = fixed_P == 0 && tol_g >= 5e-9;
    auto prepare_samples = [&]() {
        fit_samples(f.a, w.extra, w.s);
        w.gs.resize(w.s.size());
        for (size_t i = 0; i < w.s.size(); ++i)
            w.gs[i] = kind == 0 ? std::log(w.s[i]) : kind == 1 ? bessel_y0(w.kp * w.s[i]) : radial_h(w, w.s[i]);
    };

    std::vector<double> alpha;
    int P;
    double e;
    const FitKey key = fit_key(kind, w.kp, f.a, eps, fixed_P);
    if (kind != 2 && fit_cache_get(key, P, f.rho, f.C, alpha, e)) {
        // the search below would give the same normalised fit
    } else if (fixed_P > 0) {
        prepare_samples();
        build_fit(w, fixed_P);
        if (w.Pok < fixed_P) {
            err = "Gram matrix not numerically positive definite at this P (conditioning floor, Sec. 3.3)";
            return SBD_EFIT;
        }
        P = fixed_P;
        e = fit_error(w, P, alpha);
    } else {
        prepare_samples();
        const double gamma = std::max(0.5, (-std::log10(tol_g) - 0.5) / 1.5);
        const int P_start = std::max(2, static_cast<int>(std::ceil(gamma / f.a)) +
                                            static_cast<int>(std::ceil(w.extra / (2.0 * kPi))));
        const int P_max = 20000;
        build_fit(w, std::min(P_max, static_cast<int>(std::ceil(1.25 * P_start)) + 8));
        std::vector<std::pair<int, double>> cache;
        auto err_of = [&](int Pq) -> double {
            for (auto& c : cache)
                if (c.first == Pq) return c.second;
            if (Pq > w.Pok) {
                if (w.Pok < w.Pf) return 1e300;   // beyond the conditioning floor
                build_fit(w, std::min(P_max, static_cast<int>(std::ceil(1.25 * Pq)) + 8));
                cache.clear();
                if (Pq > w.Pok) return 1e300;
            }
            std::vector<double> al;
            const double v = fit_error(w, Pq, al);
            cache.emplace_back(Pq, v);
            return v;
        };
        int lo, hi;
        // start no higher than the factor reaches: near the Gram conditioning floor (Sec. 3.3)
        // the larger factorisation stops early, and the search then proceeds from below
        int Pc = std::max(1, std::min(P_start, w.Pok));
        if (err_of(Pc) > tol_g) {
            lo = Pc;
            hi = static_cast<int>(std::ceil(Pc * 1.1));
            bool found = true;
            while (err_of(hi) > tol_g) {
                if (hi >= P_max || (w.Pok < w.Pf && hi > w.Pok)) {
                    found = false;
                    break;
                }
                lo = hi;
                hi = std::min(P_max, static_cast<int>(std::ceil(hi * 1.1)));
            }
            if (!found) {
                // at the conditioning floor the error stops falling with P (Sec. 3.3): a smaller P
                // whose rounding is lower may still pass; scan down from the start in small steps
                const int step = std::max(1, Pc / 32);
                hi = -1;
                for (int q = Pc - step; q >= 1 && q >= Pc / 2; q -= step)
                    if (err_of(q) <= tol_g) {
                        hi = q;
                        lo = std::max(0, q - step);
                        break;
                    }
                if (hi < 0) {
                    err = "the SBD fit does not reach the tolerance (conditioning floor ~1e-10, Sec. 4.1)";
                    return SBD_EFIT;
                }
            }
        } else {
            hi = Pc;
            lo = static_cast<int>(std::floor(Pc * 0.9));
            while (lo >= 1 && err_of(lo) <= tol_g) {
                hi = lo;
                lo = static_cast<int>(std::floor(lo * 0.9));
            }
            lo = std::max(lo, 0);
        }
        const int res = std::max(1, hi / 128);
        while (hi - lo > res) {
            const int mid = (lo + hi) / 2;
            if (mid >= 1 && err_of(mid) <= tol_g) hi = mid;
            else lo = mid;
        }
        P = hi;
        e = fit_error(w, P, alpha);
    }
    if (static_cast<int>(f.rho.size()) != P) {   // computed here, not taken from the cache
        f.rho.assign(w.rho.begin(), w.rho.begin() + P);
        f.C.assign(w.C.begin(), w.C.begin() + P);
        if (kind != 2) fit_cache_put(key, P, f.rho, f.C, alpha, e);
    }
    f.P = P;
    f.alpha = alpha;
    f.coef.resize(P);
    for (int p = 0; p < P; ++p) f.coef[p] = f.gscale * alpha[p] * f.C[p];
    f.fit_err_g = e;
    f.fit_err = e * std::fabs(f.gscale);
    // circular quadrature sizes (Sec. 5) and weights omega_hat = alpha_p C_p / M_p (Sec. 6.2)
    const int n_enf = static_cast<int>(f.enf_omega.size());
    f.n_circles = P + (kind == 1 ? 1 : 0) + n_enf;
    const double tol_c = (eps / 3.0) / f.n_circles;
    f.M.assign(f.n_circles, 0);
    f.radius.assign(f.n_circles, 0.0);
    f.weight.assign(f.n_circles, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < P; ++p) {
        f.M[p] = circle_size(f.rho[p], std::fabs(f.coef[p]), tol_c);
        f.radius[p] = f.rho[p] / f.scale_R;
        f.weight[p] = f.coef[p] / f.M[p];
    }
    if (kind == 1) {
        const double kd = kappa * delta_max;
        const int Mj = circle_size(kd, 0.25, tol_c);
        f.M[P] = Mj;
        f.radius[P] = kappa;
        f.weight[P] = cplx(0.0, 0.25 / Mj);
    }
    for (int t = 0; t < n_enf; ++t) {
        // K's terms: mu_t / J0(omega_t) J0(omega_t r / delta_max), exact circles (Sec. 1 identity)
        const double wt = f.enf_mu[t] / bessel_j0(f.enf_omega[t]);
        const int Mt = circle_size(f.enf_omega[t], std::fabs(wt), tol_c);
        f.M[P + t] = Mt;
        f.radius[P + t] = f.enf_omega[t] / delta_max;
        f.weight[P + t] = wt / Mt;
    }
    f.n_xi = 0;
    for (int c = 0; c < f.n_circles; ++c) f.n_xi += f.M[c];
    out = std::move(f);
    return SBD_OK;
}
}  // namespace

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from Tricomi's guess).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

void gauss_legendre_0a(int Q, double a, std::vector<double>& s, std::vector<double>& w) {
    std::vector<double> x;
    gauss_legendre(Q, x, w);
    s.resize(Q);
    for (int k = 0; k < Q; ++k) {
        s[k] = 0.5 * a * (x[k] + 1.0);
        w[k] *= 0.5 * a;
    }
}

static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

namespace {
// Composite 24-point Gauss-Legendre rule on [a, b], panels of length <= h growing from a (each
// twice the previous, starting at min(h, a)), so that integrands singular at 0 stay resolved.
void composite_gl(double a, double b, double h, std::vector<double>& s, std::vector<double>& wt) {
    std::vector<double> x, w;
    gauss_legendre(24, x, w);
    s.clear();
    wt.clear();
    double lo = a, step = a > 0.0 ? std::min(h, a) : h;
    while (lo < b) {
        const double hi = std::min(b, lo + step);
        const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
        for (int k = 0; k < 24; ++k) {
            s.push_back(mid + half * x[k]);
            wt.push_back(half * w[k]);
        }
        lo = hi;
        step = std::min(h, 2.0 * step);
    }
}
}  // namespace

namespace {
// b_p = int_{A(a)} grad h . grad e_p = -2 pi C_p rho_p int_a^1 s h'(s) J1(rho_p s) ds for p < Pf
// (Eq. LinearSystem's right-hand side), by the composite rule: the integrand oscillates with
// angular frequency <= rho_max + the correction's largest frequency, and a 24-point panel
// spanning about one period integrates it to rounding.
void radial_rhs(FitWork& w, int Pf) {
    const double fmax = w.rho[Pf - 1] + 0.5 * w.extra;
    std::vector<double> sq, wq;
    composite_gl(w.a, 1.0, std::min(0.125, 3.0 / fmax), sq, wq);
    std::vector<double> hw(sq.size());
    for (size_t k = 0; k < sq.size(); ++k) hw[k] = wq[k] * sq[k] * radial_dh(w, sq[k]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < Pf; ++p) {
        double acc = 0.0;
        for (size_t k = 0; k < sq.size(); ++k) acc += hw[k] * bessel_j1(w.rho[p] * sq[k]);
        w.b[p] = -2.0 * kPi * w.C[p] * w.rho[p] * acc;
        // a_H's boundary term at r = 1: 2 pi H g(1) e_p(1), g(1) = Y0(kp)
        if (w.robin) w.b[p] += 2.0 * kPi * w.H * bessel_y0(w.kp) * w.C[p] * bessel_j0(w.rho[p]);
    }
}
}  // namespace

// Fourier transform of the ES window on [-1, 1]: int exp(beta (sqrt(1 - z^2) - 1)) cos(k z) dz,
// with z = sin(theta) so the integrand is smooth.
static double es_hat(double k, double beta, const std::vector<double>& gx, const std::vector<double>& gw) {
    double s = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
        const double th = 0.5 * kPi * gx[i];
        s += gw[i] * std::exp(beta * (std::cos(th) - 1.0)) * std::cos(k * std::sin(th)) * std::cos(th);
    }
    return 0.5 * kPi * s;
}

static double cheb_eval(const std::vector<double>& c, double x) {
    double b1 = 0.0, b2 = 0.0;
    for (size_t i = c.size() - 1; i >= 1; --i) {
        const double t = 2.0 * x * b1 - b2 + c[i];
        b2 = b1;
        b1 = t;
    }
    return x * b1 - b2 + c[0];
}

// Chebyshev series of log psi(k), psi(k) = 1 / phi_hat(k), in x = 2 (k / kmax)^2 - 1 on
// [0, kmax] (psi is even in k and positive), phi_hat(k) = (P/2) es_hat(k P / 2, beta) the
// Fourier transform of the ES window of width P cells.  The logarithm keeps the relative
// accuracy of psi where it is small (psi spans up to 10^3 over the band for wide windows);
// the degree is doubled until 257 check points agree with the quadrature to 1e-13 (the
// quadrature's own rounding: phi_hat falls to ~1e-3 of its peak at the band edge).
static int es_deconv_series(int P, double beta, double kmax, std::vector<double>& coef, double& psi_max,
                            std::string& err) {
    std::vector<double> gx, gw;
    gauss_legendre(200, gx, gw);
    auto log_psi = [&](double k) { return -std::log(0.5 * P * es_hat(0.5 * P * k, beta, gx, gw)); };
    for (int deg = 24; deg <= 192; deg *= 2) {
        const int nn = deg + 1;
        std::vector<double> fv(nn);
        for (int j = 0; j < nn; ++j) {
            const double x = std::cos(kPi * (j + 0.5) / nn);
            fv[j] = log_psi(kmax * std::sqrt(0.5 * (x + 1.0)));
        }
        coef.assign(nn, 0.0);
        for (int i = 0; i < nn; ++i) {
            double acc = 0.0;
            for (int j = 0; j < nn; ++j) acc += fv[j] * std::cos(kPi * i * (j + 0.5) / nn);
            coef[i] = (i == 0 ? 1.0 : 2.0) * acc / nn;
        }
        double worst = 0.0, most = -1e300;
        bool finite = true;
        for (int t = 0; t <= 256; ++t) {
            const double k = kmax * t / 256.0;
            const double want = log_psi(k);
            if (!std::isfinite(want)) {
                finite = false;
                break;
            }
            const double got = cheb_eval(coef, 2.0 * (k / kmax) * (k / kmax) - 1.0);
            worst = std::max(worst, std::fabs(got - want));
            most = std::max(most, want);
        }
        if (!finite) break;
        if (worst <= 1e-13) {
            psi_max = std::exp(most);
            return SBD_OK;
        }
    }
    err = "the ES deconvolution series does not reach 1e-13";
    return SBD_ENOTSUP;
}

int nufft_params(const SbdFit& fit, double half_extent, double cx, double cy, double tol,
                 bool fp32, int kwin, int swin, int sigma_mode, long n_points, NufftParams& o,
                 std::string& err) {
    double S = 0.0;
    for (int c = 0; c < fit.n_circles; ++c) S = std::max(S, fit.radius[c]);
    if (!(S > 0.0) || !(half_extent > 0.0)) {
        err = "degenerate geometry for the transform";
        return SBD_EINVAL;
    }
    if (fp32) tol = std::max(tol, 3e-7);
    tol = std::max(tol, 1e-15);
    const int pmax = fp32 ? 16 : 32;
    // Oversampling of the spreading grid (spacing h = pi / (sigma S)): 2, or 1.5 with the ES
    // window, which shrinks the spreading grid and the FFT rows by a quarter for a wider
    // stencil.  Automatic: 1.5 where the grid of sigma = 2 has more than 20 cells per point
    // (there the transforms outweigh the point stencils; measured break-even on GB300).
    double sig = 2.0;
    if (swin == 1) {
        if (sigma_mode == 1) {
            sig = 1.5;
        } else if (sigma_mode == 3) {
            sig = 1.25;
        } else if (sigma_mode == 0) {
            // cells per point of the grid at sigma = 2: past 20 the transforms outweigh the point
            // stencils (1.5), past 60 by far (1.25: N = 10^6 on the curves, 120 cells per point,
            // 8.19 -> 7.68 ms against 1.5)
            const double m2 = 2.0 * half_extent * (2.0 * S) / kPi;   // cells per side at sigma = 2
            const double cells = m2 * m2 / static_cast<double>(n_points);
            if (cells > 60.0) sig = 1.25;
            else if (cells > 20.0) sig = 1.5;
        }
    }
    // spreading side: ES error ~ 10 exp(-pi P sqrt(1 - 1 / sigma)) (10^-(P - 1) at sigma = 2);
    // Gaussian ~ 0.1 exp(-pi P / 3) at sigma = 2
    int Ps;
    if (swin == 1) {
        Ps = static_cast<int>(std::ceil(std::log(10.0 / tol) / (kPi * std::sqrt(1.0 - 1.0 / sig))));
    } else {
        Ps = static_cast<int>(std::ceil((3.0 / kPi) * std::log(0.1 / tol)));
    }
    Ps = std::max(4, std::min(pmax, Ps + (Ps & 1)));
    // node side: ES error ~ 10^-P (two-fold oversampling), Gaussian as the spreading side
    int Pk;
    if (kwin == 1) {
        Pk = static_cast<int>(std::ceil(-std::log10(tol)));
        Pk = std::max(4, std::min(pmax, Pk + (Pk & 1)));
    } else {
        Pk = static_cast<int>(std::ceil((3.0 / kPi) * std::log(0.1 / tol)));
        Pk = std::max(4, std::min(pmax, Pk + (Pk & 1)));
    }
    o.Ps = Ps;
    o.Pk = Pk;
    o.kwin = kwin;
    o.swin = swin;
    o.tol = tol;
    o.sigma_s = sig;
    o.h = kPi / (sig * S);
    if (swin == 1) {
        o.tau = 0.0;
        o.beta_s = 2.3 * Ps * (1.0 - 0.5 / sig) / 0.75;   // 2.3 P at sigma = 2
    } else {
        const double u = Ps * kPi / 24.0;   // balanced truncation / aliasing of the Gaussian at two-fold oversampling
        o.tau = u / (S * S);
        o.beta_s = o.h * o.h / (4.0 * o.tau);
    }
    o.m = good_fft_size(static_cast<int>(std::ceil(2.0 * half_extent / o.h)) + Ps + 4);
    o.n = 2 * o.m;
    const double Xg = 0.5 * o.m * o.h;
    o.deta = 2.0 * kPi / (o.n * o.h);
    {
        // stored frequency grid: every node (|xi| <= S) with its stencil; m + Pk + 4 at sigma = 2
        const int nk = static_cast<int>(std::ceil(2.0 * S / o.deta - 1e-9)) + Pk + 4;
        o.nk = nk + (nk & 1);
    }
    if (o.nk > o.n) {
        // a very small grid: the node stencils at sigma < 2 reach past the FFT length
        if (sigma_mode == 0 && sig != 2.0)
            return nufft_params(fit, half_extent, cx, cy, tol, fp32, kwin, swin, sig < 1.5 ? 1 : 2, n_points, o,
                                err) == SBD_OK
                       ? SBD_OK
                       : nufft_params(fit, half_extent, cx, cy, tol, fp32, kwin, swin, 2, n_points, o, err);
        err = "the frequency grid exceeds the FFT length (grid too small for this oversampling)";
        return SBD_ENOTSUP;
    }
    o.cx = cx;
    o.cy = cy;
    o.dec.resize(o.m);
    double knode;   // node-side constant of the per-node scale c(xi)
    if (kwin == 1) {
        o.beta_k = 2.3 * Pk;
        o.sigma = 0.0;
        const double half = 0.5 * Pk * o.deta;
        std::vector<double> gx, gw;
        gauss_legendre(160, gx, gw);
        for (int i = 0; i < o.m; ++i) {
            const double x = (i - 0.5 * o.m) * o.h;
            o.dec[i] = 1.0 / (half * es_hat(x * half, o.beta_k, gx, gw));
        }
        knode = o.deta * o.deta;
    } else {
        const double v = Pk * kPi / 24.0;
        o.sigma = v / (Xg * Xg);
        o.beta_k = o.deta * o.deta / (4.0 * o.sigma);
        for (int i = 0; i < o.m; ++i) {
            const double x = (i - 0.5 * o.m) * o.h;
            o.dec[i] = std::exp(o.sigma * x * x);
        }
        knode = o.deta * o.deta / (4.0 * kPi * o.sigma);
    }
    o.circle_factor.resize(fit.n_circles);
    o.psi.clear();
    o.kmax = 0.0;
    o.psi_max = 1.0;
    if (swin == 1) {
        // c(xi) = knode psi(xi_x h) psi(xi_y h): the circle keeps knode^2, the node the rest
        for (int c = 0; c < fit.n_circles; ++c) o.circle_factor[c] = knode * knode;
        o.kmax = S * o.h * (1.0 + 1e-12);
        int rc = es_deconv_series(Ps, o.beta_s, o.kmax, o.psi, o.psi_max, err);
        // automatic oversampling below 2 whose window series cannot be set up: 1.5, then 2
        if (rc && sigma_mode == 0 && sig < 1.5 &&
            nufft_params(fit, half_extent, cx, cy, tol, fp32, kwin, swin, 1, n_points, o, err) == SBD_OK)
            return SBD_OK;
        if (rc && sigma_mode == 0 && sig != 2.0)
            return nufft_params(fit, half_extent, cx, cy, tol, fp32, kwin, swin, 2, n_points, o, err);
        if (rc) return rc;
    } else {
        // c(|xi|) = knode h^2 exp(tau |xi|^2) / (4 pi tau), radial: one factor per circle
        const double c0 = knode * o.h * o.h / (4.0 * kPi * o.tau);
        for (int c = 0; c < fit.n_circles; ++c)
            o.circle_factor[c] = c0 * c0 * std::exp(2.0 * o.tau * fit.radius[c] * fit.radius[c]);
    }
    return SBD_OK;
}

int uniform_params(const SbdFit& fit, double half_extent, double cx, double cy, double tol, bool fp32, int swin,
                   int sigma_mode, long n_points, NufftParams& o, std::string& err) {
    double S = 0.0;
    for (int c = 0; c < fit.n_circles; ++c) S = std::max(S, fit.radius[c]);
    if (!(S > 0.0) || !(half_extent > 0.0)) {
        err = "degenerate geometry for the transform";
        return SBD_EINVAL;
    }
    if (fp32) tol = std::max(tol, 3e-7);
    tol = std::max(tol, 1e-15);
    // window of the periodised series: flat on the differences of the points (|t| <= 2 half),
    // an ES-bump transition over a tenth of that; its spectrum reaches B = 2 beta / tau
    o.uniform = true;
    o.wa = 2.0 * half_extent;
    o.wtau = 0.1 * o.wa;
    o.wbeta = std::max(8.0, 1.1 * std::log(1.0 / tol));
    const double B = 2.0 * o.wbeta / o.wtau;
    o.kcut = S + B;
    // spreading: the rules of nufft_params, with K in place of S
    double sig = 2.0;
    if (swin == 1) {
        if (sigma_mode == 1) {
            sig = 1.5;
        } else if (sigma_mode == 3) {
            sig = 1.25;
        } else if (sigma_mode == 0) {
            const double m2 = 2.0 * half_extent * (2.0 * o.kcut) / kPi;
            const double cells = m2 * m2 / static_cast<double>(n_points);
            if (cells > 60.0) sig = 1.25;
            else if (cells > 20.0) sig = 1.5;
        }
    }
    const int pmax = fp32 ? 16 : 32;
    int Ps;
    if (swin == 1) Ps = static_cast<int>(std::ceil(std::log(10.0 / tol) / (kPi * std::sqrt(1.0 - 1.0 / sig))));
    else Ps = static_cast<int>(std::ceil((3.0 / kPi) * std::log(0.1 / tol)));
    Ps = std::max(4, std::min(pmax, Ps + (Ps & 1)));
    o.Ps = Ps;
    o.Pk = 0;
    o.kwin = 1;
    o.swin = swin;
    o.tol = tol;
    o.sigma_s = sig;
    o.h = kPi / (sig * o.kcut);
    if (swin == 1) {
        o.tau = 0.0;
        o.beta_s = 2.3 * Ps * (1.0 - 0.5 / sig) / 0.75;
    } else {
        const double u = Ps * kPi / 24.0;
        o.tau = u / (o.kcut * o.kcut);
        o.beta_s = o.h * o.h / (4.0 * o.tau);
    }
    o.m = good_fft_size(static_cast<int>(std::ceil(2.0 * half_extent / o.h)) + Ps + 4);
    o.n = good_fft_size(std::max(o.m + Ps + 4, static_cast<int>(std::ceil(2.0 * (o.wa + o.wtau) / o.h)) + 2));
    o.deta = 2.0 * kPi / (o.n * o.h);
    {
        const int nk = 2 * static_cast<int>(std::ceil(o.kcut / o.deta)) + 2;
        o.nk = nk + (nk & 1);
    }
    if (o.nk > o.n) {
        if (sigma_mode == 0 && sig != 2.0)
            return uniform_params(fit, half_extent, cx, cy, tol, fp32, swin, sig < 1.5 ? 1 : 2, n_points, o, err) ==
                           SBD_OK
                       ? SBD_OK
                       : uniform_params(fit, half_extent, cx, cy, tol, fp32, swin, 2, n_points, o, err);
        err = "uniform grid: the frequency window exceeds the FFT length";
        return SBD_ENOTSUP;
    }
    o.cx = cx;
    o.cy = cy;
    o.dec.assign(o.m, 1.0);           // no node window: nothing to precorrect on the spreading grid
    o.beta_k = 0.0;
    o.sigma = 0.0;
    o.circle_factor.assign(fit.n_circles, 1.0);
    o.psi.clear();
    o.kmax = 0.0;
    o.psi_max = 1.0;
    if (swin == 1) {
        o.kmax = o.kcut * o.h * (1.0 + 1e-12);
        int rc = es_deconv_series(Ps, o.beta_s, o.kmax, o.psi, o.psi_max, err);
        // as nufft_params: automatic oversampling falls back to 1.5, then 2
        if (rc && sigma_mode == 0 && sig < 1.5 &&
            uniform_params(fit, half_extent, cx, cy, tol, fp32, swin, 1, n_points, o, err) == SBD_OK)
            return SBD_OK;
        if (rc && sigma_mode == 0 && sig != 2.0)
            return uniform_params(fit, half_extent, cx, cy, tol, fp32, swin, 2, n_points, o, err);
        if (rc) return rc;
    }
    // psi_w at the FFT positions: 1 - (integral of the ES bump over [0, (|t| - wa) / wtau]) / (its total)
    std::vector<double> gx, gw;
    gauss_legendre(64, gx, gw);
    auto bump = [&](double u) { const double v = 2.0 * u - 1.0; return std::exp(o.wbeta * (std::sqrt(std::max(0.0, 1.0 - v * v)) - 1.0)); };
    // the integral over [0, 1] in 8 panels (the bump is peaked)
    double total = 0.0;
    for (int k = 0; k < 8; ++k) {
        double acc = 0.0;
        for (size_t j = 0; j < gx.size(); ++j) acc += gw[j] * bump((k + 0.5 * (gx[j] + 1.0)) / 8.0);
        total += acc / 16.0;
    }
    o.wtab.resize(o.n);
    for (int i = 0; i < o.n; ++i) {
        const double t = std::fabs((i - 0.5 * o.n) * o.h);
        if (t <= o.wa) o.wtab[i] = 1.0;
        else if (t >= o.wa + o.wtau) o.wtab[i] = 0.0;
        else {
            const double u = (t - o.wa) / o.wtau;
            // piecewise: panels of 1/8 below u, Gauss-Legendre on each
            double acc = 0.0;
            const int full = static_cast<int>(u * 8.0);
            for (int k = 0; k < full; ++k) {
                double pa = 0.0;
                for (size_t j = 0; j < gx.size(); ++j) pa += gw[j] * bump((k + 0.5 * (gx[j] + 1.0)) / 8.0);
                acc += pa / 16.0;
            }
            const double u0 = full / 8.0, du = u - u0;
            if (du > 0.0) {
                double pa = 0.0;
                for (size_t j = 0; j < gx.size(); ++j) pa += gw[j] * bump(u0 + 0.5 * du * (gx[j] + 1.0));
                acc += 0.5 * du * pa;
            }
            o.wtab[i] = std::max(0.0, std::min(1.0, 1.0 - acc / total));
        }
    }
    return SBD_OK;
}

int near_tables(const SbdFit& fit, NearTables& o, std::string& err, bool radial) {
    const double dmin = fit.delta_min;
    // tables in t = r^2 (the kernels' smooth parts are even in r), or in r for a general kernel
    o.in_r = fit.kind == 2;
    o.tmax = o.in_r ? dmin : dmin * dmin;
    double scale = std::abs(fit.w0);
    for (int p = 0; p < fit.P; ++p) scale += std::fabs(fit.coef[p]);
    scale = std::max(1.0, scale);
    // circles whose aliasing terms (Sec. 5) are not negligible within delta_min
    o.small.clear();
    double phase = 0.0;
    bool j0_circle_small = false;
    for (int c = 0; c < fit.n_circles; ++c) {
        const double x = fit.radius[c] * dmin;
        phase = std::max(phase, x);
        std::vector<double> J;
        bessel_jn_range(x, fit.M[c], fit.M[c], J);
        const double mag = 2.0 * std::fabs(J[0]) * std::abs(fit.weight[c]) * fit.M[c];
        if (!radial && mag > 1e-18 * scale) {
            o.small.push_back(c);
            if (fit.kind == 1 && c == fit.P) j0_circle_small = true;
        }
    }
    std::vector<char> is_small(fit.n_circles, 0);
    for (int c : o.small) is_small[c] = 1;
    auto T1f = [&](double u) -> cplx {
        if (fit.kind == 0) return -1.0 / (2.0 * kPi);
        if (fit.kind == 2) return fit.radial.log_coef;
        return -bessel_j0(fit.kappa * std::sqrt(u)) / (2.0 * kPi);
    };
    auto T2f = [&](double u) -> cplx {
        const double r = o.in_r ? u : std::sqrt(u);
        cplx v = 0.0;
        if (fit.kind == 2) {
            // G - c log r, smooth at 0, minus the series of every circle not summed exactly
            v = fit.radial.value(r, fit.radial.ctx) - fit.radial.log_coef * std::log(r) - fit.w0;
            for (int c = 0; c < fit.n_circles; ++c)
                if (!is_small[c]) v -= fit.weight[c] * static_cast<double>(fit.M[c]) * bessel_j0(fit.radius[c] * r);
            return v;
        }
        if (fit.kind == 0) {
            v = -fit.w0;
        } else {
            const double x = fit.kappa * r;
            const double j0 = bessel_j0(x);
            const double yreg = x > 0.0 ? bessel_y0_regular(x) : (2.0 / kPi) * 0.57721566490153286061;
            v = -std::log(0.5 * fit.kappa) * j0 / (2.0 * kPi) - 0.25 * yreg;
            if (j0_circle_small) v += cplx(0.0, 0.25 * j0);
        }
        for (int p = 0; p < fit.P; ++p)
            if (!is_small[p]) v -= fit.coef[p] * bessel_j0(fit.rho[p] * r / fit.scale_R);
        return v;
    };
    o.deg = 18;
    o.pieces = std::max(2, static_cast<int>(std::ceil(phase / 2.0)));
    // Refinement aims at 1e-14 x scale.  With thousands of terms the direct evaluation
    // that checks the table has a rounding floor of a few 1e-14; once refining stops
    // helping, a table within 1e-3 eps (a negligible share of the eps bound on q) is kept.
    const double accept = std::max(1e-14 * scale, 1e-3 * fit.eps);
    double prev_worst = 1e300;
    for (int attempt = 0; attempt < 6; ++attempt) {
        const int K = o.pieces, D = o.deg;
        o.T1.assign(static_cast<size_t>(K) * D * 2, 0.0);
        o.T2.assign(static_cast<size_t>(K) * D * 2, 0.0);
        const double wdt = o.tmax / K;
#pragma omp parallel for schedule(dynamic, 1)
        for (int q = 0; q < K; ++q) {
            std::vector<cplx> f1(D), f2(D);
            for (int k = 0; k < D; ++k) {
                const double tt = std::cos(kPi * (k + 0.5) / D);
                const double t = (q + 0.5 * (tt + 1.0)) * wdt;
                f1[k] = T1f(t);
                f2[k] = T2f(t);
            }
            for (int j = 0; j < D; ++j) {
                cplx s1 = 0.0, s2 = 0.0;
                for (int k = 0; k < D; ++k) {
                    const double c = std::cos(kPi * j * (k + 0.5) / D);
                    s1 += f1[k] * c;
                    s2 += f2[k] * c;
                }
                const double sc = (j == 0 ? 1.0 : 2.0) / D;
                o.T1[(static_cast<size_t>(q) * D + j) * 2 + 0] = (s1 * sc).real();
                o.T1[(static_cast<size_t>(q) * D + j) * 2 + 1] = (s1 * sc).imag();
                o.T2[(static_cast<size_t>(q) * D + j) * 2 + 0] = (s2 * sc).real();
                o.T2[(static_cast<size_t>(q) * D + j) * 2 + 1] = (s2 * sc).imag();
            }
        }
        // check against direct evaluation between the interpolation points
        double worst = 0.0;
        for (int q = 0; q < K; ++q) {
            for (int k = 0; k < 7; ++k) {
                const double tt = -1.0 + 2.0 * (k + 0.37) / 7.0;
                const double t = (q + 0.5 * (tt + 1.0)) * wdt;
                cplx b1 = 0.0, b2 = 0.0, c1 = 0.0, c2 = 0.0;
                for (int j = D - 1; j >= 1; --j) {
                    const cplx a1(o.T1[(q * D + j) * 2], o.T1[(q * D + j) * 2 + 1]);
                    const cplx a2(o.T2[(q * D + j) * 2], o.T2[(q * D + j) * 2 + 1]);
                    const cplx n1 = 2.0 * tt * b1 - c1 + a1;
                    const cplx n2 = 2.0 * tt * b2 - c2 + a2;
                    c1 = b1; b1 = n1;
                    c2 = b2; b2 = n2;
                }
                const cplx v1 = tt * b1 - c1 + cplx(o.T1[q * D * 2], o.T1[q * D * 2 + 1]);
                const cplx v2 = tt * b2 - c2 + cplx(o.T2[q * D * 2], o.T2[q * D * 2 + 1]);
                worst = std::max(worst, std::abs(v1 - T1f(t)) + std::abs(v2 - T2f(t)));
            }
        }
        if (worst <= 1e-14 * scale) break;
        if (worst <= accept && (attempt == 5 || worst > 0.5 * prev_worst)) break;   // at the rounding floor
        prev_worst = worst;
        if (attempt == 5) {
            char buf[128];
            std::snprintf(buf, sizeof buf, "near-field table does not converge (%.3g)", worst);
            err = buf;
            return SBD_EFIT;
        }
        o.pieces *= 2;
    }
    cplx g0 = fit.w0;
    for (int c = 0; c < fit.n_circles; ++c) g0 += fit.weight[c] * static_cast<double>(fit.M[c]);
    o.self_value = -g0;
    return SBD_OK;
}

void set_fit_device(int mode) { g_fit_device = mode; }
int fit_device_mode() { return g_fit_device; }
void last_factorisation(double* seconds, int* where) {
    if (seconds) *seconds = g_last_seconds;
    if (where) *where = g_last_where;
}

}  // namespace sbd
