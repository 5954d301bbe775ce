// Off-line part on the host (FP64): SBD fit, P search, circular quadrature sizes,
// weights, type-3 transform parameters and the near-field tables.
#pragma once
#include <complex>
#include <string>
#include <vector>

namespace sbd {

using cplx = std::complex<double>;

// A general real radial kernel (Sec. 4.3) given on the host by callbacks, which are called
// only while a plan is built: value(r) = G(r) and deriv(r) = G'(r) for r > 0, laplacian(j, r)
// = (Delta^j G)(r) for j >= 1 (Delta the radial Laplacian), log_coef = c with G - c log r
// smooth at 0, and n_enforce the number of iterates the multi-Dirichlet correction enforces.
struct RadialKernel {
    double (*value)(double r, void* ctx) = nullptr;
    double (*deriv)(double r, void* ctx) = nullptr;
    double (*laplacian)(int j, double r, void* ctx) = nullptr;
    void* ctx = nullptr;
    double log_coef = 0.0;
    int n_enforce = 0;
};

struct SbdFit {
    int kind = 0;            // 0 Laplace, 1 Helmholtz, 2 general radial (Sec. 4.3)
    double kappa = 0.0;
    double eps = 0.0;
    double delta_min = 0.0, delta_max = 0.0;
    double scale_R = 0.0;    // delta_max (Laplace) or k'/kappa (Helmholtz Y0 part)
    double a = 0.0;          // delta_min / scale_R
    double kprime = 0.0;     // k' for Helmholtz
    double gscale = 0.0;     // kernel = gscale * g(r / scale_R) + ...
    int P = 0;
    int n_circles = 0;       // P (+1 Helmholtz J0 circle, stored last)
    std::vector<double> rho, C, alpha;   // per Bessel term (size P)
    std::vector<double> coef;            // gscale * alpha_p * C_p (kernel units), size P
    std::vector<int> M;                  // nodes per circle, size n_circles
    std::vector<double> radius;          // circle radius in frequency units, size n_circles
    std::vector<cplx> weight;            // omega_hat per node of the circle, size n_circles
    cplx w0 = 0.0;                       // weight of the xi = 0 node
    double fit_err_g = 0.0;              // L_inf fit error of g on the sample set
    double fit_err = 0.0;                // the same in kernel units
    long long n_xi = 0;                  // sum M
    // general radial kernel: the callbacks (valid while the plan is built) and the correction
    // K(s) = sum_t enf_mu_t J0(enf_omega_t s) / J0(enf_omega_t), s = r / scale_R (Sec. 4.3)
    RadialKernel radial;
    std::vector<double> enf_omega, enf_mu;
    // low-wavenumber Helmholtz (kind 1): the Dini basis of the Robin condition with constant
    // robin_H, at scale_R = delta_max (Sec. 2.3, Sec. 4.2)
    bool robin = false;
    double robin_H = 0.0;
};

// Sec. 4.2, third case: the Dini (Robin) series is used for Y0(kappa r) when kappa delta_max is
// below half the first root of Y0.
bool robin_applies(double k);

// The Gram matrix of Eq. LinearSystem built and Cholesky-factored on the GPU (fit_gpu.cu):
// packed receives the lower factor in the host's packed layout (row i at i (i + 1) / 2), *Pok
// the number of leading rows factored (P, or the first non-positive pivot).
int gram_cholesky_gpu(const std::vector<double>& rho, const std::vector<double>& C, const std::vector<double>& j0a,
                      const std::vector<double>& j1a, double a, int P, std::vector<double>& packed, int* Pok,
                      std::string& err);
bool fit_gpu_available();
// Where the fit's full Cholesky runs: 0 the device for P >= 3000 when one is present, else the
// host; 1 always the host; 2 the device when present (sbd_set_fit_device).
void set_fit_device(int mode);
int fit_device_mode();
// Seconds of the last full factorisation and where it ran (1 host, 2 device); for tests.
void last_factorisation(double* seconds, int* where);

// The fit of a general real radial kernel (Sec. 4.3 with Sec. 3): the correction K and the
// constant c enforce the multi-Dirichlet condition up to order n_enforce at r = delta_max, the
// SBD fits h = g - K - c (g(s) = G(delta_max s)); circles: P Bessel terms, then the n_enforce
// terms of K; w0 = c.  Not cached (the callbacks are arbitrary).
int offline_fit_radial(const RadialKernel& k, double delta_min, double delta_max, double eps, int fixed_P,
                       SbdFit& out, std::string& err);

// Key of the normalised-fit cache used by offline_fit (see offline.cpp).
struct FitKey {
    int kind;
    double kp;
    long long a_q;
    double eps;
    int fixed_P;
    bool operator<(const FitKey& o) const {
        if (kind != o.kind) return kind < o.kind;
        if (kp != o.kp) return kp < o.kp;
        if (a_q != o.a_q) return a_q < o.a_q;
        if (eps != o.eps) return eps < o.eps;
        return fixed_P < o.fixed_P;
    }
};
FitKey fit_key(int kind, double kp, double a, double eps, int fixed_P);
bool fit_cache_get(const FitKey& k, int& P, std::vector<double>& rho, std::vector<double>& C,
                   std::vector<double>& alpha, double& e);
void fit_cache_put(const FitKey& k, int P, const std::vector<double>& rho, const std::vector<double>& C,
                   const std::vector<double>& alpha, double e);
void fit_cache_stats(long long& hits, long long& misses, long long& entries);
void fit_cache_clear();

// Fit for the given geometry bound; fixed_P > 0 skips the P search.
// Returns 0, or a negative SBD_E* code with a message in err.
int offline_fit(int kind, double kappa, double delta_min, double delta_max, double eps,
                int fixed_P, SbdFit& out, std::string& err);

// Parameters of the type-3 transform: spreading of the points with an ES (exponential of
// semicircle) or Gaussian window on a spreading grid oversampled 1.5- or 2-fold, a two-fold
// zero-padded FFT, and a node window that is ES or Gaussian.
struct NufftParams {
    int Ps = 0, Pk = 0;        // stencil widths (cells per dimension, even)
    int kwin = 1;              // node window: 0 Gaussian, 1 ES
    int swin = 1;              // spreading window: 0 Gaussian, 1 ES
    double h = 0.0;            // spreading-grid spacing pi / (sigma_s S)
    double sigma_s = 2.0;      // oversampling of the spreading grid (2, or 1.5 with the ES window)
    int m = 0;                 // spreading-grid side (cells), even, 5-smooth
    int n = 0;                 // FFT length = 2 m
    int nk = 0;                // stored frequency-grid side (cells), even: 2 S / deta + Pk + 4
    double deta = 0.0;         // frequency-grid spacing 2 pi / (n h)
    double tau = 0.0, sigma = 0.0;
    double beta_s = 0.0;       // spreading window: Gaussian h^2 / (4 tau) (weight exp(-beta_s d^2), d in
                               // cells), ES 2.3 Ps
    double beta_k = 0.0;       // node window: Gaussian deta^2 / (4 sigma), ES 2.3 Pk
    double cx = 0.0, cy = 0.0; // centre of the point set (bounding box)
    double tol = 0.0;          // tolerance aimed at for each transform
    std::vector<double> dec;   // spreading-grid precorrection 1 / psi_hat(x_i) (one dimension), size m
    std::vector<double> circle_factor;   // c(|xi|)^2 per circle, c = h^2 deta^2 exp(tau |xi|^2) / (4 pi tau) [x Gaussian 1/(4 pi sigma)]
                                         // for the Gaussian spreading window; deta^4 [/(4 pi sigma)^2] for ES,
                                         // whose deconvolution is a per-node factor (psi below)
    // ES spreading window: psi(k) = 1 / phi_hat_s(k), phi_hat_s(k) = integral over the window of
    // exp(-i k d) (d in cells, k = xi h in [0, kmax], kmax = S h = pi / sigma_s); log psi as a
    // Chebyshev series in 2 (k / kmax)^2 - 1; the node xi = (xi_x, xi_y) takes the factor
    // psi(xi_x h) psi(xi_y h).
    std::vector<double> psi;
    double kmax = 0.0;
    double psi_max = 1.0;      // psi(kmax), the largest value of psi on [0, kmax]
    // Uniform-grid variant (uniform_params): the series G_fit, windowed by psi_w(y_x) psi_w(y_y)
    // and periodised on the FFT period L = n h, enters as Fourier coefficients on the frequency
    // grid; psi_w = 1 on |t| <= wa (the points' differences), 0 beyond wa + wtau, an ES bump's
    // integral in between.
    bool uniform = false;
    double wa = 0.0, wtau = 0.0, wbeta = 0.0;
    double kcut = 0.0;         // largest frequency kept, S + the window's spectral reach
    std::vector<double> wtab;  // psi_w at the n FFT positions, t = (i - n / 2) h
};

// Parameters of the uniform-grid variant (the fast summation the paper cites: the node step
// replaced by a multiplication on the frequency grid): same spreading windows and rules as
// nufft_params; the spreading grid resolves K = S + B, B the spectral reach of the window
// psi_w; the FFT length n covers the period L >= 2 (2 half + wtau) so that the periodised
// window never overlaps itself on the points' differences; nk covers |k| <= K.
int uniform_params(const SbdFit& fit, double half_extent, double cx, double cy, double tol, bool fp32, int swin,
                   int sigma_mode, long n_points, NufftParams& out, std::string& err);

// sigma_mode: 0 automatic, 1 spreading oversampling 1.5, 2 oversampling 2 (the Gaussian
// spreading window always uses 2); n_points feeds the automatic choice.
int nufft_params(const SbdFit& fit, double half_extent, double cx, double cy, double tol,
                 bool fp32, int kwin, int swin, int sigma_mode, long n_points, NufftParams& out,
                 std::string& err);

// Smallest even 5-smooth integer >= n.
int good_fft_size(int n);

// Near-field tables: D(y) = T1(t) * 0.5 log t + T2(t) - sum_{small circles} w_p sum_m e^{i y.xi},
// t = |y|^2 in [0, delta_min^2]; T1, T2 piecewise Chebyshev in t (complex, re/im interleaved).
struct NearTables {
    int pieces = 0, deg = 0;
    double tmax = 0.0;               // table range: r^2 in [0, tmax], or r in [0, tmax] when in_r
    bool in_r = false;               // tables in r (general kernels, whose smooth part may be odd in r)
    std::vector<double> T1, T2;      // [pieces][deg][2]
    std::vector<int> small;          // circles whose plane-wave sum is evaluated exactly
    cplx self_value = 0.0;           // D_kk = -G_approx(0)
};

// radial: every circle enters as its exact J0 term (no plane-wave sums): D = G - G_fit for the
// uniform-grid variant, whose far part uses the series without the circle quadrature.
int near_tables(const SbdFit& fit, NearTables& out, std::string& err, bool radial = false);

}  // namespace sbd
