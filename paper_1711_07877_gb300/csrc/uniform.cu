// Uniform-grid multiplier variant: plan-time Fourier coefficients of the windowed, periodised
// series G_fit and the on-line multiplication on the frequency grid (see uniform.cuh).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fft.cuh"
#include "sbd.h"
#include "uniform.cuh"

namespace sbd {

namespace {

constexpr double kPiU = 3.14159265358979323846;

// out[i] = sum_p coef[p] J0(rr[p] r[i]) (+ i/4 J0(kappa r[i]) when kappa > 0): one warp per
// radius, the lanes splitting the terms, FP64 throughout.
__global__ void radial_series_kernel(const double* __restrict__ coef, const double* __restrict__ rr, int P,
                                     double kappa, const double* __restrict__ r, long nr, double2* __restrict__ out) {
    const long w = (blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nr) return;                      // whole warps leave together
    const double x = r[w];
    double acc = 0.0;
    for (int p = lane; p < P; p += 32) acc = fma(coef[p], j0(rr[p] * x), acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[w] = make_double2(acc, kappa > 0.0 ? 0.25 * j0(kappa * x) : 0.0);
}

// Piecewise Chebyshev table in r: piece q covers [q w, (q + 1) w], coefficients [q][D][re, im].
struct RadialTable {
    int pieces, deg;
    double w;
    const double* coef;
};

__device__ __forceinline__ double2 radial_eval(const RadialTable& t, double r) {
    int q = static_cast<int>(r / t.w);
    q = min(max(q, 0), t.pieces - 1);
    const double tt = 2.0 * (r / t.w - q) - 1.0;
    const double* c = t.coef + static_cast<long>(q) * t.deg * 2;
    double br1 = 0.0, bi1 = 0.0, br2 = 0.0, bi2 = 0.0;
    for (int j = t.deg - 1; j >= 1; --j) {
        const double nr = 2.0 * tt * br1 - br2 + c[2 * j];
        const double ni = 2.0 * tt * bi1 - bi2 + c[2 * j + 1];
        br2 = br1;
        bi2 = bi1;
        br1 = nr;
        bi1 = ni;
    }
    return make_double2(tt * br1 - br2 + c[0], tt * bi1 - bi2 + c[1]);
}

// H[i][j] = psi_w(t_i) psi_w(t_j) g(|t|), t = ((i - n/2) h, (j - n/2) h), g from the table.
__global__ void window_grid_kernel(int n, double h, const double* __restrict__ wtab, RadialTable tab,
                                   double2* __restrict__ H) {
    const long idx = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (idx >= static_cast<long>(n) * n) return;
    const int i = static_cast<int>(idx / n), j = static_cast<int>(idx - static_cast<long>(i) * n);
    const double wv = wtab[i] * wtab[j];
    double2 v = make_double2(0.0, 0.0);
    if (wv != 0.0) {
        const double x = (i - 0.5 * n) * h, y = (j - 0.5 * n) * h;
        const double2 g = radial_eval(tab, sqrt(x * x + y * y));
        v = make_double2(wv * g.x, wv * g.y);
    }
    H[idx] = v;
}

// c[a][b] = K[a][b] / n^2 (psi(kx h) psi(ky h))^2, k = (index - nk/2) deta: the series'
// coefficients with the spreading window's deconvolution for the forward and inverse passes.
template <typename T, bool CPLX>
__global__ void coefficient_window_kernel(int nk, double deta, double inv_n2, SpreadDeconv sd,
                                          const double2* __restrict__ K, void* __restrict__ c) {
    const long idx = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (idx >= static_cast<long>(nk) * nk) return;
    const int a = static_cast<int>(idx / nk), b = static_cast<int>(idx - static_cast<long>(a) * nk);
    const double2 xi = make_double2((a - 0.5 * nk) * deta, (b - 0.5 * nk) * deta);
    const double f = spread_deconv(sd, xi);
    const double sc = inv_n2 * f * f;
    const double2 v = K[idx];
    if (CPLX) static_cast<cx_t<T>*>(c)[idx] = mk<T>(static_cast<T>(v.x * sc), static_cast<T>(v.y * sc));
    else static_cast<T*>(c)[idx] = static_cast<T>(v.x * sc);
}

// kout = c kin over rows [row0, nk) of nrhs grids; two complex elements per thread.
template <typename T, bool CPLX>
__global__ void multiply_kernel(const cx_t<T>* __restrict__ kin, const void* __restrict__ c,
                                cx_t<T>* __restrict__ kout, int nk, int row0, long kbatch) {
    const long half = static_cast<long>(nk) / 2;            // pairs per row (nk even)
    const long pairs = static_cast<long>(nk - row0) * half;
    const long t = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (t >= pairs) return;
    const long r = row0 + t / half, j = 2 * (t % half);
    const long e = r * nk + j;
    const cx_t<T>* src = kin + blockIdx.y * kbatch;
    cx_t<T>* dst = kout + blockIdx.y * kbatch;
    const cx_t<T> v0 = src[e], v1 = src[e + 1];
    if (CPLX) {
        const cx_t<T>* cc = static_cast<const cx_t<T>*>(c);
        dst[e] = cmul(cc[e], v0);
        dst[e + 1] = cmul(cc[e + 1], v1);
    } else {
        const T* cc = static_cast<const T*>(c);
        const T c0 = cc[e], c1 = cc[e + 1];
        dst[e] = mk<T>(c0 * v0.x, c0 * v0.y);
        dst[e + 1] = mk<T>(c1 * v1.x, c1 * v1.y);
    }
}

inline unsigned blocks(long n, int t = 256) { return static_cast<unsigned>((n + t - 1) / t); }

// Direct sums at the radii r (device), copied back to the host.
int radial_samples(const double* coef_d, const double* rr_d, int P, double kappa, const std::vector<double>& r,
                   std::vector<double2>& out, cudaStream_t s) {
    double* rd = nullptr;
    double2* od = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&rd, sizeof(double) * r.size(), s));
    SBD_CUDA_TRY(cudaMallocAsync(&od, sizeof(double2) * r.size(), s));
    SBD_CUDA_TRY(cudaMemcpyAsync(rd, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice, s));
    radial_series_kernel<<<blocks(static_cast<long>(r.size()) * 32), 256, 0, s>>>(coef_d, rr_d, P, kappa, rd,
                                                                                  static_cast<long>(r.size()), od);
    SBD_LAUNCH_CHECK();
    out.resize(r.size());
    SBD_CUDA_TRY(cudaMemcpyAsync(out.data(), od, sizeof(double2) * r.size(), cudaMemcpyDeviceToHost, s));
    SBD_CUDA_TRY(cudaFreeAsync(rd, s));
    SBD_CUDA_TRY(cudaFreeAsync(od, s));
    SBD_CUDA_TRY(cudaStreamSynchronize(s));
    return SBD_OK;
}

}  // namespace

template <typename T>
int uniform_coefficients(const SbdFit& fit, const NufftParams& np, const SpreadDeconv& sd, bool complex_c, void* c,
                         cudaStream_t s) {
    const int P = fit.P;
    const double kappa = fit.kind == 1 ? fit.kappa : 0.0;
    double smax = 0.0, scale = std::abs(fit.w0);
    for (int q = 0; q < fit.n_circles; ++q) smax = std::max(smax, fit.radius[q]);
    for (int p = 0; p < P; ++p) scale += std::fabs(fit.coef[p]);
    scale = std::max(scale + (kappa > 0 ? 0.25 : 0.0), 1e-300);
    std::vector<double> rr(P);
    for (int p = 0; p < P; ++p) rr[p] = fit.rho[p] / fit.scale_R;
    double *coef_d = nullptr, *rr_d = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&coef_d, sizeof(double) * std::max(P, 1), s));
    SBD_CUDA_TRY(cudaMallocAsync(&rr_d, sizeof(double) * std::max(P, 1), s));
    SBD_CUDA_TRY(cudaMemcpyAsync(coef_d, fit.coef.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s));
    SBD_CUDA_TRY(cudaMemcpyAsync(rr_d, rr.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s));
    // table of g(r) = G_fit(r) - w0 on [0, r_max], r_max the farthest corner of the window's support
    const double rmax = std::sqrt(2.0) * (np.wa + np.wtau) * (1.0 + 1e-9);
    const int D = 20;
    int pieces = static_cast<int>(std::ceil(1.25 * smax * rmax / kPiU)) + 1;
    const double accept = std::max(1e-13 * scale, 1e-3 * np.tol * scale);
    std::vector<double> table;
    double wpiece = 0.0;
    int rc = SBD_OK;
    for (int attempt = 0;; ++attempt) {
        wpiece = rmax / pieces;
        std::vector<double> r(static_cast<size_t>(pieces) * D);
        for (int q = 0; q < pieces; ++q)
            for (int k = 0; k < D; ++k) r[static_cast<size_t>(q) * D + k] =
                (q + 0.5 * (std::cos(kPiU * (k + 0.5) / D) + 1.0)) * wpiece;
        std::vector<double2> f;
        if ((rc = radial_samples(coef_d, rr_d, P, kappa, r, f, s))) break;
        table.assign(static_cast<size_t>(pieces) * D * 2, 0.0);
        for (int q = 0; q < pieces; ++q)
            for (int j = 0; j < D; ++j) {
                double sr = 0.0, si = 0.0;
                for (int k = 0; k < D; ++k) {
                    const double cs = std::cos(kPiU * j * (k + 0.5) / D);
                    sr += f[static_cast<size_t>(q) * D + k].x * cs;
                    si += f[static_cast<size_t>(q) * D + k].y * cs;
                }
                const double sc = (j == 0 ? 1.0 : 2.0) / D;
                table[(static_cast<size_t>(q) * D + j) * 2] = sr * sc;
                table[(static_cast<size_t>(q) * D + j) * 2 + 1] = si * sc;
            }
        // check between the interpolation points against the direct sums
        std::vector<double> rc_pts;
        for (int q = 0; q < pieces; ++q)
            for (double u : {0.137, 0.503, 0.871}) rc_pts.push_back((q + u) * wpiece);
        std::vector<double2> fc;
        if ((rc = radial_samples(coef_d, rr_d, P, kappa, rc_pts, fc, s))) break;
        double worst = 0.0;
        for (size_t i = 0; i < rc_pts.size(); ++i) {
            const int q = static_cast<int>(i / 3);
            const double tt = 2.0 * (rc_pts[i] / wpiece - q) - 1.0;
            double br1 = 0, bi1 = 0, br2 = 0, bi2 = 0;
            for (int j = D - 1; j >= 1; --j) {
                const double nr = 2.0 * tt * br1 - br2 + table[(static_cast<size_t>(q) * D + j) * 2];
                const double ni = 2.0 * tt * bi1 - bi2 + table[(static_cast<size_t>(q) * D + j) * 2 + 1];
                br2 = br1;
                bi2 = bi1;
                br1 = nr;
                bi1 = ni;
            }
            const double vr = tt * br1 - br2 + table[static_cast<size_t>(q) * D * 2];
            const double vi = tt * bi1 - bi2 + table[static_cast<size_t>(q) * D * 2 + 1];
            worst = std::max(worst, std::hypot(vr - fc[i].x, vi - fc[i].y));
        }
        if (worst <= accept) break;
        if (attempt == 3) {
            set_error("uniform grid: the radial table of the series does not converge");
            rc = SBD_EFIT;
            break;
        }
        pieces *= 2;
    }
    cudaFreeAsync(coef_d, s);
    cudaFreeAsync(rr_d, s);
    if (rc) return rc;
    // H on the n x n grid, its 2-D FFT (FP64) into the nk x nk window, the coefficients
    const int n = np.n, nk = np.nk;
    double *tab_d = nullptr, *wtab_d = nullptr;
    double2 *H = nullptr, *A = nullptr, *Tr = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&tab_d, sizeof(double) * table.size(), s));
    SBD_CUDA_TRY(cudaMallocAsync(&wtab_d, sizeof(double) * n, s));
    SBD_CUDA_TRY(cudaMemcpyAsync(tab_d, table.data(), sizeof(double) * table.size(), cudaMemcpyHostToDevice, s));
    SBD_CUDA_TRY(cudaMemcpyAsync(wtab_d, np.wtab.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    SBD_CUDA_TRY(cudaMallocAsync(&H, sizeof(double2) * static_cast<size_t>(n) * n, s));
    SBD_CUDA_TRY(cudaMallocAsync(&A, sizeof(double2) * static_cast<size_t>(n) * nk, s));
    SBD_CUDA_TRY(cudaMallocAsync(&Tr, sizeof(double2) * static_cast<size_t>(nk) * n, s));
    const RadialTable tab{pieces, D, wpiece, tab_d};
    window_grid_kernel<<<blocks(static_cast<long>(n) * n), 256, 0, s>>>(n, np.h, wtab_d, tab, H);
    SBD_LAUNCH_CHECK();
    // element t of a row sits at position t - n/2 (t = n/2 is y = 0); output e is frequency e - nk/2
    rc = fft_rows<double>(H, n, n, -n / 2, A, nk, nk, -nk / 2, n, n, -1, nullptr, nullptr, nullptr, nullptr, s);
    if (!rc) rc = transpose<double>(A, nk, 0, Tr, n, 0, n, nk, 1, s);
    if (!rc) rc = fft_rows<double>(Tr, n, n, -n / 2, A, nk, nk, -nk / 2, nk, n, -1, nullptr, nullptr, nullptr, nullptr, s);
    if (!rc) {
        const double inv_n2 = 1.0 / (static_cast<double>(n) * n);
        const long cells = static_cast<long>(nk) * nk;
        if (complex_c)
            coefficient_window_kernel<T, true><<<blocks(cells), 256, 0, s>>>(nk, np.deta, inv_n2, sd, A, c);
        else
            coefficient_window_kernel<T, false><<<blocks(cells), 256, 0, s>>>(nk, np.deta, inv_n2, sd, A, c);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error(std::string("uniform grid: ") + cudaGetErrorString(e));
            rc = SBD_ECUDA;
        }
    }
    cudaFreeAsync(H, s);
    cudaFreeAsync(A, s);
    cudaFreeAsync(Tr, s);
    cudaFreeAsync(tab_d, s);
    cudaFreeAsync(wtab_d, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc) {
        set_error(std::string("uniform grid: ") + cudaGetErrorString(cudaGetLastError()));
        rc = SBD_ECUDA;
    }
    return rc;
}

template <typename T>
int uniform_multiply(const cx_t<T>* kin, const void* c, bool complex_c, cx_t<T>* kout, int nk, int row0, int nrhs,
                     long kbatch, cudaStream_t s) {
    if (nk & 1 || row0 < 0 || row0 >= nk || nrhs < 1 || nrhs > 65535) {
        set_error("uniform multiply: invalid grid");
        return SBD_EINVAL;
    }
    const long pairs = static_cast<long>(nk - row0) * (nk / 2);
    const dim3 grid(blocks(pairs), static_cast<unsigned>(nrhs));
    if (complex_c) multiply_kernel<T, true><<<grid, 256, 0, s>>>(kin, c, kout, nk, row0, kbatch);
    else multiply_kernel<T, false><<<grid, 256, 0, s>>>(kin, c, kout, nk, row0, kbatch);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template int uniform_coefficients<float>(const SbdFit&, const NufftParams&, const SpreadDeconv&, bool, void*,
                                         cudaStream_t);
template int uniform_coefficients<double>(const SbdFit&, const NufftParams&, const SpreadDeconv&, bool, void*,
                                          cudaStream_t);
template int uniform_multiply<float>(const float2*, const void*, bool, float2*, int, int, int, long, cudaStream_t);
template int uniform_multiply<double>(const double2*, const void*, bool, double2*, int, int, int, long, cudaStream_t);

}  // namespace sbd
