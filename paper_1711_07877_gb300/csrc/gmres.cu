// Restarted GMRES on (shift I + scale A) x = b with A the SBD matvec of a plan, as a
// resumable session whose matvecs the caller computes (sbd_gmres runs one session alone with
// the plan's graph matvec; a server merges many sessions' matvecs into batched calls).
//
// The paper's motivation (Introduction): boundary-element systems are solved by
// iterative methods whose cost is the discrete convolution.  Arnoldi with two-pass
// classical Gram-Schmidt (the projections of a pass are one multi-dot kernel and one
// multi-axpy kernel), Givens rotations and the small least-squares solve on the host;
// one device-to-host read of the projections per pass.  Vectors are float64 (Laplace)
// or complex128 (Helmholtz).
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"
#include "sbd.h"

namespace sbd {

namespace {

using zc = std::complex<double>;

template <bool CPLX> struct V;
template <> struct V<false> { using t = double; };
template <> struct V<true>  { using t = double2; };

__device__ __forceinline__ double2 dconj_mul(double a, double b) { return make_double2(a * b, 0.0); }
__device__ __forceinline__ double2 dconj_mul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// out[j] = sum_i conj(Vj[i]) w[i] for j < k (one block row of partial sums per vector)
template <bool CPLX>
__global__ void multi_dot_kernel(const typename V<CPLX>::t* __restrict__ Vb, long n, int k,
                                 const typename V<CPLX>::t* __restrict__ w, double2* __restrict__ partial) {
    const int j = blockIdx.y;
    double sr = 0.0, si = 0.0;
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        const double2 p = dconj_mul(Vb[j * n + i], w[i]);
        sr += p.x;
        si += p.y;
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; }
    __syncthreads();
    if (wid == 0) {
        sr = lane < blockDim.x / 32 ? red[0][lane] : 0.0;
        si = lane < blockDim.x / 32 ? red[1][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, o);
            si += __shfl_down_sync(0xffffffffu, si, o);
        }
        if (lane == 0) partial[j * gridDim.x + blockIdx.x] = make_double2(sr, si);
    }
}

__device__ __forceinline__ double axpy_term(double v, double2 h) { return h.x * v; }
__device__ __forceinline__ double2 axpy_term(double2 v, double2 h) {
    return make_double2(h.x * v.x - h.y * v.y, h.x * v.y + h.y * v.x);
}
__device__ __forceinline__ void sub_to(double& a, double b) { a -= b; }
__device__ __forceinline__ void sub_to(double2& a, double2 b) { a.x -= b.x; a.y -= b.y; }
__device__ __forceinline__ void add_to(double& a, double b) { a += b; }
__device__ __forceinline__ void add_to(double2& a, double2 b) { a.x += b.x; a.y += b.y; }

// w[i] -= sum_j h[j] Vj[i]   (sign = -1)   or   w[i] += sum_j h[j] Vj[i]   (sign = +1)
template <bool CPLX>
__global__ void multi_axpy_kernel(const typename V<CPLX>::t* __restrict__ Vb, long n, int k,
                                  const double2* __restrict__ h, int sign, typename V<CPLX>::t* __restrict__ w) {
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        typename V<CPLX>::t acc = w[i];
        for (int j = 0; j < k; ++j) {
            const auto t = axpy_term(Vb[j * n + i], h[j]);
            if (sign < 0) sub_to(acc, t);
            else add_to(acc, t);
        }
        w[i] = acc;
    }
}

// y = alpha x + beta y  (alpha, beta complex; real vectors use the real parts)
template <bool CPLX>
__global__ void axpby_kernel(long n, double2 alpha, const typename V<CPLX>::t* __restrict__ x, double2 beta,
                             typename V<CPLX>::t* __restrict__ y) {
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        if constexpr (CPLX) {
            const double2 a = x[i], b = y[i];
            y[i] = make_double2(alpha.x * a.x - alpha.y * a.y + beta.x * b.x - beta.y * b.y,
                                alpha.x * a.y + alpha.y * a.x + beta.x * b.y + beta.y * b.x);
        } else {
            y[i] = alpha.x * x[i] + beta.x * y[i];
        }
    }
}

// x *= a
template <bool CPLX>
__global__ void scale_kernel(long n, double2 a, typename V<CPLX>::t* __restrict__ x) {
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        if constexpr (CPLX) {
            const double2 v = x[i];
            x[i] = make_double2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
        } else {
            x[i] = a.x * x[i];
        }
    }
}

__global__ void sum_partials_kernel(const double2* __restrict__ partial, int nb, int k, double2* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < nb; ++b) {
        sr += partial[j * nb + b].x;
        si += partial[j * nb + b].y;
    }
    out[j] = make_double2(sr, si);
}

template <bool CPLX>
struct Solver {
    using T = typename V<CPLX>::t;
    sbd_plan_t plan;
    long n;
    cudaStream_t s;
    zc shift, scale;
    T* Vb = nullptr;        // (m + 1) x n basis
    T* tmp = nullptr;       // n
    double2* partial = nullptr;
    double2* hd = nullptr;  // device projections
    int nblk = 0;
    std::vector<double2> hh;

    int dots(int k, const T* w, std::vector<zc>& out) {
        multi_dot_kernel<CPLX><<<dim3(nblk, k), 256, 0, s>>>(Vb, n, k, w, partial);
        sum_partials_kernel<<<(k + 127) / 128, 128, 0, s>>>(partial, nblk, k, hd);
        SBD_LAUNCH_CHECK();
        hh.resize(k);
        SBD_CUDA_TRY(cudaMemcpyAsync(hh.data(), hd, sizeof(double2) * k, cudaMemcpyDeviceToHost, s));
        SBD_CUDA_TRY(cudaStreamSynchronize(s));
        out.resize(k);
        for (int j = 0; j < k; ++j) out[j] = zc(hh[j].x, hh[j].y);
        return SBD_OK;
    }
    int axpy(int k, const std::vector<zc>& h, int sign, T* w) {
        hh.resize(k);
        for (int j = 0; j < k; ++j) hh[j] = make_double2(h[j].real(), h[j].imag());
        SBD_CUDA_TRY(cudaMemcpyAsync(hd, hh.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, s));
        multi_axpy_kernel<CPLX><<<nblk, 256, 0, s>>>(Vb, n, k, hd, sign, w);
        SBD_LAUNCH_CHECK();
        return SBD_OK;
    }
    int norm(const T* w, double* out) {
        // <w, w> through the multi-dot kernel with w as the single basis vector
        multi_dot_kernel<CPLX><<<dim3(nblk, 1), 256, 0, s>>>(w, n, 1, w, partial);
        sum_partials_kernel<<<1, 128, 0, s>>>(partial, nblk, 1, hd);
        SBD_LAUNCH_CHECK();
        double2 v;
        SBD_CUDA_TRY(cudaMemcpyAsync(&v, hd, sizeof(double2), cudaMemcpyDeviceToHost, s));
        SBD_CUDA_TRY(cudaStreamSynchronize(s));
        *out = std::sqrt(std::max(v.x, 0.0));
        return SBD_OK;
    }
    int scal(T* x, zc a) {
        scale_kernel<CPLX><<<nblk, 256, 0, s>>>(n, make_double2(a.real(), a.imag()), x);
        SBD_LAUNCH_CHECK();
        return SBD_OK;
    }
};

// GMRES as a resumable session: the solver stops wherever it needs y = A v (the plan's plain
// matvec; the shift and scale are applied here), so that a caller can compute many sessions'
// matvecs together.  States: RESIDUAL (v = x, y = V0: r = b - (shift I + scale A) x),
// ARNOLDI (v = V_j, y = V_{j+1}), CHECK (v = x, y = tmp: the true residual before stopping).
struct SessionBase {
    virtual ~SessionBase() = default;
    virtual int next(const void** in, void** out) = 0;
    virtual int advance() = 0;
    virtual void finish(int32_t* iters, double* rel) = 0;
};

template <bool CPLX>
struct Session : SessionBase {
    using T = typename V<CPLX>::t;
    enum State { RESIDUAL, ARNOLDI, CHECK, DONE };
    Solver<CPLX> S;
    sbd_gmres_options o{};
    int m = 1;
    const T* bb = nullptr;
    T* xx = nullptr;
    double bnorm = 0.0, rel = 1.0;
    int total = 0, j = 0;
    State st = RESIDUAL;
    std::vector<zc> h, h2, cs, sn, g;
    std::vector<std::vector<zc>> H;

    ~Session() override {
        if (S.Vb) cudaFreeAsync(S.Vb, S.s);
        if (S.tmp) cudaFreeAsync(S.tmp, S.s);
        if (S.partial) cudaFreeAsync(S.partial, S.s);
        if (S.hd) cudaFreeAsync(S.hd, S.s);
        cudaStreamSynchronize(S.s);
    }

    int begin(sbd_plan_t plan, long n, const void* b, void* x, const sbd_gmres_options& opt, cudaStream_t s) {
        o = opt;
        m = std::max(1, o.restart);
        S.plan = plan;
        S.n = n;
        S.s = s;
        S.shift = zc(o.shift_re, o.shift_im);
        S.scale = zc(o.scale_re, o.scale_im);
        S.nblk = static_cast<int>(std::min<long>(1024, (n + 255) / 256));
        if (cudaMallocAsync(&S.Vb, sizeof(T) * n * (m + 1), s) != cudaSuccess ||
            cudaMallocAsync(&S.tmp, sizeof(T) * n, s) != cudaSuccess ||
            cudaMallocAsync(&S.partial, sizeof(double2) * S.nblk * (m + 1), s) != cudaSuccess ||
            cudaMallocAsync(&S.hd, sizeof(double2) * (m + 1), s) != cudaSuccess) {
            cudaGetLastError();
            set_error("sbd_gmres: workspace allocation failed");
            return SBD_ENOMEM;
        }
        bb = static_cast<const T*>(b);
        xx = static_cast<T*>(x);
        H.assign(m + 1, std::vector<zc>(m, zc(0)));
        cs.assign(m, zc(0));
        sn.assign(m, zc(0));
        g.assign(m + 1, zc(0));
        int rc = S.norm(bb, &bnorm);
        if (rc) return rc;
        if (bnorm == 0.0) {
            SBD_CUDA_TRY(cudaMemsetAsync(xx, 0, sizeof(T) * n, s));
            rel = 0.0;
            st = DONE;
        } else if (total >= o.max_iter) {
            st = DONE;
        }
        return SBD_OK;
    }

    int next(const void** in, void** out) override {
        switch (st) {
            case RESIDUAL: *in = xx; *out = S.Vb; return 1;
            case ARNOLDI: *in = S.Vb + static_cast<long>(j) * S.n; *out = S.Vb + static_cast<long>(j + 1) * S.n; return 1;
            case CHECK: *in = xx; *out = S.tmp; return 1;
            default: *in = nullptr; *out = nullptr; return 0;
        }
    }

    // y = shift v + scale y (y held A v)
    void shifted(const T* v, T* y) {
        axpby_kernel<CPLX><<<S.nblk, 256, 0, S.s>>>(S.n, make_double2(S.shift.real(), S.shift.imag()), v,
                                                    make_double2(S.scale.real(), S.scale.imag()), y);
    }

    // x += V y after j Arnoldi steps (upper triangular solve on the host)
    int update_x() {
        std::vector<zc> y(j);
        for (int i = j - 1; i >= 0; --i) {
            zc t = g[i];
            for (int k = i + 1; k < j; ++k) t -= H[i][k] * y[k];
            y[i] = H[i][i] != zc(0) ? t / H[i][i] : zc(0);
        }
        return j > 0 ? S.axpy(j, y, +1, xx) : SBD_OK;
    }

    int advance() override {
        int rc = SBD_OK;
        const long n = S.n;
        if (st == RESIDUAL) {
            T* v0 = S.Vb;
            shifted(xx, v0);
            axpby_kernel<CPLX><<<S.nblk, 256, 0, S.s>>>(n, make_double2(1, 0), bb, make_double2(-1, 0), v0);
            SBD_LAUNCH_CHECK();
            double beta;
            if ((rc = S.norm(v0, &beta))) return rc;
            rel = beta / bnorm;
            if (rel <= o.tol) {
                st = DONE;
                return SBD_OK;
            }
            if ((rc = S.scal(v0, zc(1.0 / beta, 0)))) return rc;
            std::fill(g.begin(), g.end(), zc(0));
            g[0] = beta;
            j = 0;
            st = ARNOLDI;
            return SBD_OK;
        }
        if (st == ARNOLDI) {
            T* w = S.Vb + static_cast<long>(j + 1) * n;
            shifted(S.Vb + static_cast<long>(j) * n, w);
            SBD_LAUNCH_CHECK();
            if ((rc = S.dots(j + 1, w, h)) || (rc = S.axpy(j + 1, h, -1, w))) return rc;
            if ((rc = S.dots(j + 1, w, h2)) || (rc = S.axpy(j + 1, h2, -1, w))) return rc;   // second pass
            for (int i = 0; i <= j; ++i) H[i][j] = h[i] + h2[i];
            double hn;
            if ((rc = S.norm(w, &hn))) return rc;
            H[j + 1][j] = hn;
            if (hn > 0 && (rc = S.scal(w, zc(1.0 / hn, 0)))) return rc;
            for (int i = 0; i < j; ++i) {   // previous rotations
                const zc t = cs[i] * H[i][j] + sn[i] * H[i + 1][j];
                H[i + 1][j] = -std::conj(sn[i]) * H[i][j] + cs[i] * H[i + 1][j];
                H[i][j] = t;
            }
            // rotation [c s; -conj(s) c] (c real) zeroing H[j+1][j]
            const zc a = H[j][j], bq = H[j + 1][j];
            const double den = std::sqrt(std::norm(a) + std::norm(bq));
            if (den == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else if (std::abs(a) == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
            } else {
                cs[j] = std::abs(a) / den;
                sn[j] = (a / std::abs(a)) * std::conj(bq) / den;
            }
            const zc hjj = cs[j] * H[j][j] + sn[j] * H[j + 1][j];
            H[j + 1][j] = 0.0;
            H[j][j] = hjj;
            g[j + 1] = -std::conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            ++total;
            rel = std::abs(g[j + 1]) / bnorm;
            ++j;
            if (rel <= o.tol) {
                if ((rc = update_x())) return rc;
                st = CHECK;                      // confirm with the true residual
            } else if (j == m || total >= o.max_iter) {
                if ((rc = update_x())) return rc;
                st = total >= o.max_iter ? DONE : RESIDUAL;   // restart
            }
            return SBD_OK;
        }
        if (st == CHECK) {
            shifted(xx, S.tmp);
            axpby_kernel<CPLX><<<S.nblk, 256, 0, S.s>>>(n, make_double2(1, 0), bb, make_double2(-1, 0), S.tmp);
            SBD_LAUNCH_CHECK();
            double r2;
            if ((rc = S.norm(S.tmp, &r2))) return rc;
            rel = r2 / bnorm;
            st = (rel <= o.tol * 1.0000001 || total >= o.max_iter) ? DONE : RESIDUAL;
            return SBD_OK;
        }
        return SBD_OK;
    }

    void finish(int32_t* iters, double* rel_res) override {
        if (iters) *iters = total;
        if (rel_res) *rel_res = rel;
    }
};

}  // namespace

}  // namespace sbd

struct sbd_gmres_session_s {
    sbd::SessionBase* impl = nullptr;
};

extern "C" int sbd_gmres_begin(sbd_plan_t plan, const void* b, void* x, const sbd_gmres_options* opt,
                               void* cuda_stream, sbd_gmres_session_t* out) {
    using namespace sbd;
    if (!plan || !b || !x || !opt || !out || opt->restart < 1 || opt->max_iter < 0 || !(opt->tol > 0)) {
        set_error("sbd_gmres: invalid argument");
        return SBD_EINVAL;
    }
    sbd_plan_stats st;
    int rc = sbd_plan_info(plan, &st);
    if (rc) return rc;
    if (st.separate_targets) {
        set_error("sbd_gmres: the plan maps sources to separate targets (not a square system)");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    auto* h = new sbd_gmres_session_s();
    if (st.kind == SBD_HELMHOLTZ) {
        auto* ss = new Session<true>();
        h->impl = ss;
        rc = ss->begin(plan, st.n_points, b, x, *opt, s);
    } else {
        auto* ss = new Session<false>();
        h->impl = ss;
        rc = ss->begin(plan, st.n_points, b, x, *opt, s);
    }
    if (rc) {
        delete h->impl;
        delete h;
        return rc;
    }
    *out = h;
    return SBD_OK;
}

extern "C" int sbd_gmres_next(sbd_gmres_session_t sess, const void** in, void** out) {
    if (!sess || !in || !out) {
        sbd::set_error("sbd_gmres_next: null argument");
        return SBD_EINVAL;
    }
    return sess->impl->next(in, out);
}

extern "C" int sbd_gmres_advance(sbd_gmres_session_t sess) {
    if (!sess) {
        sbd::set_error("sbd_gmres_advance: null session");
        return SBD_EINVAL;
    }
    return sess->impl->advance();
}

extern "C" int sbd_gmres_end(sbd_gmres_session_t sess, int32_t* iterations, double* rel_residual) {
    if (!sess) return SBD_OK;
    sess->impl->finish(iterations, rel_residual);
    delete sess->impl;
    delete sess;
    return SBD_OK;
}

extern "C" int sbd_gmres(sbd_plan_t plan, const void* b, void* x, const sbd_gmres_options* opt, int32_t* iterations,
                         double* rel_residual, void* cuda_stream) {
    sbd_gmres_session_t sess = nullptr;
    int rc = sbd_gmres_begin(plan, b, x, opt, cuda_stream, &sess);
    if (rc) return rc;
    // the matvecs replay the plan's CUDA graph (launch cost matters for the small systems a
    // solver sees)
    const void* in = nullptr;
    void* out = nullptr;
    while (!rc && sbd_gmres_next(sess, &in, &out) == 1) {
        rc = sbd_matvec_graph(plan, in, out, 1, cuda_stream);
        if (!rc) rc = sbd_gmres_advance(sess);
    }
    sbd_gmres_end(sess, iterations, rel_residual);
    return rc;
}
