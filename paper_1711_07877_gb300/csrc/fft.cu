// Batched row FFT (mixed radix 2/3/4/5, Stockham autosort in shared memory) and
// tiled transpose.  Each CTA owns one row: the row is loaded once (zero padding,
// placement shift and diagonal scaling fused into the load), all radix stages run
// between two shared buffers, and only the
// requested output window is written back.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>
#include <cmath>

#include "fft.cuh"
#include "sbd.h"

namespace sbd {

namespace {

constexpr double kPi = 3.14159265358979323846;

// exp(-2 pi i t / n), t in [0, n), per (n, precision); built on the host in FP64
// with the angle reduced to the first octant before calling cos/sin.
template <typename T>
const cx_t<T>* twiddles(int n, cudaStream_t stream) {
    static std::mutex mu;
    static std::map<int, cx_t<T>*> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(n);
    if (it != cache.end()) return it->second;
    std::vector<cx_t<T>> h(n);
    for (int t = 0; t < n; ++t) {
        // angle 2 pi t / n, reduced via symmetries so cos/sin see |angle| <= pi/4
        long long k8 = 8LL * t;  // octant arithmetic in integers
        const long long nn = n;
        const int oct = static_cast<int>(k8 / nn);       // 0..7
        const double rem = static_cast<double>(k8 - oct * nn) / (8.0 * nn);   // fraction of a turn in [0, 1/8)
        double c, s;
        const double th = 2.0 * kPi * rem;
        const double ct = std::cos(th), st = std::sin(th);
        const double r2 = 0.70710678118654752440;
        const double cq = (ct - st) * r2, sq = (ct + st) * r2;  // angle + pi/4
        switch (oct) {
            case 0: c = ct;  s = st;  break;
            case 1: c = cq;  s = sq;  break;
            case 2: c = -st; s = ct;  break;
            case 3: c = -sq; s = cq;  break;
            case 4: c = -ct; s = -st; break;
            case 5: c = -cq; s = -sq; break;
            case 6: c = st;  s = -ct; break;
            default: c = sq; s = -cq; break;
        }
        h[t] = mk<T>(static_cast<T>(c), static_cast<T>(-s));
    }
    cx_t<T>* d = nullptr;
    if (cudaMalloc(&d, sizeof(cx_t<T>) * n) != cudaSuccess) return nullptr;
    cudaMemcpyAsync(d, h.data(), sizeof(cx_t<T>) * n, cudaMemcpyHostToDevice, stream);
    cudaStreamSynchronize(stream);
    cache[n] = d;
    return d;
}

template <typename C> __device__ __forceinline__ C mul_mi(C a, int sign) {
    // a * (sign * i): sign = -1 -> a * (-i), sign = +1 -> a * i
    C r;
    if (sign < 0) { r.x = a.y; r.y = -a.x; }
    else          { r.x = -a.y; r.y = a.x; }
    return r;
}

template <typename T, int R>
__device__ __forceinline__ void small_dft(cx_t<T>* v, int sign) {
    using C = cx_t<T>;
    if constexpr (R == 2) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        C a2 = cadd(v[1], v[3]), a3 = mul_mi(csub(v[1], v[3]), sign);
        v[0] = cadd(a0, a2);
        v[2] = csub(a0, a2);
        v[1] = cadd(a1, a3);
        v[3] = csub(a1, a3);
    } else if constexpr (R == 3) {
        const T h = static_cast<T>(0.86602540378443864676);   // sqrt(3)/2
        C t1 = cadd(v[1], v[2]);
        C t2 = csub(v[0], cscale(t1, static_cast<T>(0.5)));
        C t3 = mul_mi(cscale(csub(v[1], v[2]), h), sign);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    } else if constexpr (R == 5) {
        const T c1 = static_cast<T>(0.30901699437494742410), c2 = static_cast<T>(-0.80901699437494742410);
        const T s1 = static_cast<T>(0.95105651629515357212), s2 = static_cast<T>(0.58778525229247312917);
        C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        C p1 = cadd(v[0], cadd(cscale(a1, c1), cscale(a2, c2)));
        C p2 = cadd(v[0], cadd(cscale(a1, c2), cscale(a2, c1)));
        C q1 = mul_mi(cadd(cscale(b1, s1), cscale(b2, s2)), sign);
        C q2 = mul_mi(csub(cscale(b1, s2), cscale(b2, s1)), sign);
        v[0] = cadd(v[0], cadd(a1, a2));
        v[1] = cadd(p1, q1);
        v[4] = csub(p1, q1);
        v[2] = cadd(p2, q2);
        v[3] = csub(p2, q2);
    }
}

// One radix-R Stockham stage, out of place from src to dst (both in shared memory):
// butterfly j in [0, nq/R) reads src[j + r nq/R] (consecutive j, consecutive addresses),
// twiddles by w^(r k) with k = j mod Ns, and writes dst[(j / Ns) Ns R + k + r Ns], so the
// output of the last stage is in natural order.  j / Ns uses the stage's multiplier.
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const cx_t<T>* __restrict__ src, cx_t<T>* __restrict__ dst, int nq,
                                               int Ns, unsigned magic, int sign, const cx_t<T>* __restrict__ tw,
                                               int tw_unit, int nthreads) {
    using C = cx_t<T>;
    const int nb = nq / R;
    const int tw_step = tw_unit * (nq / (Ns * R));
    for (int j = threadIdx.x; j < nb; j += nthreads) {
        const int q = Ns == 1 ? j : static_cast<int>(__umulhi(static_cast<unsigned>(j), magic));
        const int k = j - q * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * k * tw_step];
                if (sign > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        small_dft<T, R>(v, sign);
        const int o = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[o + r * Ns] = v[r];
    }
}

// One row (blockIdx.y) and one phase (blockIdx.x) of a length-n transform done as Q
// transforms of length nq = n / Q (Q = 1, 2 or 4): output k = Q k' + r is the length-nq
// DFT of y_r[t] = sum_{j < Q} x[t + j nq] w_n^{r (t + j nq)} (fold and twist on the load).
// The two shared buffers of nq elements alternate as source and destination.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) fft_rows_kernel(
    const cx_t<T>* __restrict__ in, long in_stride, int in_len, int in_shift,
    cx_t<T>* __restrict__ out, long out_stride, int out_len, int out_shift,
    int n, int Q, int sign, FftPlan1D plan, const cx_t<T>* __restrict__ tw,
    const T* __restrict__ pre_elem, const T* __restrict__ pre_row,
    const T* __restrict__ post_elem, const T* __restrict__ post_row) {
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nq = n / Q;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + nq;
    const long row = blockIdx.y;     // the phases of a row are adjacent CTAs (they read the same row)
    const int r = blockIdx.x;
    const C* src = in + row * in_stride;
    const T rs = pre_row ? pre_row[row] : static_cast<T>(1);
    for (int i = threadIdx.x; i < nq; i += NT) {
        C acc = mk<T>(0, 0);
        for (int j = 0; j < Q; ++j) {
            const int idx = i + j * nq;               // FFT index
            int t = idx - in_shift;
            if (t < 0) t += n;
            if (t < in_len) {
                C v = src[t];
                T sc = rs;
                if (pre_elem) sc *= pre_elem[t];
                v = cscale(v, sc);
                if (r) {                              // twist w_n^{r idx}
                    C w = tw[(static_cast<long>(r) * idx) % n];
                    if (sign > 0) w.y = -w.y;
                    v = cmul(v, w);
                }
                acc = cadd(acc, v);
            }
        }
        buf0[i] = acc;
    }
    __syncthreads();
    C* a = buf0;
    C* b = buf1;
    int Ns = 1;
    for (int st = 0; st < plan.nstages; ++st) {
        const int R = plan.radix[st];
        const unsigned mg = plan.magic[st];
        if (R == 4)      stockham_stage<T, 4>(a, b, nq, Ns, mg, sign, tw, Q, NT);
        else if (R == 2) stockham_stage<T, 2>(a, b, nq, Ns, mg, sign, tw, Q, NT);
        else if (R == 3) stockham_stage<T, 3>(a, b, nq, Ns, mg, sign, tw, Q, NT);
        else             stockham_stage<T, 5>(a, b, nq, Ns, mg, sign, tw, Q, NT);
        __syncthreads();
        C* t = a; a = b; b = t;
        Ns *= R;
    }
    C* dst = out + row * out_stride;
    const T ps = post_row ? post_row[row] : static_cast<T>(1);
    for (int e = threadIdx.x; e < out_len; e += NT) {
        int k = e + out_shift;
        if (k >= n) k -= n;
        if (Q > 1 && (k % Q) != r) continue;
        C v = a[k / Q];
        T sc = ps;
        if (post_elem) sc *= post_elem[e];
        dst[e] = cscale(v, sc);
    }
}

template <typename T>
__global__ void transpose_kernel(const cx_t<T>* __restrict__ in, long in_stride, long in_batch,
                                 cx_t<T>* __restrict__ out, long out_stride, long out_batch,
                                 int rows, int cols) {
    using C = cx_t<T>;
    __shared__ C tile[32][33];
    const C* src = in + blockIdx.z * in_batch;
    C* dst = out + blockIdx.z * out_batch;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = src[static_cast<long>(r) * in_stride + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[static_cast<long>(c) * out_stride + r] = tile[threadIdx.x][i];
    }
}

}  // namespace

bool fft_make_plan(int n, FftPlan1D& p) {
    p.n = n;
    p.nstages = 0;
    int v = n;
    int twos = 0;
    while (v % 2 == 0) { v /= 2; ++twos; }
    std::vector<int> rs;
    while (twos >= 2) { rs.push_back(4); twos -= 2; }
    if (twos) rs.push_back(2);
    while (v % 3 == 0) { v /= 3; rs.push_back(3); }
    while (v % 5 == 0) { v /= 5; rs.push_back(5); }
    if (v != 1 || static_cast<int>(rs.size()) > kFftMaxStages) return false;
    int Ns = 1;
    for (size_t i = 0; i < rs.size(); ++i) {
        p.radix[i] = rs[i];
        // j / Ns = umulhi(j, ceil(2^32 / Ns)), exact for j, Ns <= 2^15
        p.magic[i] = Ns == 1 ? 0u : static_cast<unsigned>((0x100000000ULL + Ns - 1) / Ns);
        Ns *= rs[i];
    }
    p.nstages = static_cast<int>(rs.size());
    p.threads = 1024;
    return true;
}

int fft_max_row(bool fp64) {
    const int smem = 227 * 1024;
    return std::min(smem / (2 * (fp64 ? 16 : 8)), 32768);
}

static int fft_phases(int n, bool fp64);

// Phases per row: the smallest Q in {1, 2, 4} dividing n whose length n / Q fits one CTA's
// shared memory twice (source and destination buffers).
static int fft_phases(int n, bool fp64) {
    const int lim = fft_max_row(fp64);
    for (int Q : {1, 2, 4})
        if (n % Q == 0 && n / Q <= lim) return Q;
    return 0;
}

int fft_max_length(bool fp64) { return 4 * fft_max_row(fp64); }

template <typename T>
int fft_rows(const cx_t<T>* in, long in_stride, int in_len, int in_shift,
             cx_t<T>* out, long out_stride, int out_len, int out_shift,
             int rows, int n, int sign,
             const T* pre_elem, const T* pre_row, const T* post_elem, const T* post_row,
             cudaStream_t stream) {
    if (rows <= 0) return SBD_OK;
    const bool fp64 = sizeof(T) == 8;
    const int Q = fft_phases(n, fp64);
    FftPlan1D plan;
    if (Q == 0 || !fft_make_plan(n / Q, plan)) {
        set_error("FFT length not supported: " + std::to_string(n));
        return SBD_ENOTSUP;
    }
    const int nq = n / Q;
    const cx_t<T>* tw = twiddles<T>(n, stream);
    if (!tw) {
        set_error("FFT table allocation failed");
        return SBD_ENOMEM;
    }
    const size_t smem = 2 * sizeof(cx_t<T>) * static_cast<size_t>(nq);
    in_shift = ((in_shift % n) + n) % n;
    out_shift = ((out_shift % n) + n) % n;
    for (int r0 = 0; r0 < rows; r0 += 65535) {          // grid.y holds at most 65535 rows
        const int nr = std::min(65535, rows - r0);
        const dim3 grid(static_cast<unsigned>(Q), static_cast<unsigned>(nr));
        const cx_t<T>* ip = in + static_cast<long>(r0) * in_stride;
        cx_t<T>* op = out + static_cast<long>(r0) * out_stride;
        const T* prr = pre_row ? pre_row + r0 : nullptr;
        const T* por = post_row ? post_row + r0 : nullptr;
        if (nq > 2048) {
            auto k = fft_rows_kernel<T, 1024>;
            SBD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
            k<<<grid, 1024, smem, stream>>>(ip, in_stride, in_len, in_shift, op, out_stride, out_len, out_shift,
                                            n, Q, sign, plan, tw, pre_elem, prr, post_elem, por);
        } else {
            auto k = fft_rows_kernel<T, 256>;
            SBD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
            k<<<grid, 256, smem, stream>>>(ip, in_stride, in_len, in_shift, op, out_stride, out_len, out_shift,
                                           n, Q, sign, plan, tw, pre_elem, prr, post_elem, por);
        }
        SBD_LAUNCH_CHECK();
    }
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int transpose(const cx_t<T>* in, long in_stride, long in_batch, cx_t<T>* out, long out_stride,
              long out_batch, int rows, int cols, int nb, cudaStream_t stream) {
    if (rows <= 0 || cols <= 0 || nb <= 0) return SBD_OK;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32, nb), block(32, 8);
    transpose_kernel<T><<<grid, block, 0, stream>>>(in, in_stride, in_batch, out, out_stride, out_batch, rows, cols);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template int fft_rows<float>(const float2*, long, int, int, float2*, long, int, int, int, int, int,
                             const float*, const float*, const float*, const float*, cudaStream_t);
template int fft_rows<double>(const double2*, long, int, int, double2*, long, int, int, int, int, int,
                              const double*, const double*, const double*, const double*, cudaStream_t);
template int transpose<float>(const float2*, long, long, float2*, long, long, int, int, int, cudaStream_t);
template int transpose<double>(const double2*, long, long, double2*, long, long, int, int, int, cudaStream_t);

}  // namespace sbd
