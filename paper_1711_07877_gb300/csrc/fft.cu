// Batched row FFT (mixed radix 2/3/4/5, in-place decimation in time in shared memory) and
// tiled transpose.  Each CTA owns one row: the row is loaded once (zero padding,
// placement shift, digit reversal and diagonal scaling fused into the load), all
// radix stages run in place in shared memory, and only the
// requested output window is written back.
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>
#include <cmath>

#include "fft.cuh"
#include "sbd.h"

namespace sbd {

namespace {

constexpr double kPi = 3.14159265358979323846;

// exp(-2 pi i t / n) on the host in FP64, the angle reduced to the first octant before
// calling cos/sin.
void host_twiddle(long long t, long long n, double& re, double& im) {
    t %= n;
    const long long k8 = 8LL * t;  // octant arithmetic in integers
    const int oct = static_cast<int>(k8 / n);        // 0..7
    const double rem = static_cast<double>(k8 - oct * n) / (8.0 * n);   // fraction of a turn in [0, 1/8)
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
    re = c;
    im = -s;
}

// Process-wide cache of device tables keyed by an int.  Its lock is held only to read or
// to insert: a miss builds and uploads the table without it, because allocating takes the
// capture lock exclusively while a thread capturing a graph holds that lock shared and may
// be waiting here for a table it already has.  A miss on a capturing stream fails instead
// of allocating (the caller reports SBD_ENOMEM); plans run one plain call before capturing.
template <typename V>
struct TableCache {
    std::mutex mu;
    std::map<int, V*> map;
    V* find(int key) {
        std::lock_guard<std::mutex> lock(mu);
        auto it = map.find(key);
        return it == map.end() ? nullptr : it->second;
    }
    V* upload(int key, const std::vector<V>& h, cudaStream_t stream) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
        V* d = nullptr;
        {
            std::unique_lock<std::shared_mutex> lock(capture_mutex());
            if (cudaMalloc(&d, sizeof(V) * h.size()) != cudaSuccess) return nullptr;
        }
        cudaMemcpyAsync(d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, stream);
        cudaStreamSynchronize(stream);
        std::lock_guard<std::mutex> lock(mu);
        auto it = map.find(key);
        if (it != map.end()) return it->second;     // another thread built it meanwhile (ours stays unused)
        map[key] = d;
        return d;
    }
};

// Two-level table of exp(-2 pi i t / n): lo[j] for j < kTwLo, then hi[i] = the twiddle of
// t = kTwLo i for i < ceil(n / kTwLo); tw(t) = hi[t / kTwLo] lo[t % kTwLo].  Small enough to
// sit in shared memory beside the row (a few KB), so the radix stages take their twiddles
// from there instead of from a global table of n entries.
constexpr int kTwLo = 128;
inline int tw2_size(int n) { return kTwLo + (n + kTwLo - 1) / kTwLo; }


template <typename T>
const cx_t<T>* twiddles2(int n, cudaStream_t stream) {
    static TableCache<cx_t<T>> cache;
    if (const cx_t<T>* d = cache.find(n)) return d;
    std::vector<cx_t<T>> h(tw2_size(n));
    double re, im;
    for (int j = 0; j < kTwLo; ++j) {
        host_twiddle(j, n, re, im);
        h[j] = mk<T>(static_cast<T>(re), static_cast<T>(im));
    }
    for (int i = 0; kTwLo + i < static_cast<int>(h.size()); ++i) {
        host_twiddle(static_cast<long long>(kTwLo) * i, n, re, im);
        h[kTwLo + i] = mk<T>(static_cast<T>(re), static_cast<T>(im));
    }
    return cache.upload(n, h, stream);
}

// exp(-2 pi i t / n), t in [0, n), per (n, precision).
template <typename T>
const cx_t<T>* twiddles(int n, cudaStream_t stream) {
    static TableCache<cx_t<T>> cache;
    if (const cx_t<T>* d = cache.find(n)) return d;
    std::vector<cx_t<T>> h(n);
    for (int t = 0; t < n; ++t) {
        double re, im;
        host_twiddle(t, n, re, im);
        h[t] = mk<T>(static_cast<T>(re), static_cast<T>(im));
    }
    return cache.upload(n, h, stream);
}


// Twiddle t of the row's table: from the two-level shared-memory table (tws non-null) or
// from the full global table.
template <typename T>
__device__ __forceinline__ cx_t<T> twid(const cx_t<T>* __restrict__ tw, const cx_t<T>* tws, int t) {
    if (tws) return cmul(tws[kTwLo + (t >> 7)], tws[t & (kTwLo - 1)]);
    return tw[t];
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

// ---- roots of unity as compile-time constants ------------------------------------------
// cos and sin of 2 pi j / R for the fixed twiddles inside a radix-R butterfly: Taylor series
// on [0, pi/4) after reducing j / R to that octant in integer arithmetic, evaluated by the
// compiler in double precision.
__host__ __device__ constexpr double ct_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int k = 1; k <= 12; ++k) {
        term *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k <= 12; ++k) {
        term *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
struct CtRoot {
    double c, s;
};
__host__ __device__ constexpr CtRoot ct_root(int j, int R) {
    j %= R;
    if (j < 0) j += R;
    const int oct = 8 * j / R;
    const int rem = 8 * j - oct * R;   // angle = 2 pi (oct R + rem) / (8 R)
    const double th = 2.0 * 3.14159265358979323846 * rem / (8.0 * R);
    const double ct = ct_cos(th), st = ct_sin(th);
    const double h = 0.70710678118654752440;
    const double cq = (ct - st) * h, sq = (ct + st) * h;   // angle + pi / 4
    switch (oct) {
        case 0: return {ct, st};
        case 1: return {cq, sq};
        case 2: return {-st, ct};
        case 3: return {-sq, cq};
        case 4: return {-ct, -st};
        case 5: return {-cq, -sq};
        case 6: return {st, -ct};
        default: return {sq, -cq};
    }
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// a exp(SIGN 2 pi i J / R), J and R fixed at compile time (quarter turns as swaps)
template <typename T, int R, int J, int SIGN>
__device__ __forceinline__ cx_t<T> mul_root(cx_t<T> a) {
    constexpr int j = ((J % R) + R) % R;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (2 * j == R) {
        return mk<T>(-a.x, -a.y);
    } else if constexpr (4 * j == R) {
        return mul_mi(a, SIGN);
    } else if constexpr (4 * j == 3 * R) {
        return mul_mi(a, -SIGN);
    } else {
        constexpr CtRoot w = ct_root(j, R);
        constexpr T c = static_cast<T>(w.c), sn = static_cast<T>(SIGN * w.s);
        return mk<T>(a.x * c - a.y * sn, a.x * sn + a.y * c);
    }
}

// In-register DFT of length R = 2^a 3^b 5^c: v[k] = sum_n v[n] exp(SIGN 2 pi i n k / R).
// Composite R = a b: with n = b n1 + n2 and k = k1 + a k2, b transforms of length a over
// n1, the twiddles exp(SIGN 2 pi i n2 k1 / R), then a transforms of length b over n2.
template <typename T, int R, int SIGN>
__device__ __forceinline__ void dft(cx_t<T>* v) {
    if constexpr (R == 2 || R == 3 || R == 4 || R == 5) {
        small_dft<T, R>(v, SIGN);
    } else {
        constexpr int a = R % 4 == 0 ? 4 : R % 2 == 0 ? 2 : R % 3 == 0 ? 3 : 5;
        constexpr int b = R / a;
        cx_t<T> y[R];
        static_for<0, b>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            cx_t<T> u[a];
#pragma unroll
            for (int n1 = 0; n1 < a; ++n1) u[n1] = v[b * n1 + n2];
            small_dft<T, a>(u, SIGN);
            static_for<0, a>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                y[n2 * a + k1] = mul_root<T, R, n2 * k1, SIGN>(u[k1]);
            });
        });
#pragma unroll
        for (int k1 = 0; k1 < a; ++k1) {
            cx_t<T> u[b];
#pragma unroll
            for (int n2 = 0; n2 < b; ++n2) u[n2] = y[n2 * a + k1];
            dft<T, b, SIGN>(u);
#pragma unroll
            for (int k2 = 0; k2 < b; ++k2) v[k1 + a * k2] = u[k2];
        }
    }
}

// Twiddles of one butterfly of a stage: w_j = W^{j t} (W = the row's root, conjugated for
// SIGN = +1) for j = 1 .. R - 1.  The powers j in {1, 2, 3, 4, 8, 16} come from the table;
// the others are products of those (at most three deep: j = 16 + 8 + 4 + 3), so that each
// twiddle carries a few roundings at most.
template <typename T>
struct StageTw {
    cx_t<T> p1, p2, p3, p4, p8, p16;
};

template <typename T, int SIGN, int R>
__device__ __forceinline__ StageTw<T> stage_lookups(const cx_t<T>* __restrict__ tw, const cx_t<T>* tws, int t) {
    StageTw<T> w;
    auto get = [&](int j) {
        cx_t<T> x = twid<T>(tw, tws, j * t);
        if (SIGN > 0) x.y = -x.y;
        return x;
    };
    w.p1 = get(1);
    if constexpr (R > 2) w.p2 = get(2);
    if constexpr (R > 3) w.p3 = get(3);
    if constexpr (R > 4) w.p4 = get(4);
    if constexpr (R > 8) w.p8 = get(8);
    if constexpr (R > 16) w.p16 = get(16);
    return w;
}

template <typename T, int J>
__device__ __forceinline__ cx_t<T> tw_pow(const StageTw<T>& w) {
    if constexpr (J == 1) return w.p1;
    else if constexpr (J == 2) return w.p2;
    else if constexpr (J == 3) return w.p3;
    else if constexpr (J == 4) return w.p4;
    else if constexpr (J == 8) return w.p8;
    else if constexpr (J == 16) return w.p16;
    else if constexpr (J > 16) return cmul(w.p16, tw_pow<T, J - 16>(w));
    else if constexpr (J > 8) return cmul(w.p8, tw_pow<T, J - 8>(w));
    else return cmul(w.p4, tw_pow<T, J - 4>(w));
}

template <typename T, int R>
__device__ __forceinline__ void apply_stage_tw(cx_t<T>* v, const StageTw<T>& w) {
    static_for<1, R>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        v[j] = cmul(v[j], tw_pow<T, j>(w));
    });
}

// Shared-memory slot of row element p.  The digit-reversed stores of the load pass step
// through the row by a multiple of 16 elements (the product of the earlier radices, even for
// every length here), which would put a half-warp's sixteen 8-byte accesses in one bank (and
// the early stages' groups, 16 k elements apart, in a few); the slot XORs the index of the
// element's 16-element block into its low four bits, which spreads such runs over the banks
// and keeps every aligned block of 16 consecutive elements in one 128-byte line (measured at
// N = 10^6: 1.04 -> 0.96 ms per forward transform; one spare slot per 16 elements instead:
// 1.14 ms).
__host__ __device__ constexpr int row_slot(int p) { return p ^ ((p >> 4) & 15); }
// Slots taken by a row of n elements (whole 16-element blocks).
__host__ __device__ constexpr int row_slots(int n) { return (n + 15) & ~15; }

template <typename T> struct MaxB;
template <> struct MaxB<float>  { static constexpr int n_max = 28672; };
template <> struct MaxB<double> { static constexpr int n_max = 14336; };

// Radices of the in-register butterflies: prime powers up to 16 and 15 (FP32) or up to 9
// (FP64, twice the registers per element), which fit the 80 registers a thread of the launch bounds.
// f(integral_constant<R>) for the runtime radix R.
template <typename T, typename F>
__device__ __forceinline__ void with_radix(int R, F&& f) {
    switch (R) {
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 5: f(std::integral_constant<int, 5>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        default:
            if constexpr (sizeof(T) == 4) {
                if (R == 16) f(std::integral_constant<int, 16>{});
                else if (R == 15) f(std::integral_constant<int, 15>{});
                else f(std::integral_constant<int, 9>{});
            } else {
                f(std::integral_constant<int, 9>{});
            }
            break;
    }
}

// Stage of the in-place mixed-radix decimation-in-time FFT: groups of L = Lp * R
// elements combine R sub-transforms of length Lp (stored as consecutive blocks)
// into one transform of length L, in place.  A thread keeps one offset k within
// the sub-transforms (so its twiddles are looked up once per stage) and walks
// the groups g; no division per butterfly.
template <typename T, int R, int SIGN>
__device__ __forceinline__ void dit_stage(cx_t<T>* s, int n, int Lp, const cx_t<T>* __restrict__ tw,
                                          const cx_t<T>* tws, int tw_scale, int nthreads) {
    using C = cx_t<T>;
    const int L = Lp * R;
    const int G = n / L;
    const int tw_step = tw_scale * G;          // twiddle table index step of exp(2 pi i k / L)
    int k, g0, gstep;
    bool active = true;
    if (Lp >= nthreads) {
        k = threadIdx.x;
        g0 = 0;
        gstep = 1;
    } else {
        k = threadIdx.x % Lp;
        g0 = threadIdx.x / Lp;
        gstep = nthreads / Lp;
        active = g0 < gstep;
    }
    for (; active && k < Lp; k += nthreads) {
        StageTw<T> w{};
        if (Lp > 1) w = stage_lookups<T, SIGN, R>(tw, tws, k * tw_step);
        for (int g = g0; g < G; g += gstep) {
            const int base = g * L + k;
            C v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[row_slot(base + r * Lp)];
            if (Lp > 1) apply_stage_tw<T, R>(v, w);
            dft<T, R, SIGN>(v);
#pragma unroll
            for (int r = 0; r < R; ++r) s[row_slot(base + r * Lp)] = v[r];
        }
    }
    __syncthreads();
}

// The last stage (G = 1, so one butterfly per offset k), writing its outputs straight to
// the destination through put(position in s, value) instead of back to shared memory.
template <typename T, int R, int SIGN, typename Put>
__device__ __forceinline__ void dit_stage_out(const cx_t<T>* s, int n, int Lp, const cx_t<T>* __restrict__ tw,
                                              const cx_t<T>* tws, int tw_scale, int nthreads, Put put) {
    using C = cx_t<T>;
    const int tw_step = tw_scale * (n / (Lp * R));
    for (int k = threadIdx.x; k < Lp; k += nthreads) {
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[row_slot(k + r * Lp)];
        if (Lp > 1) apply_stage_tw<T, R>(v, stage_lookups<T, SIGN, R>(tw, tws, k * tw_step));
        dft<T, R, SIGN>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) put(k + r * Lp, v[r]);
    }
}

// One row (blockIdx.y) and one phase (blockIdx.x) of a length-n transform done as Q
// transforms of length nq = n / Q (Q = 1 or 2): output k = Q k' + r is the length-nq DFT
// of y_r[t] = sum_{j < Q} x[t + j nq] w_n^{r (t + j nq)} (fold and twist on the load).
// Hermitian fold of the load (see fft_rows): base of the whole grid, its side (0 = off)
// and the absolute index of this launch's first row.
// lo: rows of the grid below lo are zero, so a row whose mirror row n - row lies below lo needs no fold.
template <typename T> struct HermFold { const cx_t<T>* base; int n; long row0; int lo; };

// Input element at FFT position idx of the current row (has = false: a zero).  The io mode and
// whether a Hermitian fold applies are compile-time, so each load loop carries only its own case.
template <typename T, int IO, bool FOLD>
__device__ __forceinline__ cx_t<T> load_elem(int idx, int n, const cx_t<T>* __restrict__ src,
                                             long in_stride, int in_len, int in_shift, long row,
                                             const HermFold<T>& hf, T rs0, T rs1,
                                             const T* __restrict__ pre_elem, bool& has) {
    using C = cx_t<T>;
    has = false;
    if constexpr (IO == kIoPairInv) {
        // rows 2r, 2r+1 hold frequencies 0..in_len-1 of two Hermitian spectra A0, A1;
        // z = A0 + i A1 with A(-k) = conj A(k)
        const int k = idx < n / 2 ? idx : idx - n;
        const int ka = k < 0 ? -k : k;
        if (ka >= in_len) return mk<T>(0, 0);
        C a = src[ka], b = src[in_stride + ka];
        if (k < 0) {
            a.y = -a.y;
            b.y = -b.y;
        }
        has = true;
        return mk<T>(a.x - b.y, a.y + b.x);
    }
    int t = idx - in_shift;
    if (t < 0) t += n;
    if (t >= in_len) return mk<T>(0, 0);
    C v = src[t];
    if constexpr (FOLD) {
        const long ar = hf.row0 + row;
        if (ar >= 1 && t >= 1) {
            const C mv = hf.base[(hf.n - ar) * in_stride + (hf.n - t)];
            v.x += mv.x;
            v.y -= mv.y;
        }
    }
    const T pe = pre_elem ? pre_elem[t] : static_cast<T>(1);
    v.x *= rs0 * pe;
    v.y *= rs1 * pe;
    has = true;
    return v;
}

// SIGN (-1 forward, +1 inverse) is a template argument: the factors +-i of the butterflies
// and the conjugation of the twiddles fold into the arithmetic.  NT threads and at most 80
// registers a thread: 256 threads and three CTAs per SM where three rows fit the SM's shared
// memory, 384 threads and two CTAs per SM where only two do (13824-point FP32 rows, 110 KB), so
// that an SM holds 24 warps either way and one row's loads overlap the others' butterflies
// (measured at N = 10^6: 13824-point rows 0.96 -> 0.83 ms per forward transform with 384 threads;
// the 6912-point rows of a smaller grid and the uniform-grid variant's 15360-point rows were slower
// with 384 threads everywhere: 0.16 -> 0.19 and 1.25 -> 1.53 ms).
template <int NT> struct FftCtas { static constexpr int value = NT == 384 ? 2 : 3; };
constexpr size_t kFftSmemThird = 228u * 1024u / 3u - 1024u;   // bytes a CTA may take for three per SM
template <typename T, int SIGN, int NT>
__global__ void __launch_bounds__(NT, FftCtas<NT>::value) fft_rows_kernel(
    const cx_t<T>* __restrict__ in, long in_stride, int in_len, int in_shift,
    cx_t<T>* __restrict__ out, long out_stride, int out_len, int out_shift,
    int n, int Q, FftPlan1D plan, const cx_t<T>* __restrict__ tw, const int* __restrict__ perm,
    const T* __restrict__ pre_elem, const T* __restrict__ pre_row,
    const T* __restrict__ post_elem, const T* __restrict__ post_row, HermFold<T> hf, int io,
    const cx_t<T>* __restrict__ tw2, long in_batch, long out_batch, long out_es) {
    using C = cx_t<T>;
    constexpr bool inv = SIGN > 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    // blockIdx.z: grid of a batch of equal grids (right-hand sides), in_batch / out_batch apart
    in += blockIdx.z * in_batch;
    out += blockIdx.z * out_batch;
    if (hf.n) hf.base += blockIdx.z * in_batch;
    const long row = blockIdx.y;     // phases of a row are adjacent CTAs (they read the same row)
    const int r = blockIdx.x;
    const int nq = n / Q;
    // two-level twiddle table (if given) in shared memory after the row
    C* tws = nullptr;
    if (tw2) {
        tws = s + row_slots(nq);
        const int ntw = kTwLo + (n + kTwLo - 1) / kTwLo;
        for (int i = threadIdx.x; i < ntw; i += NT) tws[i] = tw2[i];
        __syncthreads();
    }
    const C* src = in + row * in_stride * (io == kIoPairInv ? 2 : 1);
    T rs0 = static_cast<T>(1), rs1 = static_cast<T>(1);
    if (pre_row) {
        rs0 = pre_row[io == kIoPairFwd ? 2 * row : row];
        rs1 = pre_row[io == kIoPairFwd ? 2 * row + 1 : row];
    }
    // load pass: element i of the length-nq transform (the Q phases folded and twisted) goes
    // to its digit-reversed position; consecutive threads read consecutive inputs.  One loop per
    // (io mode, fold, phases), chosen once per CTA.
    // With two or more stages the first one runs here too: in the digit-reversed order the group
    // of stage one at shared positions perm[t] + q (q < R1) holds the elements t + G1 q,
    // G1 = nq / R1; consecutive threads take consecutive t, so each of the R1 reads is coalesced,
    // and the group's butterfly runs before anything is stored.
    // (Fused for the odd first radices 3, 5, 9 and 15, which every row length here has; a row of
    // 2^k points takes the plain load, which keeps the number of instantiated loops small.)
    const int R1 = plan.radix[0];
    const bool fuse1 = plan.nstages >= 2 && (R1 == 3 || R1 == 5 || R1 == 9 || R1 == 15);
    const bool twist = Q == 2 && r != 0;
    auto load_pass = [&](auto io_c, auto fold_c, auto q_c) {
        constexpr int IO = decltype(io_c)::value;
        constexpr bool FOLD = decltype(fold_c)::value;
        constexpr int QQ = decltype(q_c)::value;
        // element i of the length-nq transform: the Q phases folded and twisted
        auto fetch = [&](int i) -> C {
            C acc = mk<T>(0, 0);
#pragma unroll
            for (int j = 0; j < QQ; ++j) {
                const int idx = i + j * nq;           // FFT index
                bool has;
                C v = load_elem<T, IO, FOLD>(idx, n, src, in_stride, in_len, in_shift, row, hf, rs0, rs1, pre_elem,
                                             has);
                if (has) {
                    if (QQ == 2 && twist) {           // twist w_n^{+-idx}
                        C w = twid<T>(tw, tws, idx);
                        if (inv) w.y = -w.y;
                        v = cmul(v, w);
                    }
                    acc = cadd(acc, v);
                }
            }
            return acc;
        };
        if (fuse1) {
            auto first = [&](auto rc) {
                constexpr int R = decltype(rc)::value;
                const int G1 = nq / R;
                for (int t = threadIdx.x; t < G1; t += NT) {
                    C v[R];
#pragma unroll
                    for (int q = 0; q < R; ++q) v[q] = fetch(t + G1 * q);
                    dft<T, R, SIGN>(v);
                    const int base = perm[t];
#pragma unroll
                    for (int q = 0; q < R; ++q) s[row_slot(base + q)] = v[q];
                }
            };
            if (R1 == 3) first(std::integral_constant<int, 3>{});
            else if (R1 == 5) first(std::integral_constant<int, 5>{});
            else if (sizeof(T) == 4 && R1 == 15) first(std::integral_constant<int, sizeof(T) == 4 ? 15 : 9>{});
            else first(std::integral_constant<int, 9>{});
        } else {
#pragma unroll 4
            for (int i = threadIdx.x; i < nq; i += NT) s[row_slot(perm[i])] = fetch(i);
        }
    };
    auto with_phases = [&](auto io_c, auto fold_c) {
        if (Q == 1) load_pass(io_c, fold_c, std::integral_constant<int, 1>{});
        else load_pass(io_c, fold_c, std::integral_constant<int, 2>{});
    };
    if (io == kIoPairInv) with_phases(std::integral_constant<int, kIoPairInv>{}, std::false_type{});
    else if (io == kIoPairFwd) with_phases(std::integral_constant<int, kIoPairFwd>{}, std::false_type{});
    else if (hf.n && hf.n - (hf.row0 + row) >= hf.lo)
        with_phases(std::integral_constant<int, kIoPlain>{}, std::true_type{});
    else with_phases(std::integral_constant<int, kIoPlain>{}, std::false_type{});
    __syncthreads();
    int Lp = fuse1 ? R1 : 1;
    // output scaling of the direct store (plain and pair-inverse rows)
    T ps0 = static_cast<T>(1), ps1 = static_cast<T>(1);
    if (post_row) {
        ps0 = post_row[io == kIoPairInv ? 2 * row : row];
        ps1 = post_row[io == kIoPairInv ? 2 * row + 1 : row];
    }
    C* dst = out + row * out_stride;
    // s position p holds FFT position Q p + r; element e of the output window is FFT
    // position (e + out_shift) mod n
    auto put = [&](int pos, C v) {
        const int kk = Q == 2 ? 2 * pos + r : pos;
        int e = kk - out_shift;
        if (e < 0) e += n;
        if (e < out_len) {
            const T pe = post_elem ? post_elem[e] : static_cast<T>(1);
            v.x *= ps0 * pe;
            v.y *= ps1 * pe;
            dst[e * out_es] = v;
        }
    };
    for (int st = fuse1 ? 1 : 0; st < plan.nstages; ++st) {
        const int R = plan.radix[st];
        if (st == plan.nstages - 1 && io != kIoPairFwd) {
            // last stage: outputs go straight to global memory (uniform branch, no barrier after)
            with_radix<T>(R, [&](auto rc) {
                dit_stage_out<T, decltype(rc)::value, SIGN>(s, nq, Lp, tw, tws, Q, NT, put);
            });
            return;
        }
        with_radix<T>(R, [&](auto rc) { dit_stage<T, decltype(rc)::value, SIGN>(s, nq, Lp, tw, tws, Q, NT); });
        Lp *= R;
    }
    // kIoPairFwd: s = Z^ of z = x0 + i x1 (two real rows): X0(k) = (Z(k) + conj Z(-k)) / 2,
    // X1(k) = (Z(k) - conj Z(-k)) / 2i, written to grid rows 2 row and 2 row + 1
    C* d0 = out + 2 * row * out_stride;
    C* d1 = d0 + out_stride;
    // with two phases this CTA holds the positions k of parity r: the elements e with e + out_shift
    // of that parity (n even), every other one
    const int e0 = Q == 2 ? ((r - out_shift) & 1) : 0;
    for (int e = e0 + Q * threadIdx.x; e < out_len; e += Q * NT) {
        int k = e + out_shift;
        if (k >= n) k -= n;
        const int km = k == 0 ? 0 : n - k;        // same parity as k (n even)
        const C zk = s[row_slot(Q == 2 ? (k >> 1) : k)], zm = s[row_slot(Q == 2 ? (km >> 1) : km)];
        const T h = static_cast<T>(0.5);
        const T pe = post_elem ? post_elem[e] : static_cast<T>(1);
        const C v0 = mk<T>(h * pe * (zk.x + zm.x), h * pe * (zk.y - zm.y));
        const C v1 = mk<T>(h * pe * (zk.y + zm.y), h * pe * (zm.x - zk.x));
        if constexpr (sizeof(T) == 4) {
            if (out_stride == 1) {        // written transposed: the two rows' values are neighbours
                *reinterpret_cast<float4*>(d0 + e * out_es) = make_float4(v0.x, v0.y, v1.x, v1.y);
                continue;
            }
        }
        d0[e * out_es] = v0;
        d1[e * out_es] = v1;
    }
}

// Digit-reversal permutation of the decimation-in-time schedule: with radices
// R_1..R_s applied in that order, index i = sum of digits (least significant digit in
// base R_s, then R_{s-1}, ...) lands at position sum_k d_k R_1...R_{k-1}.
const int* digit_perm(const FftPlan1D& plan, bool fp64, cudaStream_t stream) {
    static TableCache<int> cache;
    const int key = 2 * plan.n + (fp64 ? 1 : 0);     // the schedule depends on the precision
    if (const int* d = cache.find(key)) return d;
    const int n = plan.n;
    std::vector<int> h(n);
    std::vector<int> weight(plan.nstages);
    int w = 1;
    for (int k = 0; k < plan.nstages; ++k) { weight[k] = w; w *= plan.radix[k]; }
    for (int i = 0; i < n; ++i) {
        int v = i, pos = 0;
        for (int k = plan.nstages - 1; k >= 0; --k) {
            const int R = plan.radix[k];
            pos += (v % R) * weight[k];
            v /= R;
        }
        h[i] = pos;
    }
    return cache.upload(key, h, stream);
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

bool fft_make_plan(int n, FftPlan1D& p, bool fp64) {
    // Few stages of large radices: n = 2^a 3^b 5^c split into prime-power chunks (FP32: 16,
    // 9, 5; FP64: 8, 9, 5), each an in-register butterfly, the exponents of a prime spread
    // evenly over its chunks.  Odd radices first and the powers of two last: the early
    // stages, whose accesses are strided by the radix, then use odd strides (distinct
    // shared-memory banks), and the last stage, one butterfly per offset, writes
    // consecutive positions.
    p.n = n;
    p.nstages = 0;
    if (n < 2) return false;
    int v = n, e2 = 0, e3 = 0, e5 = 0;
    while (v % 2 == 0) { v /= 2; ++e2; }
    while (v % 3 == 0) { v /= 3; ++e3; }
    while (v % 5 == 0) { v /= 5; ++e5; }
    if (v != 1) return false;
    std::vector<int> rs;
    auto chunks = [&](int prime, int e, int emax) {
        if (e == 0) return;
        const int parts = (e + emax - 1) / emax;
        for (int i = 0; i < parts; ++i) {
            const int ei = e / parts + (i < e % parts ? 1 : 0);
            int r = 1;
            for (int j = 0; j < ei; ++j) r *= prime;
            rs.push_back(r);
        }
    };
    if (!fp64 && e3 == 1 && e5 == 1) {
        rs.push_back(15);                 // a lone 3 and a lone 5: one radix-15 stage (FP32)
    } else {
        chunks(5, e5, 1);
        chunks(3, e3, 2);
    }
    chunks(2, e2, fp64 ? 3 : 4);
    if (static_cast<int>(rs.size()) > kFftMaxStages) return false;
    for (size_t i = 0; i < rs.size(); ++i) p.radix[i] = rs[i];
    p.nstages = static_cast<int>(rs.size());
    return true;
}

int fft_max_row(bool fp64) {
    const int slots = 227 * 1024 / (fp64 ? 16 : 8);
    int n = fp64 ? MaxB<double>::n_max : MaxB<float>::n_max;
    while (row_slots(n) > slots) --n;
    return n;
}

static int fft_phases(int n, bool fp64);

// Phases per row: the smallest Q in {1, 2} whose length n / Q fits one CTA's shared memory.
static int fft_phases(int n, bool fp64) {
    const int lim = fft_max_row(fp64);
    if (n % 2 == 0 && n > lim) return 2;
    return 1;
}

int fft_max_length(bool fp64) { return 2 * fft_max_row(fp64); }

// Launches fft_rows_kernel<T, sign> (sign -1 or +1) with the shared-memory carveout at its
// maximum (all of the SM's unified memory as shared memory).
template <typename T, int SIGN, int NT, typename... A>
int launch_fft_rows_nt(dim3 grid, size_t smem, cudaStream_t stream, A... args) {
    auto k = fft_rows_kernel<T, SIGN, NT>;
    SBD_TRY(raise_smem_limit(k, smem));
    static const bool carve = [&] {
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaGetLastError();
        return true;
    }();
    (void)carve;
    k<<<grid, NT, smem, stream>>>(args...);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

// 384 threads where a CTA's shared memory leaves room for two CTAs per SM only, else 256 (three).
template <typename T, int SIGN, typename... A>
int launch_fft_rows_sign(dim3 grid, size_t smem, cudaStream_t stream, A... args) {
    if (smem > kFftSmemThird) return launch_fft_rows_nt<T, SIGN, 384>(grid, smem, stream, args...);
    return launch_fft_rows_nt<T, SIGN, 256>(grid, smem, stream, args...);
}

template <typename T, typename... A>
int launch_fft_rows(int sign, dim3 grid, size_t smem, cudaStream_t stream, A... args) {
    return sign < 0 ? launch_fft_rows_sign<T, -1>(grid, smem, stream, args...)
                    : launch_fft_rows_sign<T, 1>(grid, smem, stream, args...);
}

template <typename T>
int fft_rows(const cx_t<T>* in, long in_stride, int in_len, int in_shift,
             cx_t<T>* out, long out_stride, int out_len, int out_shift,
             int rows, int n, int sign,
             const T* pre_elem, const T* pre_row, const T* post_elem, const T* post_row,
             cudaStream_t stream, int herm_n, int herm_row0, int io, int split, int nb, long in_batch,
             long out_batch, long out_es, int herm_lo) {
    if (rows <= 0 || nb <= 0) return SBD_OK;
    if (nb > 65535) {
        set_error("fft_rows: at most 65535 grids per batch");
        return SBD_EINVAL;
    }
    if (herm_n && (herm_row0 < 0 || herm_row0 + rows > herm_n || in_len != herm_n || io != kIoPlain)) {
        set_error("fft_rows: a Hermitian fold needs rows inside a square grid read whole");
        return SBD_EINVAL;
    }
    if (io < kIoPlain || io > kIoPairInv) {
        set_error("fft_rows: unknown io mode");
        return SBD_EINVAL;
    }
    const bool fp64 = sizeof(T) == 8;
    const int Q = split == 2 && n % 2 == 0 ? 2 : fft_phases(n, fp64);
    const int nq = n / Q;
    FftPlan1D plan;
    if (!fft_make_plan(nq, plan, fp64) || nq > fft_max_row(fp64) || n % Q) {
        set_error("FFT length not supported: " + std::to_string(n));
        return SBD_ENOTSUP;
    }
    const cx_t<T>* tw = twiddles<T>(n, stream);
    const int* perm = digit_perm(plan, fp64, stream);
    if (!tw || !perm) {
        set_error("FFT table allocation failed");
        return SBD_ENOMEM;
    }
    // the two-level twiddle table rides in shared memory when it fits beside the row
    const size_t row_bytes = sizeof(cx_t<T>) * static_cast<size_t>(row_slots(nq));
    const size_t tw2_bytes = sizeof(cx_t<T>) * static_cast<size_t>(tw2_size(n));
    const cx_t<T>* tw2 = row_bytes + tw2_bytes <= 227u * 1024u ? twiddles2<T>(n, stream) : nullptr;
    const size_t smem = row_bytes + (tw2 ? tw2_bytes : 0);
    in_shift = ((in_shift % n) + n) % n;
    out_shift = ((out_shift % n) + n) % n;
    for (int r0 = 0; r0 < rows; r0 += 65535) {          // grid.y holds at most 65535 rows
        const int nr = std::min(65535, rows - r0);
        const dim3 grid(static_cast<unsigned>(Q), static_cast<unsigned>(nr), static_cast<unsigned>(nb));
        // pair modes: one launch row is two grid rows on the paired side
        const long in_rows = io == kIoPairInv ? 2 : 1, out_rows = io == kIoPairFwd ? 2 : 1;
        const cx_t<T>* ip = in + static_cast<long>(r0) * in_stride * in_rows;
        cx_t<T>* op = out + static_cast<long>(r0) * out_stride * out_rows;
        const T* prr = pre_row ? pre_row + r0 * (io == kIoPairFwd ? 2 : 1) : nullptr;
        const T* por = post_row ? post_row + r0 * (io == kIoPairInv ? 2 : 1) : nullptr;
        const HermFold<T> hf{in - static_cast<long>(herm_row0) * in_stride, herm_n,
                             static_cast<long>(herm_row0) + r0, herm_lo};
        // half-length phases (split) fit more CTAs per SM
        const int rc = launch_fft_rows<T>(sign, grid, smem, stream, ip, in_stride, in_len, in_shift, op, out_stride,
                                          out_len, out_shift, n, Q, plan, tw, perm, pre_elem, prr, post_elem, por,
                                          hf, io, tw2, in_batch, out_batch, out_es);
        if (rc) return rc;
    }
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int fft_rows_tables(const cx_t<T>* in, long in_stride, int in_len, cx_t<T>* out, long out_stride, int out_len,
                    int rows, int n, int sign, const cx_t<T>* tw, const int* perm, cudaStream_t stream) {
    if (rows <= 0) return SBD_OK;
    FftPlan1D plan;
    if (!fft_make_plan(n, plan, sizeof(T) == 8) || n > fft_max_row(sizeof(T) == 8)) {
        set_error("FFT length not supported: " + std::to_string(n));
        return SBD_ENOTSUP;
    }
    const size_t smem = sizeof(cx_t<T>) * static_cast<size_t>(row_slots(n));
    for (int r0 = 0; r0 < rows; r0 += 65535) {
        const int nr = std::min(65535, rows - r0);
        const dim3 grid(1u, static_cast<unsigned>(nr));
        const cx_t<T>* ip = in + static_cast<long>(r0) * in_stride;
        cx_t<T>* op = out + static_cast<long>(r0) * out_stride;
        const T* none = nullptr;
        const int rc = launch_fft_rows<T>(sign, grid, smem, stream, ip, in_stride, in_len, 0, op, out_stride,
                                          out_len, 0, n, 1, plan, tw, perm, none, none, none, none,
                                          HermFold<T>{nullptr, 0, 0, 0}, static_cast<int>(kIoPlain),
                                          static_cast<const cx_t<T>*>(nullptr), 0L, 0L, 1L);
        if (rc) return rc;
    }
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
                             const float*, const float*, const float*, const float*, cudaStream_t, int, int,
                             int, int, int, long, long, long, int);
template int fft_rows<double>(const double2*, long, int, int, double2*, long, int, int, int, int, int,
                              const double*, const double*, const double*, const double*, cudaStream_t, int, int,
                              int, int, int, long, long, long, int);
template int fft_rows_tables<float>(const float2*, long, int, float2*, long, int, int, int, int, const float2*,
                                    const int*, cudaStream_t);
template int fft_rows_tables<double>(const double2*, long, int, double2*, long, int, int, int, int, const double2*,
                                     const int*, cudaStream_t);
template int transpose<float>(const float2*, long, long, float2*, long, long, int, int, int, cudaStream_t);
template int transpose<double>(const double2*, long, long, double2*, long, long, int, int, int, cudaStream_t);

}  // namespace sbd
