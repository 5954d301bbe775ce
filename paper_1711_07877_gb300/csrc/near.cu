// Near-field kernels: cell list, neighbour search, D values (FP64), CSR SpMV.
#include <algorithm>
#include <cmath>

#include "near.cuh"
#include "sbd.h"

namespace sbd {

namespace {

constexpr int kT = 256;
inline unsigned nblk(long n, int t = kT) { return static_cast<unsigned>((n + t - 1) / t); }

__device__ __forceinline__ double atomic_min_d(double* addr, double v) {
    unsigned long long* a = reinterpret_cast<unsigned long long*>(addr);
    unsigned long long old = *a, assumed;
    do {
        assumed = old;
        if (__longlong_as_double(assumed) <= v) break;
        old = atomicCAS(a, assumed, __double_as_longlong(v));
    } while (assumed != old);
    return __longlong_as_double(old);
}
__device__ __forceinline__ double atomic_max_d(double* addr, double v) {
    unsigned long long* a = reinterpret_cast<unsigned long long*>(addr);
    unsigned long long old = *a, assumed;
    do {
        assumed = old;
        if (__longlong_as_double(assumed) >= v) break;
        old = atomicCAS(a, assumed, __double_as_longlong(v));
    } while (assumed != old);
    return __longlong_as_double(old);
}

__global__ void bbox_kernel(const double* __restrict__ z, long n, double* out) {
    double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        const double x = z[2 * i], y = z[2 * i + 1];
        x0 = fmin(x0, x); y0 = fmin(y0, y); x1 = fmax(x1, x); y1 = fmax(y1, y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fmin(x0, __shfl_down_sync(0xffffffffu, x0, o));
        y0 = fmin(y0, __shfl_down_sync(0xffffffffu, y0, o));
        x1 = fmax(x1, __shfl_down_sync(0xffffffffu, x1, o));
        y1 = fmax(y1, __shfl_down_sync(0xffffffffu, y1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_min_d(&out[0], x0); atomic_min_d(&out[1], y0);
        atomic_max_d(&out[2], x1); atomic_max_d(&out[3], y1);
    }
}

__global__ void maxd2_kernel(const double* __restrict__ z, long n, double cx, double cy, double* out) {
    double m = 0.0;
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        const double dx = z[2 * i] - cx, dy = z[2 * i + 1] - cy;
        m = fmax(m, dx * dx + dy * dy);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_d(out, m);
}

// |z_k - z_l|^2 rounded the same way everywhere it is compared with delta_min^2
// (no contraction into FMA), so the counting and filling passes agree bit for bit.
__device__ __forceinline__ double dist2(double x, double y, double x2, double y2) {
    const double dx = __dsub_rn(x, x2), dy = __dsub_rn(y, y2);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

struct CellGrid {
    double x0, y0, inv;   // inv = 1 / cell size
    int ncx, ncy;
};

__device__ __forceinline__ int2 cell_of(const CellGrid& g, double x, double y) {
    int cx = static_cast<int>(floor((x - g.x0) * g.inv));
    int cy = static_cast<int>(floor((y - g.y0) * g.inv));
    cx = min(max(cx, 0), g.ncx - 1);
    cy = min(max(cy, 0), g.ncy - 1);
    return make_int2(cx, cy);
}

__global__ void cell_count_kernel(const double* __restrict__ z, long n, CellGrid g, int* __restrict__ cell_of_pt,
                                  long long* __restrict__ count) {
    const long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int2 c = cell_of(g, z[2 * i], z[2 * i + 1]);
    const int id = c.y * g.ncx + c.x;
    cell_of_pt[i] = id;
    atomicAdd(reinterpret_cast<unsigned long long*>(&count[id]), 1ULL);
}

__global__ void cell_fill_kernel(long n, const int* __restrict__ cell_of_pt, const long long* __restrict__ start,
                                 int* __restrict__ cursor, int* __restrict__ sorted) {
    const long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int id = cell_of_pt[i];
    const int k = atomicAdd(&cursor[id], 1);
    sorted[start[id] + k] = static_cast<int>(i);
}

// insertion sort of each cell's members by point index (deterministic CSR column order)
__global__ void cell_sort_kernel(long ncells, const long long* __restrict__ start, int* __restrict__ sorted) {
    const long c = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (c >= ncells) return;
    const long b = start[c], e = start[c + 1];
    for (long i = b + 1; i < e; ++i) {
        const int v = sorted[i];
        long j = i - 1;
        while (j >= b && sorted[j] > v) {
            sorted[j + 1] = sorted[j];
            --j;
        }
        sorted[j + 1] = v;
    }
}

// Row k of D: the query point zq[k] (a target) against the points z (the sources) in the 3 x 3
// cells around it.  square: zq is z, the row holds its diagonal first and skips l == k.
__global__ void neighbour_count_kernel(const double* __restrict__ z, const double* __restrict__ zq, long nq,
                                       bool square, CellGrid g, double d2, const long long* __restrict__ start,
                                       const int* __restrict__ sorted, long long* __restrict__ cnt) {
    const long k = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (k >= nq) return;
    const double x = zq[2 * k], y = zq[2 * k + 1];
    const int2 c = cell_of(g, x, y);
    long long m = square ? 1 : 0;   // the diagonal
    for (int cy = max(c.y - 1, 0); cy <= min(c.y + 1, g.ncy - 1); ++cy)
        for (int cx = max(c.x - 1, 0); cx <= min(c.x + 1, g.ncx - 1); ++cx) {
            const int id = cy * g.ncx + cx;
            for (long long j = start[id]; j < start[id + 1]; ++j) {
                const int l = sorted[j];
                if (square && l == k) continue;
                if (dist2(x, y, z[2 * l], z[2 * l + 1]) <= d2) ++m;
            }
        }
    cnt[k] = m;
}

__device__ double2 clenshaw2(const double* __restrict__ c, int deg, double tt) {
    double br1 = 0.0, bi1 = 0.0, br2 = 0.0, bi2 = 0.0;
    for (int j = deg - 1; j >= 1; --j) {
        const double nr = 2.0 * tt * br1 - br2 + c[2 * j];
        const double ni = 2.0 * tt * bi1 - bi2 + c[2 * j + 1];
        br2 = br1; bi2 = bi1;
        br1 = nr;  bi1 = ni;
    }
    return make_double2(tt * br1 - br2 + c[0], tt * bi1 - bi2 + c[1]);
}

__device__ double2 d_value(const NearDev& tb, double yx, double yy) {
    const double t = yx * yx + yy * yy;
    const double u = tb.in_r ? sqrt(t) : t;          // the tables' variable
    const double w = tb.tmax / tb.pieces;
    int q = static_cast<int>(u / w);
    q = min(q, tb.pieces - 1);
    const double tt = 2.0 * (u / w - q) - 1.0;
    const double2 a1 = clenshaw2(tb.T1 + static_cast<long>(q) * tb.deg * 2, tb.deg, tt);
    const double2 a2 = clenshaw2(tb.T2 + static_cast<long>(q) * tb.deg * 2, tb.deg, tt);
    const double lg = 0.5 * log(t);
    double vr = a1.x * lg + a2.x, vi = a1.y * lg + a2.y;
    for (int s = 0; s < tb.n_small; ++s) {
        double acc = 0.0;
        for (int j = tb.small_start[s]; j < tb.small_start[s + 1]; ++j)
            acc += cos(yx * tb.small_xi[2 * j] + yy * tb.small_xi[2 * j + 1]);
        vr -= tb.small_w[2 * s] * acc;
        vi -= tb.small_w[2 * s + 1] * acc;
    }
    return make_double2(vr, vi);
}

__global__ void neighbour_fill_kernel(const double* __restrict__ z, const double* __restrict__ zq, long nq,
                                      bool square, CellGrid g, double d2,
                                      const long long* __restrict__ start, const int* __restrict__ sorted,
                                      const long long* __restrict__ rowptr, int* __restrict__ col,
                                      void* __restrict__ val, bool cval, NearDev tb,
                                      unsigned long long* __restrict__ n_coinc) {
    const long k = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (k >= nq) return;
    const double x = zq[2 * k], y = zq[2 * k + 1];
    const int2 c = cell_of(g, x, y);
    long long o = rowptr[k];
    const long long o_end = rowptr[k + 1];
    if (square) {
        col[o] = static_cast<int>(k);
        if (cval) static_cast<double2*>(val)[o] = make_double2(tb.self_re, tb.self_im);
        else static_cast<double*>(val)[o] = tb.self_re;
        ++o;
    }
    for (int cy = max(c.y - 1, 0); cy <= min(c.y + 1, g.ncy - 1); ++cy)
        for (int cx = max(c.x - 1, 0); cx <= min(c.x + 1, g.ncx - 1); ++cx) {
            const int id = cy * g.ncx + cx;
            for (long long j = start[id]; j < start[id + 1]; ++j) {
                const int l = sorted[j];
                if (square && l == k) continue;
                const double t = dist2(x, y, z[2 * l], z[2 * l + 1]);
                if (t > d2 || o >= o_end) continue;
                const double dx = x - z[2 * l], dy = y - z[2 * l + 1];
                double2 v;
                if (t == 0.0) {
                    v = make_double2(tb.self_re, tb.self_im);   // coincident points: as the self pair
                    atomicAdd(n_coinc, 1ULL);
                } else {
                    v = d_value(tb, dx, dy);
                }
                col[o] = l;
                if (cval) static_cast<double2*>(val)[o] = v;
                else static_cast<double*>(val)[o] = v.x;
                ++o;
            }
        }
}

template <bool CPLX>
__global__ void spmv_kernel(const long long* __restrict__ rowptr, const int* __restrict__ col,
                            const void* __restrict__ val, long n, int nrhs, const void* __restrict__ f,
                            void* __restrict__ q, bool acc) {
    const long row = (blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const long long b = rowptr[row], e = rowptr[row + 1];
    for (int r = 0; r < nrhs; ++r) {
        double sr = 0.0, si = 0.0;
        if (CPLX) {
            const double2* v = static_cast<const double2*>(val);
            const double2* fr = static_cast<const double2*>(f) + r * n;
            for (long long j = b + lane; j < e; j += 32) {
                const double2 a = v[j], x = fr[col[j]];
                sr += a.x * x.x - a.y * x.y;
                si += a.x * x.y + a.y * x.x;
            }
        } else {
            const double* v = static_cast<const double*>(val);
            const double* fr = static_cast<const double*>(f) + r * n;
            for (long long j = b + lane; j < e; j += 32) sr += v[j] * fr[col[j]];
        }
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, o);
            si += __shfl_down_sync(0xffffffffu, si, o);
        }
        if (lane == 0) {
            if (CPLX) {
                double2* qr = static_cast<double2*>(q) + r * n + row;
                if (acc) { qr->x += sr; qr->y += si; }
                else *qr = make_double2(sr, si);
            } else {
                double* qr = static_cast<double*>(q) + r * n + row;
                if (acc) *qr += sr;
                else *qr = sr;
            }
        }
    }
}

// qp = D fp for one right-hand side in FP64 (values, products and sums), G lanes per row:
// a warp takes 32 / G rows, and the G lanes of a row read consecutive entries, so one
// warp-wide load covers 32 / G rows' contiguous segments.  Against a warp per row this
// cuts the FP64 shuffle-adds of the row reduction from 5 per row to log2(G) per 32 / G
// rows (GB300's FP64 pipe is narrow, and with ~10^2 entries a row the warp-wide
// reduction cost as much FP64 issue as the products).  Whole warps run the reduction
// (rows past n only contribute zeros), so the shuffles see every lane.
template <bool CPLX, int G>
__global__ void spmv_group_kernel(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                  const void* __restrict__ val, long n, const void* __restrict__ fp,
                                  void* __restrict__ qp) {
    const long row = (blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x) / G;
    const int sub = threadIdx.x & (G - 1);
    const bool live = row < n;
    long long b = 0, e = 0;
    if (live) {
        b = rowptr[row];
        e = rowptr[row + 1];
    }
    double sr = 0.0, si = 0.0;
    if (CPLX) {
        const double2* v = static_cast<const double2*>(val);
        const double2* x = static_cast<const double2*>(fp);
        for (long long j = b + sub; j < e; j += G) {
            const double2 a = v[j], y = x[col[j]];
            sr = fma(a.x, y.x, fma(-a.y, y.y, sr));
            si = fma(a.x, y.y, fma(a.y, y.x, si));
        }
    } else {
        const double* v = static_cast<const double*>(val);
        const double* x = static_cast<const double*>(fp);
        for (long long j = b + sub; j < e; j += G) sr = fma(v[j], x[col[j]], sr);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o, G);
        if (CPLX) si += __shfl_down_sync(0xffffffffu, si, o, G);
    }
    if (live && sub == 0) {
        if (CPLX) static_cast<double2*>(qp)[row] = make_double2(sr, si);
        else static_cast<double*>(qp)[row] = sr;
    }
}

// Internal (spatially sorted) order: fp[i * nrhs + r] = f[r * n + perm[i]].
template <bool CPLX, bool F32>
__global__ void gather_rows_kernel(const void* __restrict__ f, long n, int nrhs, const int* __restrict__ perm,
                                   void* __restrict__ fp) {
    const long t = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (t >= n * nrhs) return;
    const long i = t / nrhs;
    const int r = static_cast<int>(t - i * nrhs);
    const long src = static_cast<long>(r) * n + perm[i];
    if (CPLX) {
        const double2 v = static_cast<const double2*>(f)[src];
        if (F32) static_cast<float2*>(fp)[t] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
        else static_cast<double2*>(fp)[t] = v;
    } else {
        const double v = static_cast<const double*>(f)[src];
        if (F32) static_cast<float*>(fp)[t] = static_cast<float>(v);
        else static_cast<double*>(fp)[t] = v;
    }
}

// q[r * n + perm[i]] = qp[i * nrhs + r]
template <bool CPLX>
__global__ void scatter_rows_kernel(const void* __restrict__ qp, long n, int nrhs, const int* __restrict__ perm,
                                    void* __restrict__ q) {
    const long t = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (t >= n * nrhs) return;
    const long i = t / nrhs;
    const int r = static_cast<int>(t - i * nrhs);
    const long dst = static_cast<long>(r) * n + perm[i];
    if (CPLX) static_cast<double2*>(q)[dst] = static_cast<const double2*>(qp)[t];
    else static_cast<double*>(q)[dst] = static_cast<const double*>(qp)[t];
}

// qp = D fp with interleaved right-hand sides, one thread per (row, rhs): the threads
// of a row share its column and value loads and read fp[col * nrhs + 0..nrhs-1]
// contiguously.  Rows and columns are in the internal order, so the columns of a row
// are nearby points whose values sit close together.
template <bool CPLX>
__global__ void spmv_rhs_kernel(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const void* __restrict__ val, long n, int nrhs, const void* __restrict__ fp,
                                void* __restrict__ qp) {
    const long t = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (t >= n * nrhs) return;
    const long row = t / nrhs;
    const int r = static_cast<int>(t - row * nrhs);
    const long long b = rowptr[row], e = rowptr[row + 1];
    if (CPLX) {
        const double2* v = static_cast<const double2*>(val);
        const double2* x = static_cast<const double2*>(fp);
        double sr = 0.0, si = 0.0;
        for (long long j = b; j < e; ++j) {
            const double2 a = v[j], y = x[static_cast<long>(col[j]) * nrhs + r];
            sr += a.x * y.x - a.y * y.y;
            si += a.x * y.y + a.y * y.x;
        }
        static_cast<double2*>(qp)[t] = make_double2(sr, si);
    } else {
        const double* v = static_cast<const double*>(val);
        const double* x = static_cast<const double*>(fp);
        double acc = 0.0;
        for (long long j = b; j < e; ++j) acc += v[j] * x[static_cast<long>(col[j]) * nrhs + r];
        static_cast<double*>(qp)[t] = acc;
    }
}

// FP32 storage of D and of the gathered f (the FP32 form): products and the per-lane
// (per-thread) partial sums in FP32, the partials of a row combined in FP64.
template <bool CPLX> struct F32Val;
template <> struct F32Val<false> { using V = float; };
template <> struct F32Val<true> { using V = float2; };
__device__ __forceinline__ void mac32(float& sr, float& si, float a, float x) { sr = fmaf(a, x, sr); (void)si; }
__device__ __forceinline__ void mac32(float& sr, float& si, float2 a, float2 x) {
    sr = fmaf(a.x, x.x, fmaf(-a.y, x.y, sr));
    si = fmaf(a.x, x.y, fmaf(a.y, x.x, si));
}

template <bool CPLX>
__global__ void spmv32_kernel(const long long* __restrict__ rowptr, const int* __restrict__ col,
                              const void* __restrict__ val, long n, const void* __restrict__ fp,
                              void* __restrict__ qp) {
    using V = typename F32Val<CPLX>::V;
    const long row = (blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const long long b = rowptr[row], e = rowptr[row + 1];
    const V* v = static_cast<const V*>(val);
    const V* x = static_cast<const V*>(fp);
    float pr = 0.f, pi = 0.f;
    for (long long j = b + lane; j < e; j += 32) mac32(pr, pi, v[j], x[col[j]]);
    double sr = pr, si = pi;
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        if (CPLX) si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
        if (CPLX) static_cast<double2*>(qp)[row] = make_double2(sr, si);
        else static_cast<double*>(qp)[row] = sr;
    }
}

template <bool CPLX>
__global__ void spmv32_rhs_kernel(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                  const void* __restrict__ val, long n, int nrhs, const void* __restrict__ fp,
                                  void* __restrict__ qp) {
    using V = typename F32Val<CPLX>::V;
    const long t = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (t >= n * nrhs) return;
    const long row = t / nrhs;
    const int r = static_cast<int>(t - row * nrhs);
    const long long b = rowptr[row], e = rowptr[row + 1];
    const V* v = static_cast<const V*>(val);
    const V* x = static_cast<const V*>(fp);
    // two partial sums (entries of even and odd offset) keep two loads in flight
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
    long long j = b;
    for (; j + 1 < e; j += 2) {
        const int c0 = col[j], c1 = col[j + 1];
        const V a0 = v[j], a1 = v[j + 1];
        const V x0 = x[static_cast<long>(c0) * nrhs + r], x1 = x[static_cast<long>(c1) * nrhs + r];
        mac32(ar, ai, a0, x0);
        mac32(br, bi, a1, x1);
    }
    if (j < e) mac32(ar, ai, v[j], x[static_cast<long>(col[j]) * nrhs + r]);
    const double sr = static_cast<double>(ar) + br, si = static_cast<double>(ai) + bi;
    if (CPLX) static_cast<double2*>(qp)[t] = make_double2(sr, si);
    else static_cast<double*>(qp)[t] = sr;
}

__global__ void to_f32_kernel(const double* __restrict__ in, long count, float* __restrict__ out) {
    const long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (i < count) out[i] = static_cast<float>(in[i]);
}

// --- exclusive scan of 64-bit integers: per-chunk scan, chunk totals, offsets ------------
constexpr int kScanT = 1024, kScanPer = 4, kChunk = kScanT * kScanPer;

__global__ void scan_chunks_kernel(long long* __restrict__ d, long n, long long* __restrict__ totals) {
    __shared__ long long warp_tot[32];
    const long base = static_cast<long>(blockIdx.x) * kChunk + threadIdx.x * kScanPer;
    long long v[kScanPer];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = (base + i < n) ? d[base + i] : 0;
        s += v[i];
    }
    // inclusive scan of the per-thread sums across the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    long long excl = x - s + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) d[base + i] = excl;
        excl += v[i];
    }
    if (threadIdx.x == kScanT - 1) totals[blockIdx.x] = excl;
}

__global__ void scan_add_kernel(long long* __restrict__ d, long n, const long long* __restrict__ offs) {
    const long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (i < n) d[i] += offs[i / kChunk];
}

}  // namespace

int scan_exclusive_i64(long long* data, long n, long long* total, cudaStream_t s) {
    if (n <= 0) {
        *total = 0;
        return SBD_OK;
    }
    const long nch = (n + kChunk - 1) / kChunk;
    long long* tot = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&tot, sizeof(long long) * (nch + 1), s));
    scan_chunks_kernel<<<static_cast<unsigned>(nch), kScanT, 0, s>>>(data, n, tot);
    SBD_LAUNCH_CHECK();
    if (nch > 1) {
        long long t2 = 0;
        int rc = scan_exclusive_i64(tot, nch, &t2, s);
        if (rc) return rc;
        scan_add_kernel<<<nblk(n), kT, 0, s>>>(data, n, tot);
        SBD_LAUNCH_CHECK();
        *total = t2;
    } else {
        SBD_CUDA_TRY(cudaMemcpyAsync(total, tot, sizeof(long long), cudaMemcpyDeviceToHost, s));
        SBD_CUDA_TRY(cudaStreamSynchronize(s));
    }
    SBD_CUDA_TRY(cudaFreeAsync(tot, s));
    SBD_CUDA_TRY(cudaStreamSynchronize(s));
    return SBD_OK;
}

int points_bbox(const double* z, long n, double* out4_host, cudaStream_t s) {
    double* d = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * 4, s));
    const double init[4] = {1e300, 1e300, -1e300, -1e300};
    SBD_CUDA_TRY(cudaMemcpyAsync(d, init, sizeof init, cudaMemcpyHostToDevice, s));
    bbox_kernel<<<static_cast<unsigned>(std::min<long>(nblk(n), 1024)), kT, 0, s>>>(z, n, d);
    SBD_LAUNCH_CHECK();
    SBD_CUDA_TRY(cudaMemcpyAsync(out4_host, d, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    SBD_CUDA_TRY(cudaFreeAsync(d, s));
    SBD_CUDA_TRY(cudaStreamSynchronize(s));
    return SBD_OK;
}

int points_max_dist2(const double* z, long n, double cx, double cy, double* out_host, cudaStream_t s) {
    double* d = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&d, sizeof(double), s));
    SBD_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(double), s));
    maxd2_kernel<<<static_cast<unsigned>(std::min<long>(nblk(n), 1024)), kT, 0, s>>>(z, n, cx, cy, d);
    SBD_LAUNCH_CHECK();
    SBD_CUDA_TRY(cudaMemcpyAsync(out_host, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    SBD_CUDA_TRY(cudaFreeAsync(d, s));
    SBD_CUDA_TRY(cudaStreamSynchronize(s));
    return SBD_OK;
}

int near_build(const double* z, long n, double delta_min, double bx0, double by0, double bx1, double by1,
               const NearDev& tab, bool cval, long long** rowptr_out, int** col_out, void** val_out,
               long long* nnz_out, long long* n_coinc_out, cudaStream_t s, const double* zq, long nq) {
    const bool square = zq == nullptr;
    if (square) {
        zq = z;
        nq = n;
    }
    CellGrid g;
    double cell = delta_min;
    // keep the cell table modest: enlarge cells (still >= delta_min) if needed
    for (;;) {
        const double ncx = std::floor((bx1 - bx0) / cell) + 1, ncy = std::floor((by1 - by0) / cell) + 1;
        if (ncx * ncy <= 6.7e7) {
            g.ncx = static_cast<int>(ncx);
            g.ncy = static_cast<int>(ncy);
            break;
        }
        cell *= 1.5;
    }
    g.x0 = bx0;
    g.y0 = by0;
    g.inv = 1.0 / cell;
    const long ncells = static_cast<long>(g.ncx) * g.ncy;
    int* cell_of_pt = nullptr;
    long long* cstart = nullptr;
    int* cursor = nullptr;
    int* sorted = nullptr;
    long long* cnt = nullptr;
    unsigned long long* coinc = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&cell_of_pt, sizeof(int) * n, s));
    SBD_CUDA_TRY(cudaMallocAsync(&cstart, sizeof(long long) * (ncells + 1), s));
    SBD_CUDA_TRY(cudaMallocAsync(&cursor, sizeof(int) * ncells, s));
    SBD_CUDA_TRY(cudaMallocAsync(&sorted, sizeof(int) * n, s));
    SBD_CUDA_TRY(cudaMallocAsync(&coinc, sizeof(unsigned long long), s));
    SBD_CUDA_TRY(cudaMemsetAsync(cstart, 0, sizeof(long long) * (ncells + 1), s));
    SBD_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * ncells, s));
    SBD_CUDA_TRY(cudaMemsetAsync(coinc, 0, sizeof(unsigned long long), s));
    cell_count_kernel<<<nblk(n), kT, 0, s>>>(z, n, g, cell_of_pt, cstart);
    SBD_LAUNCH_CHECK();
    long long tot = 0;
    int rc = scan_exclusive_i64(cstart, ncells + 1, &tot, s);
    if (rc) return rc;
    cell_fill_kernel<<<nblk(n), kT, 0, s>>>(n, cell_of_pt, cstart, cursor, sorted);
    SBD_LAUNCH_CHECK();
    cell_sort_kernel<<<nblk(ncells), kT, 0, s>>>(ncells, cstart, sorted);
    SBD_LAUNCH_CHECK();
    const double d2 = delta_min * delta_min;
    long long* rowptr = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&rowptr, sizeof(long long) * (nq + 1), s));
    SBD_CUDA_TRY(cudaMemsetAsync(rowptr, 0, sizeof(long long) * (nq + 1), s));
    neighbour_count_kernel<<<nblk(nq), kT, 0, s>>>(z, zq, nq, square, g, d2, cstart, sorted, rowptr);
    SBD_LAUNCH_CHECK();
    long long nnz = 0;
    rc = scan_exclusive_i64(rowptr, nq + 1, &nnz, s);
    if (rc) return rc;
    int* col = nullptr;
    void* val = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&col), sizeof(int) * std::max<long long>(nnz, 1), s));
    SBD_CUDA_TRY(cudaMallocAsync(&val, (cval ? 16 : 8) * std::max<long long>(nnz, 1), s));
    neighbour_fill_kernel<<<nblk(nq, 128), 128, 0, s>>>(z, zq, nq, square, g, d2, cstart, sorted, rowptr, col, val,
                                                        cval, tab, coinc);
    SBD_LAUNCH_CHECK();
    unsigned long long nc = 0;
    SBD_CUDA_TRY(cudaMemcpyAsync(&nc, coinc, sizeof nc, cudaMemcpyDeviceToHost, s));
    SBD_CUDA_TRY(cudaFreeAsync(cell_of_pt, s));
    SBD_CUDA_TRY(cudaFreeAsync(cstart, s));
    SBD_CUDA_TRY(cudaFreeAsync(cursor, s));
    SBD_CUDA_TRY(cudaFreeAsync(sorted, s));
    SBD_CUDA_TRY(cudaFreeAsync(coinc, s));
    SBD_CUDA_TRY(cudaStreamSynchronize(s));
    *rowptr_out = rowptr;
    *col_out = col;
    *val_out = val;
    *nnz_out = nnz;
    *n_coinc_out = static_cast<long long>(nc);
    return SBD_OK;
}

int near_spmv(const long long* rowptr, const int* col, const void* val, bool cval, long n, int nrhs,
              const void* f, void* q, bool accumulate, cudaStream_t s) {
    if (n <= 0) return SBD_OK;
    const long threads = n * 32;
    if (cval) spmv_kernel<true><<<nblk(threads), kT, 0, s>>>(rowptr, col, val, n, nrhs, f, q, accumulate);
    else spmv_kernel<false><<<nblk(threads), kT, 0, s>>>(rowptr, col, val, n, nrhs, f, q, accumulate);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

int near_gather(const void* f, bool cplx, long n, int nrhs, const int* perm, void* fp, cudaStream_t s, bool f32) {
    if (n <= 0) return SBD_OK;
    const long t = n * nrhs;
    if (cplx) {
        if (f32) gather_rows_kernel<true, true><<<nblk(t), kT, 0, s>>>(f, n, nrhs, perm, fp);
        else gather_rows_kernel<true, false><<<nblk(t), kT, 0, s>>>(f, n, nrhs, perm, fp);
    } else {
        if (f32) gather_rows_kernel<false, true><<<nblk(t), kT, 0, s>>>(f, n, nrhs, perm, fp);
        else gather_rows_kernel<false, false><<<nblk(t), kT, 0, s>>>(f, n, nrhs, perm, fp);
    }
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

int near_values_to_f32(void** val, long long nnz, bool cplx, cudaStream_t s) {
    const long count = static_cast<long>(nnz) * (cplx ? 2 : 1);
    float* out = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&out, sizeof(float) * std::max(count, 1L), s));
    if (count > 0) {
        to_f32_kernel<<<nblk(count), kT, 0, s>>>(static_cast<const double*>(*val), count, out);
        SBD_LAUNCH_CHECK();
    }
    SBD_CUDA_TRY(cudaFreeAsync(*val, s));
    *val = out;
    return SBD_OK;
}

int near_scatter(const void* qp, bool cplx, long n, int nrhs, const int* perm, void* q, cudaStream_t s) {
    if (n <= 0) return SBD_OK;
    const long t = n * nrhs;
    if (cplx) scatter_rows_kernel<true><<<nblk(t), kT, 0, s>>>(qp, n, nrhs, perm, q);
    else scatter_rows_kernel<false><<<nblk(t), kT, 0, s>>>(qp, n, nrhs, perm, q);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

int near_spmv_internal(const long long* rowptr, const int* col, const void* val, bool cval, long n, int nrhs,
                       const void* fp, void* qp, cudaStream_t s, bool f32) {
    if (n <= 0) return SBD_OK;
    if (f32) {
        if (nrhs == 1) {
            const long threads = n * 32;
            if (cval) spmv32_kernel<true><<<nblk(threads), kT, 0, s>>>(rowptr, col, val, n, fp, qp);
            else spmv32_kernel<false><<<nblk(threads), kT, 0, s>>>(rowptr, col, val, n, fp, qp);
        } else {
            const long t = n * nrhs;
            if (cval) spmv32_rhs_kernel<true><<<nblk(t), kT, 0, s>>>(rowptr, col, val, n, nrhs, fp, qp);
            else spmv32_rhs_kernel<false><<<nblk(t), kT, 0, s>>>(rowptr, col, val, n, nrhs, fp, qp);
        }
    } else if (nrhs == 1) {   // 8 lanes per row (rows of ~10^2 entries), FP64 throughout
        constexpr int G = 8;
        const long threads = n * G;
        if (cval) spmv_group_kernel<true, G><<<nblk(threads), kT, 0, s>>>(rowptr, col, val, n, fp, qp);
        else spmv_group_kernel<false, G><<<nblk(threads), kT, 0, s>>>(rowptr, col, val, n, fp, qp);
    } else {
        const long t = n * nrhs;
        if (cval) spmv_rhs_kernel<true><<<nblk(t), kT, 0, s>>>(rowptr, col, val, n, nrhs, fp, qp);
        else spmv_rhs_kernel<false><<<nblk(t), kT, 0, s>>>(rowptr, col, val, n, nrhs, fp, qp);
    }
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

}  // namespace sbd
