// Far-part kernels: record preparation (points, quadrature nodes), the per-node
// gather / scatter of the standalone transforms, and the sum of f for the xi = 0 term.
// The stencil operations of the matvec are the tiled kernels of node.cu.
#include <cstring>
#include "far.cuh"
#include "sbd.h"
#include "window.cuh"

namespace sbd {

namespace {

template <typename T> __device__ __forceinline__ void atomic_add_cx(cx_t<T>* p, cx_t<T> v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

template <typename T, int PMAX>
__device__ __forceinline__ void weights(T frac, int P, const FarGeom& g, T* w) {
    const Window<T> win{g.kwin, static_cast<T>(g.beta_k), static_cast<T>(2.0 / P)};
#pragma unroll
    for (int a = 0; a < PMAX; ++a) {
        if (a < P) w[a] = win(static_cast<T>(a - P / 2 + 1) - frac);
    }
}

template <typename T>
__global__ void prepare_points_kernel(const double* __restrict__ z, long n, double cx, double cy, double h,
                                      int m, int P, PointRec<T>* __restrict__ out) {
    const long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const double ux = (z[2 * i] - cx) / h + 0.5 * m;
    const double uy = (z[2 * i + 1] - cy) / h + 0.5 * m;
    const double fx = floor(ux), fy = floor(uy);
    PointRec<T> r;   // (row, column) of the spreading grid = (y, x)
    r.cell = make_int2(static_cast<int>(fy) - P / 2 + 1, static_cast<int>(fx) - P / 2 + 1);
    r.frac = mk<T>(static_cast<T>(uy - fy), static_cast<T>(ux - fx));
    out[i] = r;
}

// Circle of record nu: the c with num[c] <= nu < num[c + 1] (binary search).
__device__ __forceinline__ int find_circle(const int* __restrict__ num, int n_circles, long nu) {
    int lo = 0, hi = n_circles;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (num[mid] <= nu) lo = mid; else hi = mid;
    }
    return lo;
}

// Angle index of record mm of its circle: m = mm for the full set; the half set takes
// m in [-floor(M/4), -floor(M/4) + M/2), the nodes with cos(2 pi m / M) >= 0 (xi_x >= 0),
// one of each antipodal pair.
__device__ __forceinline__ long angle_index(bool half, long mm, int M) { return half ? mm - M / 4 : mm; }

// Record index -> circle, canonical node index and xi (FP64, Eq. (defXimp)).
struct NodeId { int circle; long canon; long antipode; double2 xi; };
__device__ __forceinline__ NodeId node_id(const NodeFrame& fr, long rec) {
    NodeId id;
    const int* num = fr.hstart ? fr.hstart : fr.start;
    const int c = find_circle(num, fr.n_circles, rec);
    const int M = fr.M[c];
    const long m = angle_index(fr.hstart != nullptr, rec - num[c], M);
    double sn, cs;
    sincospi(2.0 * static_cast<double>(m) / M, &sn, &cs);
    id.circle = c;
    id.canon = fr.start[c] + ((m % M) + M) % M;
    id.antipode = fr.start[c] + (((m + M / 2) % M) + M) % M;
    id.xi = make_double2(fr.radius[c] * cs, fr.radius[c] * sn);
    return id;
}

template <typename T>
__global__ void prepare_nodes_kernel(const int* __restrict__ start, const int* __restrict__ hstart,
                                     const double* __restrict__ radius, const int* __restrict__ M, int n_circles,
                                     long n_rec, double deta, int nk, int P, const cx_t<T>* __restrict__ omega_c,
                                     SpreadDeconv sd, NodeRec<T>* __restrict__ out) {
    const long nu = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (nu >= n_rec) return;
    const int* num = hstart ? hstart : start;
    const int c = find_circle(num, n_circles, nu);
    const long mm = angle_index(hstart != nullptr, nu - num[c], M[c]);
    double sn, cs;
    sincospi(2.0 * static_cast<double>(mm) / M[c], &sn, &cs);   // xi_m = r (cos 2pi m/M, sin 2pi m/M)
    const double kx = radius[c] * cs / deta + 0.5 * nk;
    const double ky = radius[c] * sn / deta + 0.5 * nk;
    const double fx = floor(kx), fy = floor(ky);
    NodeRec<T> r;
    r.cell = make_int2(static_cast<int>(fx) - P / 2 + 1, static_cast<int>(fy) - P / 2 + 1);
    r.frac = mk<T>(static_cast<T>(kx - fx), static_cast<T>(ky - fy));
    // both transforms divide by the spreading window's transform at xi: the square of its factor
    const double sf = spread_deconv(sd, make_double2(radius[c] * cs, radius[c] * sn));
    r.omega = mk<T>(static_cast<T>(static_cast<double>(omega_c[c].x) * sf * sf),
                    static_cast<T>(static_cast<double>(omega_c[c].y) * sf * sf));
    out[nu] = r;
}

// Stencil at the record (mirror = false) or at its antipode: the window is even, so the
// antipode's stencil is the point reflection i -> nk - i of the record's, same weights.
template <typename T>
__device__ __forceinline__ cx_t<T> stencil_gather(const cx_t<T>* __restrict__ kin, int nk, int2 c0, const T* wx,
                                                  const T* wy, int P, bool mirror) {
    cx_t<T> acc = mk<T>(0, 0);
    for (int a = 0; a < P; ++a) {
        const long r = mirror ? nk - (c0.x + a) : c0.x + a;
        cx_t<T> s = mk<T>(0, 0);
        for (int b = 0; b < P; ++b) {
            const long col = mirror ? nk - (c0.y + b) : c0.y + b;
            s = cadd(s, cscale(kin[r * nk + col], wy[b]));
        }
        acc = cadd(acc, cscale(s, wx[a]));
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ void stencil_scatter(cx_t<T>* __restrict__ kout, int nk, int2 c0, const T* wx,
                                                const T* wy, int P, bool mirror, cx_t<T> v) {
    for (int a = 0; a < P; ++a) {
        const long r = mirror ? nk - (c0.x + a) : c0.x + a;
        const cx_t<T> va = cscale(v, wx[a]);
        for (int b = 0; b < P; ++b) {
            const long col = mirror ? nk - (c0.y + b) : c0.y + b;
            atomic_add_cx<T>(kout + r * nk + col, cscale(va, wy[b]));
        }
    }
}

// exp(-i c.xi) acc (sign -1) or exp(+i c.xi) v (sign +1), FP64
__device__ __forceinline__ double2 centre_phase(const NodeFrame& fr, double2 xi, double2 v, int sign) {
    double sn, co;
    sincos(fr.cx * xi.x + fr.cy * xi.y, &sn, &co);
    sn *= sign;
    return make_double2(v.x * co - v.y * sn, v.x * sn + v.y * co);
}

template <typename T, int PMAX>
__global__ void node_gather_kernel(const NodeRec<T>* __restrict__ nodes, long n_rec, const T* __restrict__ cs,
                                   FarGeom g, const cx_t<T>* __restrict__ kin, double2* __restrict__ out,
                                   NodeFrame fr) {
    const long nu = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (nu >= n_rec) return;
    const NodeRec<T> q = nodes[nu];
    T wx[PMAX], wy[PMAX];
    weights<T, PMAX>(q.frac.x, g.Pk, g, wx);
    weights<T, PMAX>(q.frac.y, g.Pk, g, wy);
    const NodeId id = node_id(fr, fr.perm ? fr.perm[nu] : nu);
    // the grids hold z - c: multiply by exp(-i c.xi) to return sum_l exp(-i z_l.xi) f_l
    const T sc = static_cast<T>(static_cast<double>(cs[id.circle]) * spread_deconv(fr.sd, id.xi));
    cx_t<T> acc = cscale(stencil_gather<T>(kin, g.nk, q.cell, wx, wy, g.Pk, false), sc);
    out[id.canon] = centre_phase(fr, id.xi, make_double2(acc.x, acc.y), -1);
    if (fr.hstart) {
        acc = cscale(stencil_gather<T>(kin, g.nk, q.cell, wx, wy, g.Pk, true), sc);
        out[id.antipode] = centre_phase(fr, make_double2(-id.xi.x, -id.xi.y), make_double2(acc.x, acc.y), -1);
    }
}

template <typename T, int PMAX>
__global__ void node_scatter_kernel(const NodeRec<T>* __restrict__ nodes, long n_rec, const T* __restrict__ cs,
                                    FarGeom g, const double2* __restrict__ in, cx_t<T>* __restrict__ kout,
                                    NodeFrame fr) {
    const long nu = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (nu >= n_rec) return;
    const NodeRec<T> q = nodes[nu];
    T wx[PMAX], wy[PMAX];
    weights<T, PMAX>(q.frac.x, g.Pk, g, wx);
    weights<T, PMAX>(q.frac.y, g.Pk, g, wy);
    const NodeId id = node_id(fr, fr.perm ? fr.perm[nu] : nu);
    const T sc = static_cast<T>(static_cast<double>(cs[id.circle]) * spread_deconv(fr.sd, id.xi));
    // q_l = sum_nu exp(i (z_l - c).xi) [exp(i c.xi) ghat_nu]
    double2 v = centre_phase(fr, id.xi, in[id.canon], +1);
    stencil_scatter<T>(kout, g.nk, q.cell, wx, wy, g.Pk, false,
                       cscale(mk<T>(static_cast<T>(v.x), static_cast<T>(v.y)), sc));
    if (fr.hstart) {
        v = centre_phase(fr, make_double2(-id.xi.x, -id.xi.y), in[id.antipode], +1);
        stencil_scatter<T>(kout, g.nk, q.cell, wx, wy, g.Pk, true,
                           cscale(mk<T>(static_cast<T>(v.x), static_cast<T>(v.y)), sc));
    }
}

__global__ void sum_kernel(const void* __restrict__ f, bool fc, long n, double2* __restrict__ sumf) {
    const int r = blockIdx.y;
    double sr = 0.0, si = 0.0;
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        if (fc) {
            const double2 v = static_cast<const double2*>(f)[r * n + i];
            sr += v.x;
            si += v.y;
        } else {
            sr += static_cast<const double*>(f)[r * n + i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sumf[r].x, sr);
        atomicAdd(&sumf[r].y, si);
    }
}

constexpr int kThreads = 256;
inline unsigned blocks_for(long n) { return static_cast<unsigned>((n + kThreads - 1) / kThreads); }

}  // namespace

template <typename T>
int far_prepare_points(const double* z, long n, double cx, double cy, double h, int m, int P,
                       PointRec<T>* out, cudaStream_t s) {
    if (n <= 0) return SBD_OK;
    prepare_points_kernel<T><<<blocks_for(n), kThreads, 0, s>>>(z, n, cx, cy, h, m, P, out);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int far_prepare_nodes(const int* circle_start, const int* half_start, const double* radius, const int* M,
                      int n_circles, long n_rec, double deta, int nk, int P, const cx_t<T>* omega_c,
                      const SpreadDeconv& sd, NodeRec<T>* out, cudaStream_t s) {
    if (n_rec <= 0) return SBD_OK;
    prepare_nodes_kernel<T><<<blocks_for(n_rec), kThreads, 0, s>>>(circle_start, half_start, radius, M, n_circles,
                                                                   n_rec, deta, nk, P, omega_c, sd, out);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T> constexpr int pmax() { return sizeof(T) == 8 ? 32 : 16; }

template <typename T>
int far_node_gather(const NodeRec<T>* nodes, long n_rec, const T* cscale_c, const FarGeom& g,
                    const cx_t<T>* kin, double2* out, const NodeFrame& fr, cudaStream_t s) {
    if (n_rec <= 0) return SBD_OK;
    node_gather_kernel<T, pmax<T>()><<<blocks_for(n_rec), kThreads, 0, s>>>(nodes, n_rec, cscale_c, g, kin, out,
                                                                            fr);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int far_node_scatter(const NodeRec<T>* nodes, long n_rec, const T* cscale_c, const FarGeom& g,
                     const double2* in, cx_t<T>* kout, const NodeFrame& fr, cudaStream_t s) {
    SBD_CUDA_TRY(cudaMemsetAsync(kout, 0, sizeof(cx_t<T>) * static_cast<size_t>(g.nk) * g.nk, s));
    if (n_rec <= 0) return SBD_OK;
    node_scatter_kernel<T, pmax<T>()><<<blocks_for(n_rec), kThreads, 0, s>>>(nodes, n_rec, cscale_c, g, in, kout,
                                                                             fr);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

int far_sum(const void* f, bool f_complex, long n, int nrhs, double2* sumf, cudaStream_t s) {
    SBD_CUDA_TRY(cudaMemsetAsync(sumf, 0, sizeof(double2) * nrhs, s));
    if (n <= 0) return SBD_OK;
    const unsigned nb = static_cast<unsigned>(std::min<long>((n + 255) / 256, 1024));
    sum_kernel<<<dim3(nb, nrhs), 256, 0, s>>>(f, f_complex, n, sumf);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

namespace {
// largest |component| of the records' weights; non-negative floats order as their bit patterns
template <typename T>
__global__ void weight_max_kernel(const NodeRec<T>* __restrict__ rec, long n, unsigned* __restrict__ out) {
    float m = 0.f;
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x) {
        const cx_t<T> w = rec[i].omega;
        m = fmaxf(m, fmaxf(fabsf(static_cast<float>(w.x)), fabsf(static_cast<float>(w.y))));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}
}  // namespace

template <typename T>
int far_weight_max(const NodeRec<T>* rec, long n, double* wmax, cudaStream_t s) {
    unsigned* d = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&d, sizeof(unsigned), s));
    unsigned h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && n > 0) {
        const unsigned nb = static_cast<unsigned>(std::min<long>((n + 255) / 256, 2048));
        weight_max_kernel<T><<<nb, 256, 0, s>>>(rec, n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SBD_ECUDA;
    }
    float f;
    std::memcpy(&f, &h, sizeof f);
    *wmax = f;
    return SBD_OK;
}

#define SBD_FAR_INST(T)                                                                                   \
    template int far_weight_max<T>(const NodeRec<T>*, long, double*, cudaStream_t);                       \
    template int far_prepare_points<T>(const double*, long, double, double, double, int, int, PointRec<T>*,  \
                                       cudaStream_t);                                                     \
    template int far_prepare_nodes<T>(const int*, const int*, const double*, const int*, int, long, double, \
                                      int, int, const cx_t<T>*, const SpreadDeconv&, NodeRec<T>*,         \
                                      cudaStream_t);                                                       \
    template int far_node_gather<T>(const NodeRec<T>*, long, const T*, const FarGeom&, const cx_t<T>*,    \
                                    double2*, const NodeFrame&, cudaStream_t);                            \
    template int far_node_scatter<T>(const NodeRec<T>*, long, const T*, const FarGeom&, const double2*,   \
                                     cx_t<T>*, const NodeFrame&, cudaStream_t);                           \

SBD_FAR_INST(float)
SBD_FAR_INST(double)

}  // namespace sbd
