// Far-part kernels: record preparation (points, quadrature nodes), the per-node
// gather / scatter of the standalone transforms, and the sum of f for the xi = 0 term.
// The stencil operations of the matvec are the tiled kernels of node.cu.
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

// xi of node nu (FP64): circle by binary search in the prefix offsets, then Eq. (defXimp).
__device__ __forceinline__ double2 node_xi(const int* __restrict__ start, const double* __restrict__ radius,
                                           const int* __restrict__ M, int n_circles, long nu, int* circle) {
    int lo = 0, hi = n_circles;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (start[mid] <= nu) lo = mid; else hi = mid;
    }
    double sn, cs;
    sincospi(2.0 * static_cast<double>(nu - start[lo]) / M[lo], &sn, &cs);
    *circle = lo;
    return make_double2(radius[lo] * cs, radius[lo] * sn);
}

template <typename T>
__global__ void prepare_nodes_kernel(const int* __restrict__ start, const double* __restrict__ radius,
                                     const int* __restrict__ M, int n_circles, long n_xi, double deta,
                                     int nk, int P, const cx_t<T>* __restrict__ omega_c,
                                     NodeRec<T>* __restrict__ out) {
    const long nu = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (nu >= n_xi) return;
    int lo = 0, hi = n_circles;   // start[lo] <= nu < start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (start[mid] <= nu) lo = mid; else hi = mid;
    }
    const int c = lo;
    const long mm = nu - start[c];
    double sn, cs;
    sincospi(2.0 * static_cast<double>(mm) / M[c], &sn, &cs);   // xi_m = r (cos 2pi m/M, sin 2pi m/M)
    const double kx = radius[c] * cs / deta + 0.5 * nk;
    const double ky = radius[c] * sn / deta + 0.5 * nk;
    const double fx = floor(kx), fy = floor(ky);
    NodeRec<T> r;
    r.cell = make_int2(static_cast<int>(fx) - P / 2 + 1, static_cast<int>(fy) - P / 2 + 1);
    r.frac = mk<T>(static_cast<T>(kx - fx), static_cast<T>(ky - fy));
    r.omega = omega_c[c];
    out[nu] = r;
}

template <typename T, int PMAX>
__global__ void node_gather_kernel(const NodeRec<T>* __restrict__ nodes, long n_xi, const T* __restrict__ cs,
                                   FarGeom g, const cx_t<T>* __restrict__ kin, double2* __restrict__ out,
                                   NodeFrame fr) {
    // records may be in tile order: fr.perm maps a record to its canonical node index
    const long nu = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (nu >= n_xi) return;
    const NodeRec<T> q = nodes[nu];
    T wx[PMAX], wy[PMAX];
    weights<T, PMAX>(q.frac.x, g.Pk, g, wx);
    weights<T, PMAX>(q.frac.y, g.Pk, g, wy);
    cx_t<T> acc = mk<T>(0, 0);
    for (int a = 0; a < g.Pk; ++a) {
        const cx_t<T>* row = kin + static_cast<long>(q.cell.x + a) * g.nk + q.cell.y;
        cx_t<T> s = mk<T>(0, 0);
        for (int b = 0; b < g.Pk; ++b) s = cadd(s, cscale(row[b], wy[b]));
        acc = cadd(acc, cscale(s, wx[a]));
    }
    // the grids hold z - c: multiply by exp(-i c.xi) to return sum_l exp(-i z_l.xi) f_l
    const long canon = fr.perm ? fr.perm[nu] : nu;
    int circle;
    const double2 xi = node_xi(fr.start, fr.radius, fr.M, fr.n_circles, canon, &circle);
    acc = cscale(acc, cs[circle]);
    double sn, co;
    sincos(fr.cx * xi.x + fr.cy * xi.y, &sn, &co);
    const double ar = acc.x, ai = acc.y;
    out[canon] = make_double2(ar * co + ai * sn, ai * co - ar * sn);
}

template <typename T, int PMAX>
__global__ void node_scatter_kernel(const NodeRec<T>* __restrict__ nodes, long n_xi, const T* __restrict__ cs,
                                    FarGeom g, const double2* __restrict__ in, cx_t<T>* __restrict__ kout,
                                    NodeFrame fr) {
    const long nu = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (nu >= n_xi) return;
    const NodeRec<T> q = nodes[nu];
    T wx[PMAX], wy[PMAX];
    weights<T, PMAX>(q.frac.x, g.Pk, g, wx);
    weights<T, PMAX>(q.frac.y, g.Pk, g, wy);
    const long canon = fr.perm ? fr.perm[nu] : nu;
    double2 v = in[canon];
    // q_l = sum_nu exp(i (z_l - c).xi) [exp(i c.xi) ghat_nu]
    int circle;
    const double2 xi = node_xi(fr.start, fr.radius, fr.M, fr.n_circles, canon, &circle);
    double sn, co;
    sincos(fr.cx * xi.x + fr.cy * xi.y, &sn, &co);
    v = make_double2(v.x * co - v.y * sn, v.x * sn + v.y * co);
    const cx_t<T> acc = cscale(mk<T>(static_cast<T>(v.x), static_cast<T>(v.y)), cs[circle]);
    for (int a = 0; a < g.Pk; ++a) {
        const cx_t<T> va = cscale(acc, wx[a]);
        cx_t<T>* row = kout + static_cast<long>(q.cell.x + a) * g.nk + q.cell.y;
        for (int b = 0; b < g.Pk; ++b) atomic_add_cx<T>(row + b, cscale(va, wy[b]));
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
int far_prepare_nodes(const int* circle_start, const double* radius, const int* M, int n_circles,
                      long n_xi, double deta, int nk, int P, const cx_t<T>* omega_c, NodeRec<T>* out,
                      cudaStream_t s) {
    if (n_xi <= 0) return SBD_OK;
    prepare_nodes_kernel<T><<<blocks_for(n_xi), kThreads, 0, s>>>(circle_start, radius, M, n_circles, n_xi,
                                                                   deta, nk, P, omega_c, out);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T> constexpr int pmax() { return sizeof(T) == 8 ? 32 : 16; }

template <typename T>
int far_node_gather(const NodeRec<T>* nodes, long n_xi, const T* cscale_c, const FarGeom& g,
                    const cx_t<T>* kin, double2* out, const NodeFrame& fr, cudaStream_t s) {
    if (n_xi <= 0) return SBD_OK;
    node_gather_kernel<T, pmax<T>()><<<blocks_for(n_xi), kThreads, 0, s>>>(nodes, n_xi, cscale_c, g, kin, out, fr);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int far_node_scatter(const NodeRec<T>* nodes, long n_xi, const T* cscale_c, const FarGeom& g,
                     const double2* in, cx_t<T>* kout, const NodeFrame& fr, cudaStream_t s) {
    SBD_CUDA_TRY(cudaMemsetAsync(kout, 0, sizeof(cx_t<T>) * static_cast<size_t>(g.nk) * g.nk, s));
    if (n_xi <= 0) return SBD_OK;
    node_scatter_kernel<T, pmax<T>()><<<blocks_for(n_xi), kThreads, 0, s>>>(nodes, n_xi, cscale_c, g, in, kout, fr);
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

#define SBD_FAR_INST(T)                                                                                   \
    template int far_prepare_points<T>(const double*, long, double, double, double, int, int, PointRec<T>*,  \
                                       cudaStream_t);                                                     \
    template int far_prepare_nodes<T>(const int*, const double*, const int*, int, long, double, int, int, \
                                      const cx_t<T>*, NodeRec<T>*, cudaStream_t);                         \
    template int far_node_gather<T>(const NodeRec<T>*, long, const T*, const FarGeom&, const cx_t<T>*,    \
                                    double2*, const NodeFrame&, cudaStream_t);                            \
    template int far_node_scatter<T>(const NodeRec<T>*, long, const T*, const FarGeom&, const double2*,   \
                                     cx_t<T>*, const NodeFrame&, cudaStream_t);                           \

SBD_FAR_INST(float)
SBD_FAR_INST(double)

}  // namespace sbd
