// Far part of the on-line SBD (Sec. 1 steps (i)-(iii), Eq. far convolution) by a
// type-3 transform: points spread with a separable window (ES or Gaussian) onto a
// grid oversampled 1.5- or 2-fold, a two-fold zero-padded FFT, and a node window (ES or
// Gaussian).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace sbd {

// Geometry of one transform, all in cells of the respective grid.
struct FarGeom {
    int Ps;           // spreading stencil width (cells per dimension), even
    int Pk;           // node stencil width, even
    int m;            // spreading grid side
    int nk;           // frequency grid side
    int kwin;         // node window (WindowKind)
    double beta_s;    // spreading window parameter
    double beta_k;    // node window parameter
    int swin;         // spreading window (WindowKind)
    const float4* kpoly;   // FP32 plans: polynomial tables of the node and spreading windows
    const float4* spoly;   // (window.cuh), or null where the window is evaluated directly
    const double* kpoly64; // FP64 plans: the same for the FP64 kernels
    const double* spoly64;
    const void* node_bins; // binned node kernels: the per-tile bin table (node.cuh BinTable), or null,
    const int* node_order; // the tiles holding records, most records first,
    int n_node_tiles;      // and their number
};

// Deconvolution of the ES spreading window at a node: psi(k) = 1 / phi_hat_s(k) with
// k = xi h, log psi as a Chebyshev series in 2 (k / kmax)^2 - 1; the node xi takes the
// factor psi(xi_x h) psi(xi_y h).  coef null: Gaussian spreading, whose factor
// exp(tau |xi|^2) is radial and sits in the circle's weight.  FP64.
struct SpreadDeconv {
    const double* coef;
    int n;              // coefficients
    double inv_kmax2;   // 1 / kmax^2
    double h;           // spreading-grid spacing
};
__device__ __forceinline__ double spread_psi(const SpreadDeconv& d, double k) {
    const double x = 2.0 * k * k * d.inv_kmax2 - 1.0;
    double b1 = 0.0, b2 = 0.0;
    for (int i = d.n - 1; i >= 1; --i) {
        const double t = 2.0 * x * b1 - b2 + d.coef[i];
        b2 = b1;
        b1 = t;
    }
    return exp(x * b1 - b2 + d.coef[0]);
}
__device__ __forceinline__ double spread_deconv(const SpreadDeconv& d, double2 xi) {
    if (!d.coef) return 1.0;
    return spread_psi(d, xi.x * d.h) * spread_psi(d, xi.y * d.h);
}

// Point i: spreading stencil starts at (row, column) = cell of the spreading grid, whose
// rows are y; frac = position - floor(position) in the same (row, column) order.
template <typename T> struct PointRec { int2 cell; cx_t<T> frac; };
// Node: stencil start cell in the frequency grid, fraction, and its weight omega'_nu
// (omega_hat_p of its circle times the transform's scale factors at xi_nu), so the node
// step needs no second lookup.
template <typename T> struct NodeRec { int2 cell; cx_t<T> frac; cx_t<T> omega; };

// Plan-time preparation (FP64 arithmetic).
template <typename T>
int far_prepare_points(const double* z, long n, double cx, double cy, double h, int m, int P,
                       PointRec<T>* out, cudaStream_t s);
// Records of the quadrature nodes.  half_start null: every node, n_rec = N_xi, record
// numbering = canonical numbering (circle by circle, angle index m).  half_start
// non-null (prefix sums of M_p / 2; every M_p is even): per circle only the M_p / 2
// nodes with xi_x >= 0 (angle index m in [-floor(M_p/4), -floor(M_p/4) + M_p/2)), whose
// antipodes -xi the Hermitian-symmetric node step of a real-valued transform supplies
// by symmetry.
template <typename T>
int far_prepare_nodes(const int* circle_start, const int* half_start, const double* radius, const int* M,
                      int n_circles, long n_rec, double deta, int nk, int P, const cx_t<T>* omega_c,
                      const SpreadDeconv& sd, NodeRec<T>* out, cudaStream_t s);
// *wmax (host) = max over the records of max(|Re omega'|, |Im omega'|) (synchronises s).
template <typename T>
int far_weight_max(const NodeRec<T>* rec, long n, double* wmax, cudaStream_t s);

// Circle tables and the centre c of the point set, to place the canonical nodes in
// absolute coordinates (the grids hold z - c).
struct NodeFrame {
    const int* start;
    const double* radius;
    const int* M;
    int n_circles;
    double cx, cy;
    const int* perm;   // sorted record -> record numbering (null: records in that order)
    const int* hstart; // non-null: records are the half set (see far_prepare_nodes); the
                       // gather / scatter also serve each record's antipode
    int nk;            // frequency-grid side (mirror of cell i is nk - i)
    SpreadDeconv sd;   // per-node factor of the spreading window (coef null: none)
};
// Gather only: out[nu] = exp(-i c.xi_nu) c_nu sum_stencil w K  (complex128), c_nu = circle
// scale times the node's spreading deconvolution,
// for every node nu (canonical numbering; n_rec records).
template <typename T>
int far_node_gather(const NodeRec<T>* nodes, long n_rec, const T* cscale, const FarGeom& g,
                    const cx_t<T>* kin, double2* out, const NodeFrame& fr, cudaStream_t s);
// Scatter only: kout (zeroed here) += c_nu exp(i c.xi_nu) in[nu] w.
template <typename T>
int far_node_scatter(const NodeRec<T>* nodes, long n_rec, const T* cscale, const FarGeom& g,
                     const double2* in, cx_t<T>* kout, const NodeFrame& fr, cudaStream_t s);
// sumf[r] = sum_l f[r][l] (FP64).
int far_sum(const void* f, bool f_complex, long n, int nrhs, double2* sumf, cudaStream_t s);

}  // namespace sbd
