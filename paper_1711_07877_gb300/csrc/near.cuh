// Near field: fixed-radius neighbour search (Sec. 1 / Sec. 6.1) into CSR, the values
// of the close-correction matrix D (Eq. defD) in FP64 (optionally stored as FP32), and
// the SpMV q += D f.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace sbd {

// Device-side description of D(y) = T1(t) log(t)/2 + T2(t) - sum_{c small} w_c sum_m e^{i y.xi_m},
// t = |y|^2 (tables: piecewise Chebyshev in t, complex, [pieces][deg][2]).
struct NearDev {
    int pieces, deg;
    double tmax;              // table range in r^2, or in r when in_r
    int in_r;
    const double* T1;
    const double* T2;
    int n_small;              // circles evaluated exactly
    const double* small_xi;   // (sum over small circles of M) x 2 node coordinates
    const int* small_start;   // n_small + 1 offsets into small_xi
    const double* small_w;    // n_small complex weights (re, im)
    double self_re, self_im;  // D_kk
};

// Bounding box (xmin, ymin, xmax, ymax) and max squared distance to a centre.
int points_bbox(const double* z, long n, double* out4_host, cudaStream_t s);
int points_max_dist2(const double* z, long n, double cx, double cy, double* out_host, cudaStream_t s);

// Build CSR of D.  Square (zq null): rows and columns are the n points z, the diagonal
// first in every row.  Otherwise rows are the nq targets zq and columns the n sources z
// (every source within delta_min of the target, a coincident one with the self value).
// The box (bx0, by0)-(bx1, by1) must hold both sets.  Allocates rowptr/col/val
// stream-ordered on s (cudaMallocAsync; free them with cudaFreeAsync).
//   complex_vals: values are complex128 (Helmholtz) or float64 (Laplace).
int near_build(const double* z, long n, double delta_min, double bx0, double by0, double bx1, double by1,
               const NearDev& tab, bool complex_vals, long long** rowptr, int** col, void** val,
               long long* nnz, long long* n_coincident, cudaStream_t s, const double* zq = nullptr, long nq = 0);

// q[r] (+)= D f[r] for r < nrhs (q accumulated when accumulate, else overwritten).
int near_spmv(const long long* rowptr, const int* col, const void* val, bool complex_vals, long n, int nrhs,
              const void* f, void* q, bool accumulate, cudaStream_t s);

// The near field in the internal point order (the spreading records' tile order, which
// keeps the columns of a row close together): fp[i * nrhs + r] = f[r * n + perm[i]]
// (near_gather), qp = D fp with D over internal indices and interleaved right-hand
// sides (near_spmv_internal), q[r * n + perm[i]] = qp[i * nrhs + r] (near_scatter).
// f and qp are float64 (real) or complex128 (cplx).  f32: D's values (near_values_to_f32)
// and fp are float32 / complex64, products and per-thread partial sums FP32, the partial
// sums of a row combined in FP64; qp stays float64 / complex128.
int near_gather(const void* f, bool cplx, long n, int nrhs, const int* perm, void* fp, cudaStream_t s,
                bool f32 = false);
int near_spmv_internal(const long long* rowptr, const int* col, const void* val, bool complex_vals, long n,
                       int nrhs, const void* fp, void* qp, cudaStream_t s, bool f32 = false);
// Replaces the FP64 values *val (nnz entries, complex when cplx) by FP32 ones (stream-ordered).
int near_values_to_f32(void** val, long long nnz, bool cplx, cudaStream_t s);
int near_scatter(const void* qp, bool cplx, long n, int nrhs, const int* perm, void* q, cudaStream_t s);

// Exclusive scan of n 64-bit counts in place; total returned in *total (host), synchronising s.
int scan_exclusive_i64(long long* data, long n, long long* total, cudaStream_t s);

}  // namespace sbd
