// Uniform-grid multiplier variant of the far part: the fitted series G_fit (the SBD of
// Sec. 1 with each J0 term summed exactly, without the circle quadrature of Sec. 5), windowed
// and periodised, enters as Fourier coefficients on the frequency grid, so the node step
// becomes one multiplication per frequency (the fast-summation structure the paper cites
// as the alternative to its type-3 transforms).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "far.cuh"
#include "offline.h"

namespace sbd {

// c (device, nk x nk, rows = kx, allocated by the caller; T real for Laplace, cx_t<T> for
// Helmholtz) = the coefficients of H(y) = psi_w(y_x) psi_w(y_y) (G_fit(|y|) - w0) on the FFT
// period, times the square of the spreading window's deconvolution at both frequencies, so
// that K_out = c K_in between the forward and the inverse transform gives the far part
// (the xi = 0 term w0 sum f is added by the interpolation, as for the type-3 path).
// Built in FP64: a piecewise Chebyshev table of G_fit(r) - w0 from direct Bessel sums on the
// device, H on the n x n grid, a 2-D FFT, the window of |k| <= K.  Synchronous on s.
template <typename T>
int uniform_coefficients(const SbdFit& fit, const NufftParams& np, const SpreadDeconv& sd, bool complex_c, void* c,
                         cudaStream_t s);

// kout[r][j] = c[r][j] kin[r][j] for rows row0 <= r < nk and nrhs grids kbatch elements apart.
template <typename T>
int uniform_multiply(const cx_t<T>* kin, const void* c, bool complex_c, cx_t<T>* kout, int nk, int row0, int nrhs,
                     long kbatch, cudaStream_t s);

}  // namespace sbd
