// Hand-written FFT for sm_103a: batched 1-D complex transforms of contiguous rows,
// each row held in shared memory for all its radix stages, plus a tiled transpose.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace sbd {

constexpr int kFftMaxStages = 32;

struct FftPlan1D {
    int n = 0;
    int nstages = 0;
    int radix[kFftMaxStages];
};

// Radix schedule for n = 2^a 3^b 5^c (prime-power radices up to 16, and 15, for FP32; up to 9
// for FP64; odd ones first); false when n has another factor.
bool fft_make_plan(int n, FftPlan1D& p, bool fp64);

// Largest row length a single CTA can hold in shared memory for this element type.
int fft_max_row(bool fp64);
// Largest transform length fft_rows accepts (two phases of fft_max_row).
int fft_max_length(bool fp64);

// One batched row pass:
//   out[r][e] = post_row[r] post_elem[e] *
//               sum_t (pre_row[r] pre_elem[t] in[r][t]) exp(sign 2 pi i (t + in_shift)(e + out_shift) / n)
// for e < out_len, t < in_len (input element t sits at FFT position (t + in_shift) mod n,
// output element e is FFT position (e + out_shift) mod n).  Scale pointers may be null.
//
// Hermitian fold (herm_n > 0): in points at row herm_row0 of a herm_n x herm_n grid S
// (in_len == herm_n) and row r of this call is read as S[a][t] + conj(S[herm_n - a]
// [herm_n - t]) with a = herm_row0 + r (the second term only for a, t >= 1): the
// transform of S(eta) + conj(S(-eta)) for a centred grid.  herm_lo: rows of S below it are
// zero, so rows a whose mirror herm_n - a lies below it are read plainly.
//
// io modes for real data (two real rows per transform, "packed pair" rows
// z = x_{2j} + i x_{2j+1}):
//   kIoPairFwd  input row j is a packed pair (re scaled by pre_row[2j], im by
//               pre_row[2j+1]); the outputs are the two transforms X_{2j}, X_{2j+1}
//               (each Hermitian), written to output rows 2j and 2j + 1.  rows = pairs.
//   kIoPairInv  input rows 2j, 2j + 1 hold frequencies 0..in_len-1 of two Hermitian
//               spectra (the negative ones are their conjugates; FFT position idx is
//               frequency idx, or idx - n past n / 2); the output row j is the packed
//               pair of the two (real) transforms, re scaled by post_row[2j], im by
//               post_row[2j+1].  in_shift is unused.  rows = pairs.
enum { kIoPlain = 0, kIoPairFwd = 1, kIoPairInv = 2 };
template <typename T>
int fft_rows(const cx_t<T>* in, long in_stride, int in_len, int in_shift,
             cx_t<T>* out, long out_stride, int out_len, int out_shift,
             int rows, int n, int sign,
             const T* pre_elem, const T* pre_row, const T* post_elem, const T* post_row,
             cudaStream_t stream, int herm_n = 0, int herm_row0 = 0, int io = kIoPlain, int split = 0,
             int nb = 1, long in_batch = 0, long out_batch = 0, long out_es = 1, int herm_lo = 0);
// split = 2: run every even length as two half-length phases (two 512-thread CTAs per row,
// two rows' worth of CTAs per SM) even when the whole row would fit; 0: only when it must.
// nb > 1: the same pass over nb grids (right-hand sides) in one launch, grid b's input and
// output (and Hermitian fold base) offset by b in_batch / b out_batch elements; the row
// scale vectors are shared.
// out_es: element e of output row r goes to out[r * out_stride + e * out_es]; out_stride = 1
// with out_es = the row count writes the pass transposed (the next pass's rows), in place of a
// separate transpose.

// Natural-order row transforms of length n (input and output windows start at 0) with
// caller-provided tables: tw[t] = exp(-2 pi i t / n), perm = the digit reversal of
// fft_make_plan(n).  Allocates nothing.
template <typename T>
int fft_rows_tables(const cx_t<T>* in, long in_stride, int in_len, cx_t<T>* out, long out_stride, int out_len,
                    int rows, int n, int sign, const cx_t<T>* tw, const int* perm, cudaStream_t stream);

// out[c][r] = in[r][c] for a rows x cols matrix (row strides in elements), batched over nb
// matrices spaced in_batch / out_batch elements apart.
template <typename T>
int transpose(const cx_t<T>* in, long in_stride, long in_batch, cx_t<T>* out, long out_stride,
              long out_batch, int rows, int cols, int nb, cudaStream_t stream);

}  // namespace sbd
