// The O(P^3) step of the off-line fit on the GPU (Sec. 3.2: Cholesky of the Gram matrix A^P of
// Eq. LinearSystem, Sec. 6.1 complexity): the matrix is built on the device from O(P) vectors
// (closed form of Sec. 3.2, off-diagonal sign per reading R5) and factored in FP64 by a blocked
// right-looking Cholesky (diagonal block in shared memory, panel solve, trailing update of
// 64 x 64 tiles with 4 x 4 register blocks), then copied back in the host's packed layout.
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "offline.h"
#include "sbd.h"

namespace sbd {

namespace {

constexpr int kB = 64;          // block size
constexpr double kPiG = 3.14159265358979323846;

// A (row-major, leading dimension P, lower triangle): A_ij of the closed form.
__global__ void gram_kernel(const double* __restrict__ rho, const double* __restrict__ C,
                            const double* __restrict__ j0a, const double* __restrict__ j1a, double a, int P,
                            double* __restrict__ A) {
    const long idx = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (idx >= static_cast<long>(P) * P) return;
    const int i = static_cast<int>(idx / P), j = static_cast<int>(idx - static_cast<long>(i) * P);
    if (j > i) return;
    const double ri = rho[i];
    double v;
    if (j < i) {
        const double rj = rho[j];
        v = 2.0 * kPiG * C[i] * C[j] * ri * rj * a / (ri * ri - rj * rj) * (ri * j0a[i] * j1a[j] - rj * j0a[j] * j1a[i]);
    } else {
        const double x = ri * a;
        const double Fa = x * x * 0.5 * (j0a[i] * j0a[i] + j1a[i] * j1a[i]) - x * j0a[i] * j1a[i];
        v = 1.0 - 2.0 * kPiG * C[i] * C[i] * Fa;
    }
    A[idx] = v;
}

// Cholesky of the diagonal block [k0, k0 + kb)^2 in shared memory; the first non-positive pivot
// (global index) goes to *fail (which starts at P), and the block is then left as is.
__global__ void potrf_kernel(double* __restrict__ A, int P, int k0, int kb, int* __restrict__ fail) {
    __shared__ double s[kB][kB + 1];
    __shared__ int bad;
    const int t = threadIdx.x;
    for (int e = t; e < kb * kb; e += blockDim.x) {
        const int i = e / kb, j = e - i * kb;
        s[i][j] = j <= i ? A[static_cast<long>(k0 + i) * P + k0 + j] : 0.0;
    }
    if (t == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (t == 0 && !bad) {
            const double d = s[j][j];
            if (!(d > 0.0)) {
                bad = 1;
                atomicMin(fail, k0 + j);
            } else {
                s[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (!bad) {
            for (int i = j + 1 + t; i < kb; i += blockDim.x) s[i][j] /= s[j][j];
        }
        __syncthreads();
        if (!bad) {
            const int rows = kb - j - 1;
            for (int e = t; e < rows * rows; e += blockDim.x) {
                const int i = j + 1 + e / rows, c = j + 1 + e % rows;
                if (c <= i) s[i][c] -= s[i][j] * s[c][j];
            }
        }
        __syncthreads();
    }
    for (int e = t; e < kb * kb; e += blockDim.x) {
        const int i = e / kb, j = e - i * kb;
        if (j <= i) A[static_cast<long>(k0 + i) * P + k0 + j] = s[i][j];
    }
}

// Panel below the diagonal block: rows r >= k0 + kb, L21 = A21 L11^-T; one thread per row.
__global__ void trsm_kernel(double* __restrict__ A, int P, int k0, int kb) {
    __shared__ double L[kB][kB + 1];
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
        const int i = e / kb, j = e - i * kb;
        L[i][j] = j <= i ? A[static_cast<long>(k0 + i) * P + k0 + j] : 0.0;
    }
    __syncthreads();
    const long r = k0 + kb + blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (r >= P) return;
    double* row = A + r * P + k0;
    double x[kB];
#pragma unroll
    for (int c = 0; c < kB; ++c) x[c] = c < kb ? row[c] : 0.0;
    // column by column: x_c final, then removed from the later entries (all indices fixed at
    // compile time, so x stays in registers)
#pragma unroll
    for (int c = 0; c < kB; ++c) {
        if (c < kb) {
            x[c] /= L[c][c];
#pragma unroll
            for (int t = c + 1; t < kB; ++t) x[t] -= x[c] * L[t][c];
        }
    }
#pragma unroll
    for (int c = 0; c < kB; ++c)
        if (c < kb) row[c] = x[c];
}

// Trailing update A22 -= L21 L21^T on the lower tiles: CTA = one 64 x 64 tile (bi >= bj) of the
// rows / columns past k0 + kb; 256 threads, 4 x 4 outputs each; K = kb in steps of 16.
__global__ void __launch_bounds__(256) syrk_kernel(double* __restrict__ A, int P, int k0, int kb) {
    __shared__ double Ai[16][kB + 1], Aj[16][kB + 1];
    const int base = k0 + kb;
    // tile pair from the linear lower-triangle index
    const long q = blockIdx.x;
    const int bi = static_cast<int>((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
    int bI = bi;
    while (static_cast<long>(bI + 1) * (bI + 2) / 2 <= q) ++bI;
    while (static_cast<long>(bI) * (bI + 1) / 2 > q) --bI;
    const int bJ = static_cast<int>(q - static_cast<long>(bI) * (bI + 1) / 2);
    const int r0 = base + bI * kB, c0 = base + bJ * kB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4 x 4 outputs each
    double acc[4][4] = {};
    for (int k = 0; k < kb; k += 16) {
        const int kk = min(16, kb - k);
        for (int e = threadIdx.x; e < 16 * kB; e += 256) {
            const int kc = e / kB, rr = e - kc * kB;
            const int gi = r0 + rr, gj = c0 + rr;
            Ai[kc][rr] = (kc < kk && gi < P) ? A[static_cast<long>(gi) * P + k0 + k + kc] : 0.0;
            Aj[kc][rr] = (kc < kk && gj < P) ? A[static_cast<long>(gj) * P + k0 + k + kc] : 0.0;
        }
        __syncthreads();
        for (int kc = 0; kc < kk; ++kc) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = Ai[kc][ty * 4 + u];
                b[u] = Aj[kc][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gi = r0 + ty * 4 + u, gj = c0 + tx * 4 + v;
            if (gi < P && gj < P && gj <= gi) A[static_cast<long>(gi) * P + gj] -= acc[u][v];
        }
}

}  // namespace

bool fit_gpu_available() {
    int n = 0;
    const bool ok = cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
    cudaGetLastError();
    return ok;
}

int gram_cholesky_gpu(const std::vector<double>& rho, const std::vector<double>& C, const std::vector<double>& j0a,
                      const std::vector<double>& j1a, double a, int P, std::vector<double>& packed, int* Pok,
                      std::string& err) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        err = "gram_cholesky_gpu: no stream";
        return SBD_ECUDA;
    }
    double *A = nullptr, *v = nullptr;
    int* fail = nullptr;
    int rc = SBD_OK;
    auto done = [&](int r) {
        if (A) cudaFreeAsync(A, s);
        if (v) cudaFreeAsync(v, s);
        if (fail) cudaFreeAsync(fail, s);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        cudaGetLastError();
        return r;
    };
    if (cudaMallocAsync(&A, sizeof(double) * static_cast<size_t>(P) * P, s) != cudaSuccess ||
        cudaMallocAsync(&v, sizeof(double) * 4 * P, s) != cudaSuccess || cudaMallocAsync(&fail, sizeof(int), s) !=
                                                                                 cudaSuccess) {
        err = "gram_cholesky_gpu: device allocation failed";
        return done(SBD_ENOMEM);
    }
    std::vector<double> h(4 * static_cast<size_t>(P));
    for (int p = 0; p < P; ++p) {
        h[p] = rho[p];
        h[P + p] = C[p];
        h[2 * P + p] = j0a[p];
        h[3 * P + p] = j1a[p];
    }
    cudaMemcpyAsync(v, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(fail, &P, sizeof(int), cudaMemcpyHostToDevice, s);
    const long cells = static_cast<long>(P) * P;
    gram_kernel<<<static_cast<unsigned>((cells + 255) / 256), 256, 0, s>>>(v, v + P, v + 2 * P, v + 3 * P, a, P, A);
    int failed = P;
    for (int k0 = 0; k0 < P && failed == P; k0 += kB) {
        const int kb = std::min(kB, P - k0);
        potrf_kernel<<<1, 256, 0, s>>>(A, P, k0, kb, fail);
        cudaMemcpyAsync(&failed, fail, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            err = std::string("gram_cholesky_gpu: ") + cudaGetErrorString(cudaGetLastError());
            return done(SBD_ECUDA);
        }
        if (failed < P) break;
        const int rest = P - k0 - kb;
        if (rest <= 0) break;
        trsm_kernel<<<static_cast<unsigned>((rest + 127) / 128), 128, 0, s>>>(A, P, k0, kb);
        const long nt = (rest + kB - 1) / kB;
        syrk_kernel<<<static_cast<unsigned>(nt * (nt + 1) / 2), 256, 0, s>>>(A, P, k0, kb);
    }
    if (cudaGetLastError() != cudaSuccess) {
        err = "gram_cholesky_gpu: kernel launch failed";
        return done(SBD_ECUDA);
    }
    // copy back row by row into the packed lower layout (row i: entries 0..i)
    std::vector<double> full(static_cast<size_t>(P) * P);
    if (cudaMemcpyAsync(full.data(), A, sizeof(double) * full.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        err = "gram_cholesky_gpu: copy failed";
        return done(SBD_ECUDA);
    }
    packed.assign(static_cast<size_t>(P) * (P + 1) / 2, 0.0);
    for (int i = 0; i < P; ++i)
        std::copy(full.begin() + static_cast<long>(i) * P, full.begin() + static_cast<long>(i) * P + i + 1,
                  packed.begin() + static_cast<long>(i) * (i + 1) / 2);
    *Pok = failed;
    return done(rc);
}

}  // namespace sbd
