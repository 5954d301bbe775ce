// Separable stencil windows of the type-3 transform.
//   Gaussian        w(d) = exp(-beta d^2)
//   ES ("exponential of semicircle", Barnett-Magland-af Klinteberg 2019)
//                   w(d) = exp(beta (sqrt(1 - (d / (P/2))^2) - 1)), |d| < P/2
// d is the signed distance in cells between a stencil cell and the record position.
#pragma once
#include <cuda_runtime.h>

namespace sbd {

enum WindowKind { kWinGauss = 0, kWinES = 1 };

template <typename T> __device__ __forceinline__ T wexp(T x);
// FP32 form: expf (the fast __expf's error grows with |x|, ~1e-6 relative at the window's
// arguments of -10 to -20, and measurably raised the matvec's error); FP64 exp.
template <> __device__ __forceinline__ float wexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double wexp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T wsqrt(T x);
template <> __device__ __forceinline__ float wsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double wsqrt<double>(double x) { return sqrt(x); }

// Polynomial form of a window for the FP32 stencil kernels (stencils of at most 16 cells):
// the weight of stencil offset j (0 <= j < P) at fraction f in [0, 1), w(j - P/2 + 1 - f), is a
// polynomial of degree kWinPolyDeg in s = 2 f - 1 (Chebyshev interpolation of the window in
// FP64 on the host, converted to powers of s).  Layout: coefficient k (highest power first) of
// offset j is component k % 4 of entry (k / 4) * 16 + j, so the three float4 of one offset sit
// 16 entries apart and a warp's reads of one group touch consecutive 16-byte slots; offsets
// j >= P hold zeros.
constexpr int kWinPolyDeg = 11;
constexpr int kWinPolyOffsets = 16;
constexpr int kWinPolyQuads = (kWinPolyDeg + 4) / 4;              // float4 per offset
constexpr int kWinPolyEntries = kWinPolyQuads * kWinPolyOffsets;  // float4 per table

__device__ __forceinline__ float poly_quad(float acc, const float4 c, float s) {
    acc = fmaf(acc, s, c.x);
    acc = fmaf(acc, s, c.y);
    acc = fmaf(acc, s, c.z);
    return fmaf(acc, s, c.w);
}

// Weights of one offset at the fractions fx, fy (Horner in s, the two chains interleaved).
__device__ __forceinline__ void poly_weights(const float4 c0, const float4 c1, const float4 c2, float fx, float fy,
                                             float& wx, float& wy) {
    static_assert(kWinPolyQuads == 3, "three coefficient groups");
    const float sx = fmaf(2.f, fx, -1.f), sy = fmaf(2.f, fy, -1.f);
    float ax = fmaf(fmaf(fmaf(c0.x, sx, c0.y), sx, c0.z), sx, c0.w);
    float ay = fmaf(fmaf(fmaf(c0.x, sy, c0.y), sy, c0.z), sy, c0.w);
    ax = poly_quad(ax, c1, sx);
    ay = poly_quad(ay, c1, sy);
    wx = poly_quad(ax, c2, sx);
    wy = poly_quad(ay, c2, sy);
}

// The FP64 kernels' table: degree kWinPolyDeg64 in the same s, coefficient k (highest power
// first) of offset j at entry k * kWinPolyOffsets + j (a warp's reads of one coefficient touch
// consecutive doubles).
constexpr int kWinPolyDeg64 = 19;
constexpr int kWinPolyEntries64 = (kWinPolyDeg64 + 1) * kWinPolyOffsets;

// Weights of offset j at the fractions fx, fy from the FP64 table (Horner, two chains).
__device__ __forceinline__ void poly_weights64(const double* __restrict__ c, int j, double fx, double fy,
                                               double& wx, double& wy) {
    const double sx = fma(2.0, fx, -1.0), sy = fma(2.0, fy, -1.0);
    double ax = __ldg(c + j), ay = ax;
#pragma unroll
    for (int k = 1; k <= kWinPolyDeg64; ++k) {
        const double ck = __ldg(c + k * kWinPolyOffsets + j);
        ax = fma(ax, sx, ck);
        ay = fma(ay, sy, ck);
    }
    wx = ax;
    wy = ay;
}

template <typename T>
struct Window {
    int kind;
    T beta;
    T inv_half;                     // 2 / P (ES only)
    const float4* poly = nullptr;   // FP32 kernels: the polynomial table (device), or null
    const double* poly64 = nullptr; // FP64 kernels: the polynomial table (device), or null
    __device__ __forceinline__ T operator()(T d) const {
        if (kind == kWinGauss) return wexp<T>(-beta * d * d);
        // sqrt(1 - z^2) - 1 = -z^2 / (1 + sqrt(1 - z^2)): no cancellation near the centre,
        // where the weights are largest (the difference form loses ~1e-5 relative there in FP32)
        const T z = d * inv_half;
        const T z2 = z * z;
        const T r = static_cast<T>(1) - z2;
        return r > static_cast<T>(0) ? wexp<T>(-beta * z2 / (static_cast<T>(1) + wsqrt<T>(r))) : static_cast<T>(0);
    }
};

}  // namespace sbd
