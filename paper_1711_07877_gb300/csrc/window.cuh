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

template <typename T>
struct Window {
    int kind;
    T beta;
    T inv_half;   // 2 / P (ES only)
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
