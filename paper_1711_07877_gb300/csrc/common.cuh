// Shared device helpers: complex arithmetic over float / double, error plumbing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <shared_mutex>
#include <string>

namespace sbd {

template <typename T> struct Cx;
template <> struct Cx<float>  { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx_t<T> mk(T re, T im) {
    cx_t<T> v; v.x = re; v.y = im; return v;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b) when conj_b, else a * b
template <typename C> __host__ __device__ __forceinline__ C cmul_dir(C a, C b, bool conj_b) {
    if (conj_b) b.y = -b.y;
    return cmul(a, b);
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }

// Thread-local detail text of the last error (sbd_last_error_message).
void set_error(const std::string& msg);

// Raises (never lowers) a kernel's dynamic shared-memory limit on the current device to
// at least `bytes`, under a process-wide lock, so that concurrent host threads launching
// the same kernel with different sizes never shrink each other's limit.
int raise_smem_limit_fn(const void* func, size_t bytes);

// Process-wide lock between CUDA-graph capture (held shared while a thread captures) and
// calls that synchronise with every stream of the device or may (device synchronise,
// cudaFree, cudaMalloc, synchronous copies; held exclusive): those calls would otherwise
// invalidate a capture running in another thread.
std::shared_mutex& capture_mutex();
template <typename K>
inline int raise_smem_limit(K* kernel, size_t bytes) {
    return raise_smem_limit_fn(reinterpret_cast<const void*>(kernel), bytes);
}

}  // namespace sbd

#define SBD_CUDA_TRY(call)                                                        \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            ::sbd::set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? SBD_ENOMEM : SBD_ECUDA;      \
        }                                                                         \
    } while (0)

#define SBD_TRY(expr)             \
    do {                          \
        const int rc_ = (expr);   \
        if (rc_ != 0) return rc_; \
    } while (0)

#define SBD_LAUNCH_CHECK()                                                        \
    do {                                                                          \
        cudaError_t e_ = cudaGetLastError();                                      \
        if (e_ != cudaSuccess) {                                                  \
            ::sbd::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_)); \
            return SBD_ECUDA;                                                     \
        }                                                                         \
    } while (0)
