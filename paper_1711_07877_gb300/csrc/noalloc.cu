// sbd_fft2_noalloc: the 2-D FFT of sbd_fft2 without any device allocation.
//
// Its temporary grid and its twiddle and digit-reversal tables live in one file-scope
// __device__ array of fixed size, which every GPU that loads the library holds until the
// process exits.  Host code cannot use the array's name as a device address, so the
// address is obtained once per device with cudaGetSymbolAddress (on the first call made
// with that device current) and passed to the kernels.
#include <map>
#include <mutex>

#include "common.cuh"
#include "fft.cuh"
#include "sbd.h"

namespace sbd {

namespace {

constexpr size_t kDataBytes = static_cast<size_t>(SBD_NOALLOC_FFT_MAX_BYTES);
constexpr int kMaxSide = SBD_NOALLOC_FFT_MAX_SIDE;
// per dimension: twiddles (complex128 worst case) and the digit-reversal table
constexpr size_t kTableBytes = static_cast<size_t>(kMaxSide) * (16 + 4);
constexpr size_t kScratchBytes = kDataBytes + 2 * kTableBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
std::map<int, unsigned char*> g_addr;   // device -> device address of g_noalloc_scratch

int scratch_address(unsigned char** out) {
    int dev = 0;
    SBD_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_addr.find(dev);
    if (it != g_addr.end()) {
        *out = it->second;
        return SBD_OK;
    }
    void* p = nullptr;
    SBD_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = static_cast<unsigned char*>(p);
    *out = static_cast<unsigned char*>(p);
    return SBD_OK;
}

// tw[t] = exp(-2 pi i t / n), from the FP64 sincospi of the device
template <typename T>
__global__ void make_twiddles_kernel(cx_t<T>* tw, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s, c;
    sincospi(2.0 * t / n, &s, &c);
    tw[t] = mk<T>(static_cast<T>(c), static_cast<T>(-s));
}

// digit reversal of the plan's radix schedule (the load order of the row transform)
__global__ void make_perm_kernel(int* perm, FftPlan1D plan) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= plan.n) return;
    int weight[kFftMaxStages];
    int w = 1;
    for (int k = 0; k < plan.nstages; ++k) {
        weight[k] = w;
        w *= plan.radix[k];
    }
    int v = i, pos = 0;
    for (int k = plan.nstages - 1; k >= 0; --k) {
        pos += (v % plan.radix[k]) * weight[k];
        v /= plan.radix[k];
    }
    perm[i] = pos;
}

template <typename T>
int run(const void* in, void* out, int n0, int n1, int sign, cudaStream_t s) {
    using C = cx_t<T>;
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    C* tmp = reinterpret_cast<C*>(base);
    C* tw1 = reinterpret_cast<C*>(base + kDataBytes);
    int* perm1 = reinterpret_cast<int*>(base + kDataBytes + static_cast<size_t>(kMaxSide) * 16);
    C* tw0 = reinterpret_cast<C*>(base + kDataBytes + kTableBytes);
    int* perm0 = reinterpret_cast<int*>(base + kDataBytes + kTableBytes + static_cast<size_t>(kMaxSide) * 16);
    FftPlan1D p0, p1;
    if (!fft_make_plan(n0, p0, sizeof(T) == 8) || !fft_make_plan(n1, p1, sizeof(T) == 8)) {
        set_error("sbd_fft2_noalloc: sides must be products of 2, 3 and 5");
        return SBD_ENOTSUP;
    }
    make_twiddles_kernel<T><<<(n1 + 255) / 256, 256, 0, s>>>(tw1, n1);
    make_perm_kernel<<<(n1 + 255) / 256, 256, 0, s>>>(perm1, p1);
    make_twiddles_kernel<T><<<(n0 + 255) / 256, 256, 0, s>>>(tw0, n0);
    make_perm_kernel<<<(n0 + 255) / 256, 256, 0, s>>>(perm0, p0);
    SBD_LAUNCH_CHECK();
    const C* I = static_cast<const C*>(in);
    C* O = static_cast<C*>(out);
    if ((rc = fft_rows_tables<T>(I, n1, n1, tmp, n1, n1, n0, n1, sign, tw1, perm1, s))) return rc;
    if ((rc = transpose<T>(tmp, n1, 0, O, n0, 0, n0, n1, 1, s))) return rc;
    if ((rc = fft_rows_tables<T>(O, n0, n0, tmp, n0, n0, n1, n0, sign, tw0, perm0, s))) return rc;
    return transpose<T>(tmp, n0, 0, O, n1, 0, n1, n0, 1, s);
}

}  // namespace

}  // namespace sbd

extern "C" int sbd_fft2_noalloc(const void* in, void* out, int32_t n0, int32_t n1, int32_t sign, int32_t form,
                                void* cuda_stream) {
    using namespace sbd;
    if (!in || !out || (sign != 1 && sign != -1) || (form != SBD_FORM_FP32 && form != SBD_FORM_FP64)) {
        set_error("sbd_fft2_noalloc: invalid argument");
        return SBD_EINVAL;
    }
    const size_t esz = form == SBD_FORM_FP32 ? 8 : 16;
    if (n0 < 2 || n1 < 2 || n0 > kMaxSide || n1 > kMaxSide ||
        static_cast<size_t>(n0) * static_cast<size_t>(n1) * esz > kDataBytes) {
        set_error("sbd_fft2_noalloc: sides must lie in [2, " + std::to_string(kMaxSide) + "] and n0 * n1 elements in " +
                  std::to_string(kDataBytes) + " bytes");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return form == SBD_FORM_FP32 ? run<float>(in, out, n0, n1, sign, s) : run<double>(in, out, n0, n1, sign, s);
}
