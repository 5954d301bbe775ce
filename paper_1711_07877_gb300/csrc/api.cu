// C ABI of libsbd.so: plan construction (off-line part) and the on-line matvec.
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <omp.h>

#include "bessel.h"
#include "common.cuh"
#include "far.cuh"
#include "fft.cuh"
#include "near.cuh"
#include "node.cuh"
#include "offline.h"
#include "sbd.h"
#include "uniform.cuh"

namespace sbd {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

std::shared_mutex& capture_mutex() {
    static std::shared_mutex mu;
    return mu;
}

int raise_smem_limit_fn(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    SBD_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[{dev, func}];
    if (cur >= bytes) return SBD_OK;
    SBD_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes)));
    cur = bytes;
    return SBD_OK;
}

RadialKernel radial_of(const sbd_radial_kernel& k) {
    RadialKernel r;
    r.value = k.value;
    r.deriv = k.deriv;
    r.laplacian = k.laplacian;
    r.ctx = k.ctx;
    r.log_coef = k.log_coef;
    r.n_enforce = k.n_enforce;
    return r;
}

}  // namespace sbd

using namespace sbd;

struct sbd_plan_s {
    int kind = 0;
    double kappa = 0.0;
    int form = SBD_FORM_FP64;
    long n = 0;
    int max_nrhs = 1;
    SbdFit fit;
    NufftParams np;
    NearTables nt;
    FarGeom geom{};
    cplx w0 = 0.0;
    // device data
    double* z = nullptr;
    void* pts = nullptr;
    void* nodes = nullptr;
    void* omega_c = nullptr;   // per circle: omega_hat * c^2 (T complex)
    void* cscale_c = nullptr;  // per circle: c (T)
    double* psi = nullptr;     // Chebyshev series of the ES spreading deconvolution (null: Gaussian)
    void* dec = nullptr;       // T[m]
    long long* rowptr = nullptr;
    int* col = nullptr;
    void* val = nullptr;
    long long nnz = 0, n_coinc = 0;
    double* T1 = nullptr;
    double* T2 = nullptr;
    double* small_xi = nullptr;
    double* small_w = nullptr;
    int* small_start = nullptr;
    int* circle_start = nullptr;
    double* circle_radius = nullptr;
    int* circle_M = nullptr;
    int* node_perm = nullptr;          // sorted record -> record numbering
    int* half_start = nullptr;         // prefix sums of M_p / 2 (half node set), or null
    bool half_nodes = false;           // Laplace: records for m < M_p / 2 only (Hermitian symmetry); also
                                       // the real-grid path of the transforms
    bool uniform = false;              // uniform-grid variant: the node step is a multiplication by ucoef
    void* ucoef = nullptr;             // nk x nk coefficients (T real for Laplace, cx_t<T> for Helmholtz)
    long long n_rec = 0;               // node records: N_xi, or N_xi / 2 with half_nodes
    int* pt_perm = nullptr;            // sorted point record -> original point index (the
                                       // internal order of D's rows and columns)
    // separate targets (sbd_plan_st): their own records for the interpolation, D's rows in
    // their internal order; for a plan of one point set these alias the source records
    bool separate = false;
    long n_tgt = 0;
    double* zt = nullptr;
    void* tpts = nullptr;
    int* tpt_perm = nullptr;
    PointWork tpt_work{nullptr, nullptr, 0};
    void* f_int = nullptr;             // f in internal order, right-hand sides interleaved
    void* q_int = nullptr;             // D f in internal order, interleaved
    bool d32 = false;                  // D's values and f_int in FP32 (SBD_FLAG_NEAR_FP32)
    PointWork pt_work{nullptr, nullptr, 0};   // chunks of the point records (spread, interp)
    std::vector<long long> pt_ts, tpt_ts;     // tile starts of the source / target records (host)
    int pt_chunk = kPointChunk;               // records per work item (sbd_tune)
    long long* node_tile_start = nullptr;
    void* ghat = nullptr;              // n_xi weighted node values (scratch of the two-kernel node step)
    bool node_fused = true;            // one-kernel node step (shared memory permitting)
    bool node_binned = false;          // the binned node kernel applies (records sorted by bin)
    NodeTuning tuning;                 // fused node-kernel variant (sbd_tune)
    int fft_split = 0;                 // row-FFT phases (sbd_tune): 0 as needed, 2 always two
    int tuned = 0;                     // 1 once sbd_tune chose the variant
    // workspace grids, max_nrhs right-hand sides each (see GridStrides)
    void* wsX = nullptr;
    void* wsB = nullptr;
    void* wsC = nullptr;
    double2* sumf = nullptr;
    double2* zero2 = nullptr;
    // CUDA-graph replay of sbd_matvec (sbd_matvec_graph): fixed input / output buffers,
    // one instantiated graph per nrhs, recorded and launched on a plan-owned stream
    void* g_in = nullptr;
    void* g_out = nullptr;
    std::vector<cudaGraphExec_t> g_exec;
    cudaStream_t g_stream = nullptr;
    cudaEvent_t g_ev_in = nullptr, g_ev_out = nullptr;
    // the near-field product D f runs on its own stream, beside the far part, and joins it
    // before the interpolation (which adds D f)
    cudaStream_t near_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // sbd_matvec_batched: the plan's transforms run on their own stream beside the other
    // instances' (created on the plan's first batched call)
    cudaStream_t b_stream = nullptr;
    cudaEvent_t b_ev = nullptr;
    cudaStream_t alloc_stream = nullptr;   // stream of the allocations being made
    long long device_bytes = 0;
    double plan_seconds = 0.0;
    std::vector<void*> allocations;
    // step timing (sbd_profile): events recorded around each on-line step
    bool profile = false;
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    double stage_ms[SBD_N_STAGES] = {};
    long long stage_count[SBD_N_STAGES] = {};
};

namespace {

// Plan memory is stream-ordered (cudaMallocAsync on the stream the plan is being built or
// extended on, p->alloc_stream; cudaFreeAsync on destroy), so that building and destroying
// plans never synchronises the whole device, and freed memory stays in the device's pool
// for the next plan.
int dev_alloc(sbd_plan_s* p, void** ptr, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    const cudaError_t e = cudaMallocAsync(ptr, bytes, p->alloc_stream);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SBD_ENOMEM : SBD_ECUDA;
    }
    p->allocations.push_back(*ptr);
    p->device_bytes += static_cast<long long>(bytes);
    return SBD_OK;
}

template <typename X>
int upload(sbd_plan_s* p, X** dst, const std::vector<X>& src, cudaStream_t s) {
    int rc = dev_alloc(p, reinterpret_cast<void**>(dst), sizeof(X) * src.size());
    if (rc) return rc;
    if (!src.empty()) SBD_CUDA_TRY(cudaMemcpyAsync(*dst, src.data(), sizeof(X) * src.size(), cudaMemcpyHostToDevice, s));
    return SBD_OK;
}

cudaEvent_t take_event(sbd_plan_s* p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// RAII-free helpers: begin() records the start event, end() the stop event of a step.
struct StepTimer {
    sbd_plan_s* p;
    cudaStream_t s;
    int stage;
    cudaEvent_t a = nullptr;
    StepTimer(sbd_plan_s* p_, cudaStream_t s_, int stage_) : p(p_), s(s_), stage(stage_) {
        if (p->profile) {
            a = take_event(p);
            cudaEventRecord(a, s);
        }
    }
    void end() {
        if (!p->profile || !a) return;
        cudaEvent_t b = take_event(p);
        cudaEventRecord(b, s);
        p->marks.push_back({stage, a, b});
        a = nullptr;
    }
};

void collect_marks(sbd_plan_s* p) {
    for (auto& m : p->marks) {
        cudaEventSynchronize(m.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            p->stage_ms[m.stage] += ms;
            p->stage_count[m.stage] += 1;
        }
        p->event_pool.push_back(m.a);
        p->event_pool.push_back(m.b);
    }
    p->marks.clear();
}

// Frees the plan.  wait_device: first wait for the whole device (sbd_destroy, safe for any
// use of the plan on any stream); otherwise the frees are ordered on stream s after the
// caller's work there (sbd_destroy_async), with only this plan's own graph stream waited for.
void free_plan(sbd_plan_s* p, bool wait_device, cudaStream_t s) {
    if (!p) return;
    if (wait_device) {
        std::unique_lock<std::shared_mutex> lock(capture_mutex());
        cudaDeviceSynchronize();
    } else if (p->g_stream) {
        cudaStreamSynchronize(p->g_stream);
    }
    collect_marks(p);
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    for (cudaGraphExec_t g : p->g_exec)
        if (g) cudaGraphExecDestroy(g);
    if (p->g_ev_in) cudaEventDestroy(p->g_ev_in);
    if (p->g_ev_out) cudaEventDestroy(p->g_ev_out);
    if (p->g_stream) cudaStreamDestroy(p->g_stream);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->near_stream) cudaStreamDestroy(p->near_stream);
    if (p->b_ev) cudaEventDestroy(p->b_ev);
    if (p->b_stream) cudaStreamDestroy(p->b_stream);
    for (void* a : p->allocations) cudaFreeAsync(a, s);
    if (p->rowptr) cudaFreeAsync(p->rowptr, s);
    if (p->col) cudaFreeAsync(p->col, s);
    if (p->val) cudaFreeAsync(p->val, s);
    if (wait_device) cudaStreamSynchronize(s);
    delete p;
}

// Keep freed plan memory in the device's default pool (plans of a server come and go).
void keep_pool_memory() {
    static std::once_flag once;
    std::call_once(once, []() {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            unsigned long long keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
}

SpreadDeconv spread_deconv_of(const sbd_plan_s* p) {
    if (!p->psi) return SpreadDeconv{nullptr, 0, 0.0, 0.0};
    return SpreadDeconv{p->psi, static_cast<int>(p->np.psi.size()), 1.0 / (p->np.kmax * p->np.kmax), p->np.h};
}

// Fills the work list arrays of *work (capacity for the smallest chunk) from tile starts ts.
int fill_work(const std::vector<long long>& ts, int chunk, PointWork* work, cudaStream_t s) {
    std::vector<long long> wb;
    std::vector<int> wt;
    point_work_list(ts, chunk, wb, wt);
    SBD_CUDA_TRY(cudaMemcpyAsync(const_cast<long long*>(work->begin), wb.data(), sizeof(long long) * wb.size(),
                                 cudaMemcpyHostToDevice, s));
    SBD_CUDA_TRY(cudaMemcpyAsync(const_cast<int*>(work->tile), wt.data(), sizeof(int) * wt.size(),
                                 cudaMemcpyHostToDevice, s));
    SBD_CUDA_TRY(cudaStreamSynchronize(s));   // the host vectors go out of scope
    work->count = static_cast<int>(wt.size());
    return SBD_OK;
}

// Records of n points z (stencil start cell and fraction on the spreading grid), sorted by
// 64 x 64 tile (perm: record -> point index), the tile starts (host, ts) and the work list of
// the point kernels: each tile's records in chunks of at most p->pt_chunk (arrays sized for
// the smallest chunk sbd_tune tries).
template <typename T>
int point_records(sbd_plan_s* p, const double* z, long n, void** recs, int** perm, PointWork* work,
                  std::vector<long long>& ts, cudaStream_t s) {
    const NufftParams& np = p->np;
    PointRec<T>* pts0 = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&pts0, sizeof(PointRec<T>) * n, s));
    int rc = far_prepare_points<T>(z, n, np.cx, np.cy, np.h, np.m, np.Ps, pts0, s);
    if (rc) return rc;
    const int ntm = (np.m + kNodeTile - 1) / kNodeTile;
    long long* tile_start = nullptr;
    if ((rc = dev_alloc(p, recs, sizeof(PointRec<T>) * n))) return rc;
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(perm), sizeof(int) * n))) return rc;
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(&tile_start),
                        sizeof(long long) * (static_cast<size_t>(ntm) * ntm + 1)))) return rc;
    if ((rc = tile_sort<PointRec<T>>(pts0, n, np.m, static_cast<PointRec<T>*>(*recs), *perm, tile_start, s)))
        return rc;
    SBD_CUDA_TRY(cudaFreeAsync(pts0, s));
    ts.assign(static_cast<size_t>(ntm) * ntm + 1, 0);
    SBD_CUDA_TRY(cudaMemcpyAsync(ts.data(), tile_start, sizeof(long long) * ts.size(), cudaMemcpyDeviceToHost, s));
    SBD_CUDA_TRY(cudaStreamSynchronize(s));
    long long cap = 0;
    for (size_t t = 0; t + 1 < ts.size(); ++t) cap += (ts[t + 1] - ts[t] + kPointChunks[0] - 1) / kPointChunks[0];
    long long* wbd = nullptr;
    int* wtd = nullptr;
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(&wbd), sizeof(long long) * (cap + 1)))) return rc;
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(&wtd), sizeof(int) * std::max<long long>(cap, 1)))) return rc;
    *work = PointWork{wbd, wtd, 0};
    return fill_work(ts, p->pt_chunk, work, s);
}

template <typename T>
int build_far(sbd_plan_s* p, cudaStream_t s) {
    const NufftParams& np = p->np;
    const SbdFit& fit = p->fit;
    p->geom.Ps = np.Ps;
    p->geom.Pk = np.Pk;
    p->geom.m = np.m;
    p->geom.nk = np.nk;
    p->geom.kwin = np.kwin;
    p->geom.beta_s = np.beta_s;
    p->geom.beta_k = np.beta_k;
    p->geom.swin = np.swin;
    if (np.swin == 1) {
        const int urc = upload(p, &p->psi, np.psi, s);
        if (urc) return urc;
    }
    p->geom.kpoly = p->geom.spoly = nullptr;
    p->geom.kpoly64 = p->geom.spoly64 = nullptr;
    if constexpr (sizeof(T) == 8) {   // the FP64 kernels' polynomial windows, where the fit holds
        std::vector<double> tab(kWinPolyEntries64);
        double* d = nullptr;
        if (window_poly64(np.kwin, np.beta_k, np.Pk, np.tol, tab.data())) {
            const int urc = upload(p, &d, tab, s);
            if (urc) return urc;
            p->geom.kpoly64 = d;
        }
        if (window_poly64(np.swin, np.beta_s, np.Ps, np.tol, tab.data())) {
            const int urc = upload(p, &d, tab, s);
            if (urc) return urc;
            p->geom.spoly64 = d;
        }
    }
    p->geom.node_bins = nullptr;
    p->geom.node_order = nullptr;
    p->geom.n_node_tiles = 0;
    if constexpr (sizeof(T) == 4) {   // the FP32 kernels' polynomial windows, where the fit holds
        std::vector<float4> tab(kWinPolyEntries);
        float4* d = nullptr;
        if (window_poly(np.kwin, np.beta_k, np.Pk, np.tol, tab.data())) {
            const int urc = upload(p, &d, tab, s);
            if (urc) return urc;
            p->geom.kpoly = d;
        }
        if (window_poly(np.swin, np.beta_s, np.Ps, np.tol, tab.data())) {
            const int urc = upload(p, &d, tab, s);
            if (urc) return urc;
            p->geom.spoly = d;
        }
    }
    int rc = point_records<T>(p, p->z, p->n, &p->pts, &p->pt_perm, &p->pt_work, p->pt_ts, s);
    if (rc) return rc;
    if (p->separate) {
        if ((rc = point_records<T>(p, p->zt, p->n_tgt, &p->tpts, &p->tpt_perm, &p->tpt_work, p->tpt_ts, s)))
            return rc;
    } else {
        p->tpts = p->pts;
        p->tpt_perm = p->pt_perm;
        p->tpt_work = p->pt_work;
    }
    if (p->uniform) {
        // no quadrature nodes: the coefficients of the windowed series on the frequency grid
        p->half_nodes = p->kind != SBD_HELMHOLTZ;
        p->n_rec = 0;
        p->node_fused = false;
        const bool cc = p->kind == SBD_HELMHOLTZ;
        const size_t nk = np.nk;
        if ((rc = dev_alloc(p, &p->ucoef, (cc ? sizeof(cx_t<T>) : sizeof(T)) * nk * nk))) return rc;
        if ((rc = uniform_coefficients<T>(fit, np, spread_deconv_of(p), cc, p->ucoef, s))) return rc;
        const size_t e = sizeof(cx_t<T>) * static_cast<size_t>(p->max_nrhs);
        const size_t m = np.m;
        if ((rc = dev_alloc(p, &p->wsX, e * m * m))) return rc;
        if ((rc = dev_alloc(p, &p->wsB, e * nk * nk))) return rc;
        if ((rc = dev_alloc(p, &p->wsC, e * nk * nk))) return rc;
        return SBD_OK;
    }
    std::vector<int> start(fit.n_circles + 1, 0);
    for (int c = 0; c < fit.n_circles; ++c) start[c + 1] = start[c] + fit.M[c];
    if (fit.n_xi > 2000000000LL) {
        set_error("too many quadrature nodes for 32-bit circle offsets");
        return SBD_ENOTSUP;
    }
    if ((rc = upload(p, &p->circle_start, start, s))) return rc;
    // Laplace: f, the spreading grid and omega' are real, so the frequency grid K is
    // Hermitian (K(-eta) = conj K(eta)) and the node at -xi gives the conjugate of the
    // one at xi.  Only the nodes m < M_p / 2 of each circle (M_p is even) are stored;
    // the node step's output S over those nodes completes to S(eta) + conj(S(-eta)),
    // which the inverse transform folds into its load.
    p->half_nodes = p->kind != SBD_HELMHOLTZ;
    p->n_rec = fit.n_xi;
    if (p->half_nodes) {
        std::vector<int> hstart(fit.n_circles + 1, 0);
        for (int c = 0; c < fit.n_circles; ++c) hstart[c + 1] = hstart[c] + fit.M[c] / 2;
        if ((rc = upload(p, &p->half_start, hstart, s))) return rc;
        p->n_rec = hstart[fit.n_circles];
    }
    if ((rc = upload(p, &p->circle_radius, fit.radius, s))) return rc;
    if ((rc = upload(p, &p->circle_M, fit.M, s))) return rc;
    std::vector<cx_t<T>> om(fit.n_circles);
    std::vector<T> cs(fit.n_circles);
    for (int c = 0; c < fit.n_circles; ++c) {
        const cplx w = fit.weight[c] * np.circle_factor[c];
        om[c] = mk<T>(static_cast<T>(w.real()), static_cast<T>(w.imag()));
        cs[c] = static_cast<T>(std::sqrt(np.circle_factor[c]));
    }
    if ((rc = upload(p, reinterpret_cast<cx_t<T>**>(&p->omega_c), om, s))) return rc;
    if ((rc = upload(p, reinterpret_cast<T**>(&p->cscale_c), cs, s))) return rc;
    NodeRec<T>* canon = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&canon, sizeof(NodeRec<T>) * std::max<long long>(p->n_rec, 1), s));
    rc = far_prepare_nodes<T>(p->circle_start, p->half_start, p->circle_radius, p->circle_M, fit.n_circles,
                              p->n_rec, np.deta, np.nk, np.Pk, static_cast<const cx_t<T>*>(p->omega_c),
                              spread_deconv_of(p), canon, s);
    if (rc) return rc;
    {
        // bound of one product g w_a w_b of the fixed-point node variant: the largest record weight
        // (deconvolution included) x 2 (complex product) x P_k^2 (window values <= 1)
        double wmax = 0.0;
        if ((rc = far_weight_max<T>(canon, p->n_rec, &wmax, s))) return rc;
        p->tuning.wbound = static_cast<float>(2.0 * wmax * np.Pk * np.Pk);
    }
    const int ntx = (np.nk + kNodeTile - 1) / kNodeTile;
    if ((rc = dev_alloc(p, &p->nodes, sizeof(NodeRec<T>) * p->n_rec))) return rc;
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(&p->node_perm), sizeof(int) * p->n_rec))) return rc;
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(&p->node_tile_start),
                        sizeof(long long) * (static_cast<size_t>(ntx) * ntx + 1)))) return rc;
    // FP32 records go in bin order (the binned node kernel needs it; the others take any)
    const bool by_bin = sizeof(T) == 4 && np.Pk <= kBinSide;
    rc = tile_sort<NodeRec<T>>(canon, p->n_rec, np.nk, static_cast<NodeRec<T>*>(p->nodes), p->node_perm,
                               p->node_tile_start, s, by_bin);
    if (rc) return rc;
    SBD_CUDA_TRY(cudaFreeAsync(canon, s));
    // the fused node kernel holds the tile plus halo and two accumulator planes in shared memory
    p->node_fused = node_fused_smem<T>(np.Pk) <= 227 * 1024;
    if (by_bin) {
        // the binned kernel also needs every tile sorted, i.e. within the sort's capacity
        std::vector<long long> ts(static_cast<size_t>(ntx) * ntx + 1);
        SBD_CUDA_TRY(cudaMemcpyAsync(ts.data(), p->node_tile_start, sizeof(long long) * ts.size(),
                                     cudaMemcpyDeviceToHost, s));
        SBD_CUDA_TRY(cudaStreamSynchronize(s));
        long long most = 0;
        for (size_t t = 0; t + 1 < ts.size(); ++t) most = std::max(most, ts[t + 1] - ts[t]);
        p->node_binned = p->node_fused && most <= kTileSortMax && node_fused_smem<T>(np.Pk, 3) <= 227 * 1024;
        if (p->node_binned) {
            p->tuning.acc = 3, p->tuning.sched = 1;   // the fastest untuned choice
            if constexpr (sizeof(T) == 4) {
                void* bins = nullptr;
                const int ntiles = ntx * ntx;
                if ((rc = dev_alloc(p, &bins, sizeof(BinTable) * static_cast<size_t>(ntiles)))) return rc;
                if ((rc = node_bin_tables(static_cast<const NodeRec<float>*>(p->nodes), p->node_tile_start, ntiles,
                                          static_cast<BinTable*>(bins), s))) return rc;
                p->geom.node_bins = bins;
                // the persistent kernel's walk: tiles with records, most first (ties by tile)
                std::vector<int> order;
                for (int t = 0; t < ntiles; ++t)
                    if (ts[t + 1] > ts[t]) order.push_back(t);
                std::stable_sort(order.begin(), order.end(),
                                 [&](int a, int b) { return ts[a + 1] - ts[a] > ts[b + 1] - ts[b]; });
                if (!order.empty()) {
                    int* d = nullptr;
                    if ((rc = upload(p, &d, order, s))) return rc;
                    p->geom.node_order = d;
                    p->geom.n_node_tiles = static_cast<int>(order.size());
                }
            }
        }
    }
    if (!p->node_fused && (rc = dev_alloc(p, &p->ghat, sizeof(cx_t<T>) * p->n_rec))) return rc;
    std::vector<T> dec(np.m);
    for (int i = 0; i < np.m; ++i) dec[i] = static_cast<T>(np.dec[i]);
    if ((rc = upload(p, reinterpret_cast<T**>(&p->dec), dec, s))) return rc;
    // workspace grids for max_nrhs right-hand sides at once (grid r at r times the grid size)
    const size_t e = sizeof(cx_t<T>) * static_cast<size_t>(p->max_nrhs);
    const size_t m = np.m, nk = np.nk;
    if ((rc = dev_alloc(p, &p->wsX, e * m * m))) return rc;
    if ((rc = dev_alloc(p, &p->wsB, e * nk * nk))) return rc;
    if ((rc = dev_alloc(p, &p->wsC, e * nk * nk))) return rc;
    return SBD_OK;
}

// Workspace grids hold nb right-hand sides each, grid b at b times the grid's size (complex
// elements): X (spreading grid) m x m, or m^2 / 2 for the packed real grid of Laplace, B and C
// (frequency grids) nk x nk, which also hold the transposed first pass (nk x m) of a transform.
struct GridStrides {
    long X, K;
};
GridStrides grid_strides(const NufftParams& np, bool real = false) {
    const long m = np.m, nk = np.nk;
    return {real ? m * m / 2 : m * m, nk * nk};
}

// spreading grid X (m x m, rows = y) -> frequency grid K (nk x nk, rows = kx), forward transform.
// Tr (>= nk x m) is scratch.  nb grids in one pass each.
template <typename T>
int forward_fft(sbd_plan_s* p, const cx_t<T>* X, cx_t<T>* Tr, cx_t<T>* K, cudaStream_t s, int nb = 1) {
    const NufftParams& np = p->np;
    const int m = np.m, nk = np.nk, n = np.n;
    const GridStrides g = grid_strides(np);
    const T* dec = p->uniform ? nullptr : static_cast<const T*>(p->dec);
    // along x (rows y), precorrection exp(sigma |x|^2) fused into the load
    const int sp = p->fft_split;
    // written transposed: [kx][y], the rows of the pass along y
    int rc = fft_rows<T>(X, m, m, -m / 2, Tr, 1, nk, -nk / 2, m, n, -1, dec, dec, nullptr, nullptr, s, 0, 0, kIoPlain,
                         sp, nb, g.X, g.K, m);
    if (rc) return rc;
    // along y (rows kx)
    return fft_rows<T>(Tr, m, m, -m / 2, K, nk, nk, -nk / 2, nk, n, -1, nullptr, nullptr, nullptr, nullptr, s, 0, 0,
                       kIoPlain, sp, nb, g.K, g.K);
}

// frequency grid K2 (nk x nk, rows = kx) -> spreading grid X (m x m), adjoint transform.
// Tr (>= m x nk) is scratch.
// With fold, K2 holds the node step's S over the half node set and the transform is
// taken of S(eta) + conj(S(-eta)).
template <typename T>
int inverse_fft(sbd_plan_s* p, const cx_t<T>* K2, cx_t<T>* Tr, cx_t<T>* X, cudaStream_t s,
                bool fold, int nb = 1) {
    const NufftParams& np = p->np;
    const int m = np.m, nk = np.nk, n = np.n;
    const GridStrides g = grid_strides(np);
    const T* dec = p->uniform ? nullptr : static_cast<const T*>(p->dec);
    const int sp = p->fft_split;
    // written transposed: [y][kx]
    int rc = fft_rows<T>(K2, nk, nk, -nk / 2, Tr, 1, m, -m / 2, nk, n, +1, nullptr, nullptr, nullptr, nullptr, s,
                         fold ? nk : 0, 0, kIoPlain, sp, nb, g.K, g.K, nk);
    if (rc) return rc;
    return fft_rows<T>(Tr, nk, nk, -nk / 2, X, m, m, -m / 2, m, n, +1, nullptr, nullptr, dec, dec, s, 0, 0, kIoPlain,
                       sp, nb, g.K, g.X);
}

// Real data (Laplace): the spreading grid X is real, stored as packed row pairs
// (m / 2 x m complex), and K is Hermitian.  Forward: one transform per row pair,
// split into the two rows' spectra, of which only kx >= kx_lo (the half plane of the
// half node set plus the stencil reach) is kept; then the transforms along y for
// those kx only, into rows kx_lo.. of K.
template <typename T>
int kx_low(const sbd_plan_s* p) { return p->np.nk / 2 - (p->np.Pk / 2 + 2); }

template <typename T>
int forward_fft_real(sbd_plan_s* p, const cx_t<T>* Xp, cx_t<T>* Tr, cx_t<T>* K, cudaStream_t s,
                     int nb = 1) {
    const NufftParams& np = p->np;
    const int m = np.m, nk = np.nk, n = np.n;
    const GridStrides g = grid_strides(np, true);
    const int lo = kx_low<T>(p), w2 = nk - lo;
    const T* dec = p->uniform ? nullptr : static_cast<const T*>(p->dec);
    const int sp = p->fft_split;
    // written transposed: [kx][y]
    int rc = fft_rows<T>(Xp, m, m, -m / 2, Tr, 1, w2, lo - nk / 2, m / 2, n, -1, dec, dec, nullptr, nullptr, s, 0, 0,
                         kIoPairFwd, sp, nb, g.X, g.K, m);
    if (rc) return rc;
    return fft_rows<T>(Tr, m, m, -m / 2, K + static_cast<long>(lo) * nk, nk, nk, -nk / 2, w2, n, -1, nullptr, nullptr,
                       nullptr, nullptr, s, 0, 0, kIoPlain, sp, nb, g.K, g.K);
}

// Adjoint for real data: S (node step over the half node set) completes to
// S(eta) + conj(S(-eta)), which is Hermitian, so only kx >= 0 is transformed along y
// (the fold is applied on the load); then each pair of y rows is one transform along
// x from its two half spectra, giving the packed real X.
template <typename T>
int inverse_fft_real(sbd_plan_s* p, const cx_t<T>* S, cx_t<T>* Tr, cx_t<T>* Xp, cudaStream_t s,
                     int nb = 1) {
    const NufftParams& np = p->np;
    const int m = np.m, nk = np.nk, n = np.n;
    const GridStrides g = grid_strides(np, true);
    const int J = nk / 2;
    const T* dec = p->uniform ? nullptr : static_cast<const T*>(p->dec);
    const int sp = p->fft_split;
    // the node step's S completes by the Hermitian fold; the uniform variant's product is whole
    const int herm = p->uniform ? 0 : nk;
    // written transposed: [y][kx]
    int rc = fft_rows<T>(S + static_cast<long>(J) * nk, nk, nk, -nk / 2, Tr, 1, m, -m / 2, J, n, +1, nullptr, nullptr,
                         nullptr, nullptr, s, herm, herm ? J : 0, kIoPlain, sp, nb, g.K, g.K, J, kx_low<T>(p));
    if (rc) return rc;
    return fft_rows<T>(Tr, J, J, 0, Xp, m, m, -m / 2, m / 2, n, +1, nullptr, nullptr, dec, dec, s, 0, 0, kIoPairInv,
                       sp, nb, g.K, g.X);
}

// q = far part of f (+ the internal-order near term add[i * nrhs + r] when add is given).
// Every step takes all nrhs right-hand sides in one launch (grids stored right-hand side
// by right-hand side in the workspace): 9 launches per call whatever nrhs.
template <typename T>
int far_apply(sbd_plan_s* p, const void* f, void* q, int nrhs, cudaStream_t s, const void* add,
              cudaEvent_t join = nullptr) {
    const bool cplx_io = p->kind == SBD_HELMHOLTZ;
    StepTimer t_sum(p, s, SBD_STAGE_SUM);
    int rc = far_sum(f, cplx_io, p->n, nrhs, p->sumf, s);
    if (rc) return rc;
    t_sum.end();
    auto* X = static_cast<cx_t<T>*>(p->wsX);
    auto* B = static_cast<cx_t<T>*>(p->wsB);
    auto* C = static_cast<cx_t<T>*>(p->wsC);
    const double2 w0 = make_double2(p->w0.real(), p->w0.imag());
    const bool real = p->half_nodes;   // Laplace: real grids, half the transforms and nodes
    StepTimer t1(p, s, SBD_STAGE_SPREAD);
    if ((rc = spread_tiled<T>(static_cast<const PointRec<T>*>(p->pts), p->pt_perm, p->pt_work, p->geom, f, cplx_io,
                              X, s, real, nrhs, p->n))) return rc;
    t1.end();
    StepTimer t2(p, s, SBD_STAGE_FFT_FWD);
    if ((rc = real ? forward_fft_real<T>(p, X, C, B, s, nrhs) : forward_fft<T>(p, X, C, B, s, nrhs))) return rc;
    t2.end();
    StepTimer t3(p, s, SBD_STAGE_NODE);
    if (p->uniform) {
        // rows kx >= 0 (the real path's inverse reads only those) or all rows
        const int nk = p->np.nk;
        if ((rc = uniform_multiply<T>(B, p->ucoef, p->kind == SBD_HELMHOLTZ, C, nk, real ? nk / 2 : 0, nrhs,
                                      static_cast<long>(nk) * nk, s))) return rc;
    } else if (p->node_fused) {
        // the real path's inverse reads rows kx_low.. only
        if ((rc = node_step_fused<T>(static_cast<const NodeRec<T>*>(p->nodes), p->node_tile_start, p->geom, B, C,
                                     p->tuning, s, nrhs, real ? kx_low<T>(p) : 0))) return rc;
    } else if ((rc = node_step_tiled<T>(static_cast<const NodeRec<T>*>(p->nodes), p->node_tile_start, p->geom, B,
                                        static_cast<cx_t<T>*>(p->ghat), C, s, nrhs))) {
        return rc;
    }
    t3.end();
    StepTimer t4(p, s, SBD_STAGE_FFT_INV);
    if ((rc = real ? inverse_fft_real<T>(p, C, B, X, s, nrhs) : inverse_fft<T>(p, C, B, X, s, false, nrhs)))
        return rc;
    t4.end();
    if (join) SBD_CUDA_TRY(cudaStreamWaitEvent(s, join, 0));   // D f is ready
    StepTimer t5(p, s, SBD_STAGE_INTERP);
    if ((rc = interp_tiled<T>(static_cast<const PointRec<T>*>(p->tpts), p->tpt_perm, p->tpt_work, p->geom, X, w0,
                              p->sumf, q, cplx_io, s, real, add, nrhs, nrhs, p->n_tgt))) return rc;
    t5.end();
    return SBD_OK;
}

template <typename T>
int nufft_minus_impl(sbd_plan_s* p, const void* f, void* fhat, cudaStream_t s) {
    auto* X = static_cast<cx_t<T>*>(p->wsX);
    auto* B = static_cast<cx_t<T>*>(p->wsB);
    auto* C = static_cast<cx_t<T>*>(p->wsC);
    int rc = spread_tiled<T>(static_cast<const PointRec<T>*>(p->pts), p->pt_perm, p->pt_work, p->geom, f,
                             true, X, s);
    if (rc) return rc;
    if ((rc = forward_fft<T>(p, X, C, B, s))) return rc;
    const NodeFrame fr{p->circle_start, p->circle_radius, p->circle_M, p->fit.n_circles, p->np.cx, p->np.cy,
                       p->node_perm, p->half_start, p->np.nk, spread_deconv_of(p)};
    return far_node_gather<T>(static_cast<const NodeRec<T>*>(p->nodes), p->n_rec,
                              static_cast<const T*>(p->cscale_c), p->geom, B, static_cast<double2*>(fhat), fr, s);
}

template <typename T>
int nufft_plus_impl(sbd_plan_s* p, const void* ghat, void* q, cudaStream_t s) {
    auto* X = static_cast<cx_t<T>*>(p->wsX);
    auto* B = static_cast<cx_t<T>*>(p->wsB);
    auto* C = static_cast<cx_t<T>*>(p->wsC);
    const NodeFrame fr{p->circle_start, p->circle_radius, p->circle_M, p->fit.n_circles, p->np.cx, p->np.cy,
                       p->node_perm, p->half_start, p->np.nk, spread_deconv_of(p)};
    int rc = far_node_scatter<T>(static_cast<const NodeRec<T>*>(p->nodes), p->n_rec,
                                 static_cast<const T*>(p->cscale_c), p->geom, static_cast<const double2*>(ghat), C,
                                 fr, s);
    if (rc) return rc;
    if ((rc = inverse_fft<T>(p, C, B, X, s, false))) return rc;
    SBD_CUDA_TRY(cudaMemsetAsync(p->zero2, 0, sizeof(double2), s));
    return interp_tiled<T>(static_cast<const PointRec<T>*>(p->tpts), p->tpt_perm, p->tpt_work, p->geom, X,
                           make_double2(0, 0), p->zero2, q, true, s);
}

int check_plan_call(sbd_plan_t p, const void* a, const void* b) {
    if (!p || !a || !b) {
        set_error("null plan or buffer");
        return SBD_EINVAL;
    }
    return SBD_OK;
}

// Options that every entry point taking sbd_options accepts: a known form and flag set,
// non-negative counts and tolerances.
bool options_valid(const sbd_options& o) {
    const int known = SBD_FLAG_GAUSSIAN_NODES | SBD_FLAG_GAUSSIAN_SPREAD | SBD_FLAG_SPREAD_SIGMA_2 |
                      SBD_FLAG_SPREAD_SIGMA_15 | SBD_FLAG_NEAR_FP32 | SBD_FLAG_UNIFORM_GRID |
                      SBD_FLAG_SPREAD_SIGMA_125;
    const int sig = o.flags & (SBD_FLAG_SPREAD_SIGMA_2 | SBD_FLAG_SPREAD_SIGMA_15 | SBD_FLAG_SPREAD_SIGMA_125);
    const int not_uniform = SBD_FLAG_GAUSSIAN_NODES | SBD_FLAG_GAUSSIAN_SPREAD;
    return (o.form == SBD_FORM_FP64 || o.form == SBD_FORM_FP32) && (o.flags & ~known) == 0 &&
           !((o.flags & SBD_FLAG_UNIFORM_GRID) && (o.flags & not_uniform)) &&
           !((o.flags & SBD_FLAG_NEAR_FP32) && o.form != SBD_FORM_FP32) &&
           (sig & (sig - 1)) == 0 &&   // at most one oversampling flag
           !((o.flags & SBD_FLAG_GAUSSIAN_SPREAD) && (o.flags & (SBD_FLAG_SPREAD_SIGMA_15 | SBD_FLAG_SPREAD_SIGMA_125))) &&
           o.fixed_P >= 0 &&
           o.max_nrhs >= 0 && o.nufft_tol >= 0 && o.delta_max >= 0 && o.host_threads >= 0;
}

// Transform parameters of a plan (sbd_plan and sbd_transform_params): each type-3 transform
// gets eps / (6 sum_nu |omega_nu|) unless options.nufft_tol is given, with the windows and
// spreading oversampling the flags select; half = half side of the points' bounding box.
int plan_transform_params(const SbdFit& fit, const sbd_options& o, double eps, double half, double cx, double cy,
                          long n, NufftParams& np, std::string& err) {
    double W = 0.0;
    for (int c = 0; c < fit.n_circles; ++c) W += fit.M[c] * std::abs(fit.weight[c]);
    const double tol = o.nufft_tol > 0 ? o.nufft_tol : eps / (6.0 * std::max(W, 1e-300));
    const int kwin = (o.flags & SBD_FLAG_GAUSSIAN_NODES) ? 0 : 1;
    const int swin = (o.flags & SBD_FLAG_GAUSSIAN_SPREAD) ? 0 : 1;
    const int sigma_mode = (o.flags & SBD_FLAG_SPREAD_SIGMA_15)    ? 1
                           : (o.flags & SBD_FLAG_SPREAD_SIGMA_2)   ? 2
                           : (o.flags & SBD_FLAG_SPREAD_SIGMA_125) ? 3
                                                                   : 0;
    int rc = (o.flags & SBD_FLAG_UNIFORM_GRID)
                 ? uniform_params(fit, half, cx, cy, tol, o.form == SBD_FORM_FP32, swin, sigma_mode, n, np, err)
                 : nufft_params(fit, half, cx, cy, tol, o.form == SBD_FORM_FP32, kwin, swin, sigma_mode, n, np, err);
    if (rc) return rc;
    if (np.n > fft_max_length(o.form == SBD_FORM_FP64)) {
        err = "sbd_plan: FFT length " + std::to_string(np.n) + " exceeds the row kernel limit";
        return SBD_ENOTSUP;
    }
    return SBD_OK;
}

}  // namespace

extern "C" {

const char* sbd_version(void) { return "sbd-gb300 0.1"; }

const char* sbd_error_string(int code) {
    switch (code) {
        case SBD_OK: return "ok";
        case SBD_EINVAL: return "invalid argument";
        case SBD_ENOMEM: return "out of memory";
        case SBD_ECUDA: return "CUDA error";
        case SBD_EFIT: return "SBD fit cannot reach the tolerance";
        case SBD_ETIMEOUT: return "device wait timed out";
        case SBD_ENOTSUP: return "not supported";
        default: return "unknown error";
    }
}

const char* sbd_last_error_message(void) { return g_last_error.c_str(); }

int sbd_offline_fit(sbd_kernel kernel, double delta_min, double delta_max, double eps, int32_t fixed_P,
                    int64_t cap, double* rho, double* alpha, int32_t* M, int64_t* P_out, int64_t* n_circles_out,
                    double* fit_err) {
    SbdFit fit;
    std::string err;
    const int rc = offline_fit(kernel.kind, kernel.kappa, delta_min, delta_max, eps, fixed_P, fit, err);
    if (rc) {
        set_error(err);
        return rc;
    }
    if (cap < fit.n_circles) {
        set_error("capacity below the number of circles");
        return SBD_EINVAL;
    }
    for (int c = 0; c < fit.n_circles; ++c) {
        if (rho) rho[c] = c < fit.P ? fit.rho[c] : 0.0;
        if (alpha) alpha[c] = c < fit.P ? fit.alpha[c] : 0.0;
        if (M) M[c] = fit.M[c];
    }
    if (P_out) *P_out = fit.P;
    if (n_circles_out) *n_circles_out = fit.n_circles;
    if (fit_err) *fit_err = fit.fit_err;
    return SBD_OK;
}

int sbd_offline_fit_radial(const sbd_radial_kernel* kernel, double delta_min, double delta_max, double eps,
                           int32_t fixed_P, int64_t cap, double* rho, double* alpha, int32_t* M, int64_t* P_out,
                           int64_t* n_circles_out, double* fit_err, double* w0_out) {
    if (!kernel) {
        set_error("sbd_offline_fit_radial: null kernel");
        return SBD_EINVAL;
    }
    SbdFit fit;
    std::string err;
    const int rc = offline_fit_radial(radial_of(*kernel), delta_min, delta_max, eps, fixed_P, fit, err);
    if (rc) {
        set_error(err);
        return rc;
    }
    if (cap < fit.n_circles) {
        set_error("capacity below the number of circles");
        return SBD_EINVAL;
    }
    for (int c = 0; c < fit.n_circles; ++c) {
        const bool bessel = c < fit.P;
        const int t = c - fit.P;
        if (rho) rho[c] = bessel ? fit.rho[c] : fit.enf_omega[t];
        if (alpha) alpha[c] = bessel ? fit.alpha[c] : fit.enf_mu[t] / bessel_j0(fit.enf_omega[t]);
        if (M) M[c] = fit.M[c];
    }
    if (P_out) *P_out = fit.P;
    if (n_circles_out) *n_circles_out = fit.n_circles;
    if (fit_err) *fit_err = fit.fit_err;
    if (w0_out) *w0_out = fit.w0.real();
    return SBD_OK;
}

int sbd_transform_params(sbd_kernel kernel, double delta_min, double delta_max, double eps, int64_t n_points,
                         double half_extent, const sbd_options* opt, sbd_transform_stats* out) {
    sbd_options o{};
    o.form = SBD_FORM_FP64;
    if (opt) o = *opt;
    if (!out || n_points < 1 || !(half_extent > 0) || !(delta_min > 0) || !(delta_min < delta_max) ||
        !(eps >= 1e-10 && eps <= 0.1) || !options_valid(o) ||
        (kernel.kind != SBD_LAPLACE && kernel.kind != SBD_HELMHOLTZ) ||
        (kernel.kind == SBD_HELMHOLTZ && !(kernel.kappa > 0))) {
        set_error("sbd_transform_params: null output, n_points < 1, half_extent <= 0, delta_min outside "
                  "(0, delta_max), eps outside [1e-10, 0.1], invalid options or kernel");
        return SBD_EINVAL;
    }
    SbdFit fit;
    NufftParams np;
    std::string err;
    int rc = offline_fit(kernel.kind, kernel.kappa, delta_min, delta_max, eps, o.fixed_P, fit, err);
    if (!rc) rc = plan_transform_params(fit, o, eps, half_extent, 0.0, 0.0, static_cast<long>(n_points), np, err);
    if (rc) {
        set_error(err);
        return rc;
    }
    out->sigma_s = np.sigma_s;
    out->h = np.h;
    out->deta = np.deta;
    out->nufft_tol = np.tol;
    out->grid_x = np.m;
    out->grid_k = np.nk;
    out->fft_n = np.n;
    out->stencil_x = np.Ps;
    out->stencil_k = np.Pk;
    out->spread_window = np.swin;
    out->P = fit.P;
    out->n_circles = fit.n_circles;
    out->n_xi = fit.n_xi;
    return SBD_OK;
}

int sbd_fit_cache_stats(int64_t* hits, int64_t* misses, int64_t* entries) {
    long long h, m, e;
    fit_cache_stats(h, m, e);
    if (hits) *hits = h;
    if (misses) *misses = m;
    if (entries) *entries = e;
    return SBD_OK;
}

int sbd_y0_root(int32_t k, double* root) {
    if (k < 1 || !root) {
        set_error("sbd_y0_root: need k >= 1 and an output pointer");
        return SBD_EINVAL;
    }
    *root = y0_root(k);
    return SBD_OK;
}

int sbd_set_fit_device(int32_t mode) {
    if (mode < 0 || mode > 2) {
        set_error("sbd_set_fit_device: mode outside 0..2");
        return SBD_EINVAL;
    }
    set_fit_device(mode);
    return SBD_OK;
}

int sbd_fit_last_factorisation(double* seconds, int32_t* where) {
    int w = 0;
    last_factorisation(seconds, &w);
    if (where) *where = w;
    return SBD_OK;
}

int sbd_fit_cache_clear(void) {
    fit_cache_clear();
    return SBD_OK;
}

}  // extern "C"

namespace {

// The off-line part for sources `points` (n) and, when targets is non-null, separate targets
// (n_t); targets null is the plan of one point set (D square, its diagonal the self pairs).
int plan_impl(const double* targets, int64_t n_t, const double* points, int64_t n, sbd_kernel kernel,
              double delta_min, double eps, const sbd_options* opt, void* cuda_stream, sbd_plan_t* out,
              const RadialKernel* radial = nullptr) {
    const auto t0 = std::chrono::steady_clock::now();
    const bool separate = targets != nullptr;
    if (!points || !out || n < 1 || (separate && n_t < 1)) {
        set_error("sbd_plan: null pointer or a point count below 1");
        return SBD_EINVAL;
    }
    if (n > 2000000000LL || n_t > 2000000000LL) {
        set_error("sbd_plan: point count exceeds 32-bit column indices");
        return SBD_ENOTSUP;
    }
    sbd_options o{};
    o.form = SBD_FORM_FP64;
    if (opt) o = *opt;
    if (!options_valid(o)) {
        set_error("sbd_plan: invalid options (form, flags or a negative count or tolerance)");
        return SBD_EINVAL;
    }
    if (kernel.kind == SBD_HELMHOLTZ && !(kernel.kappa > 0)) {
        set_error("sbd_plan: Helmholtz needs kappa > 0");
        return SBD_EINVAL;
    }
    if (kernel.kind != SBD_LAPLACE && kernel.kind != SBD_HELMHOLTZ && !(kernel.kind == SBD_RADIAL && radial)) {
        set_error("sbd_plan: unknown kernel");
        return SBD_EINVAL;
    }
    if (radial && (o.flags & SBD_FLAG_UNIFORM_GRID)) {
        set_error("sbd_plan_radial: the uniform-grid variant takes the Laplace and Helmholtz kernels only");
        return SBD_ENOTSUP;
    }
    if (!(eps >= 1e-10 && eps <= 0.1) || !(delta_min > 0)) {
        set_error("sbd_plan: need 1e-10 <= eps <= 0.1 and delta_min > 0");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (o.host_threads > 0) omp_set_num_threads(o.host_threads);   // this thread's parallel regions
    keep_pool_memory();
    auto* p = new sbd_plan_s();
    if (cudaStreamCreateWithFlags(&p->near_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        set_error("sbd_plan: cannot create the plan's stream and events");
        free_plan(p, false, s);
        return SBD_ECUDA;
    }
    p->alloc_stream = s;
    p->kind = kernel.kind;
    p->kappa = kernel.kappa;
    p->form = o.form;
    p->n = static_cast<long>(n);
    p->separate = separate;
    p->n_tgt = separate ? static_cast<long>(n_t) : p->n;
    p->max_nrhs = std::max(1, o.max_nrhs);
    auto fail = [&](int rc) {
        free_plan(p, false, s);
        cudaStreamSynchronize(s);
        return rc;
    };
    int rc = dev_alloc(p, reinterpret_cast<void**>(&p->z), sizeof(double) * 2 * n);
    if (rc) return fail(rc);
    if (cudaMemcpyAsync(p->z, points, sizeof(double) * 2 * n, cudaMemcpyDefault, s) != cudaSuccess) {
        set_error("sbd_plan: copying the points failed (device pointer expected)");
        cudaGetLastError();
        return fail(SBD_ECUDA);
    }
    if (separate) {
        if ((rc = dev_alloc(p, reinterpret_cast<void**>(&p->zt), sizeof(double) * 2 * n_t))) return fail(rc);
        if (cudaMemcpyAsync(p->zt, targets, sizeof(double) * 2 * n_t, cudaMemcpyDefault, s) != cudaSuccess) {
            set_error("sbd_plan_st: copying the targets failed (device pointer expected)");
            cudaGetLastError();
            return fail(SBD_ECUDA);
        }
    }
    // bounding box and delta_max of all the points (targets and sources): every x_k - y_l is
    // then within delta_max (R2)
    double bb[4];
    if ((rc = points_bbox(p->z, p->n, bb, s))) return fail(rc);
    if (separate) {
        double bt[4];
        if ((rc = points_bbox(p->zt, p->n_tgt, bt, s))) return fail(rc);
        bb[0] = std::min(bb[0], bt[0]);
        bb[1] = std::min(bb[1], bt[1]);
        bb[2] = std::max(bb[2], bt[2]);
        bb[3] = std::max(bb[3], bt[3]);
    }
    const double cx = 0.5 * (bb[0] + bb[2]), cy = 0.5 * (bb[1] + bb[3]);
    double md2 = 0.0;
    if ((rc = points_max_dist2(p->z, p->n, cx, cy, &md2, s))) return fail(rc);
    if (separate) {
        double mt2 = 0.0;
        if ((rc = points_max_dist2(p->zt, p->n_tgt, cx, cy, &mt2, s))) return fail(rc);
        md2 = std::max(md2, mt2);
    }
    double delta_max = 2.0 * std::sqrt(md2);
    if (o.delta_max > 0.0) {
        if (o.delta_max < delta_max) {
            set_error("sbd_plan: options.delta_max is below 2 max |z - c| = " + std::to_string(delta_max));
            return fail(SBD_EINVAL);
        }
        delta_max = o.delta_max;
    }
    if (!(delta_min < delta_max)) {
        set_error("sbd_plan: delta_min must be below delta_max = 2 max |z - c|");
        return fail(SBD_EINVAL);
    }
    std::string err;
    rc = radial ? offline_fit_radial(*radial, delta_min, delta_max, eps, o.fixed_P, p->fit, err)
                : offline_fit(kernel.kind, kernel.kappa, delta_min, delta_max, eps, o.fixed_P, p->fit, err);
    if (rc) {
        set_error(err);
        return fail(rc);
    }
    const SbdFit& fit = p->fit;
    p->w0 = fit.w0;
    const double half = std::max(std::max(bb[2] - cx, bb[3] - cy), 1e-300);
    if ((rc = plan_transform_params(fit, o, eps, half, cx, cy, std::max(p->n, p->n_tgt), p->np, err))) {
        set_error(err);
        return fail(rc);
    }
    p->uniform = (o.flags & SBD_FLAG_UNIFORM_GRID) != 0;
    if ((rc = near_tables(fit, p->nt, err, p->uniform))) {
        set_error(err);
        return fail(rc);
    }
    p->fit.radial = RadialKernel{};   // the callbacks are not called after the plan is built
    // near-field device tables
    const NearTables& nt = p->nt;
    if ((rc = upload(p, &p->T1, nt.T1, s))) return fail(rc);
    if ((rc = upload(p, &p->T2, nt.T2, s))) return fail(rc);
    std::vector<double> sxi, sw;
    std::vector<int> sst(1, 0);
    for (int c : nt.small) {
        for (int m = 0; m < fit.M[c]; ++m) {
            const double th = 2.0 * 3.14159265358979323846 * m / fit.M[c];
            sxi.push_back(fit.radius[c] * std::cos(th));
            sxi.push_back(fit.radius[c] * std::sin(th));
        }
        sst.push_back(sst.back() + fit.M[c]);
        sw.push_back(fit.weight[c].real());
        sw.push_back(fit.weight[c].imag());
    }
    if ((rc = upload(p, &p->small_xi, sxi, s))) return fail(rc);
    if ((rc = upload(p, &p->small_w, sw, s))) return fail(rc);
    if ((rc = upload(p, &p->small_start, sst, s))) return fail(rc);
    NearDev nd;
    nd.pieces = nt.pieces;
    nd.deg = nt.deg;
    nd.tmax = nt.tmax;
    nd.in_r = nt.in_r ? 1 : 0;
    nd.T1 = p->T1;
    nd.T2 = p->T2;
    nd.n_small = static_cast<int>(nt.small.size());
    nd.small_xi = p->small_xi;
    nd.small_start = p->small_start;
    nd.small_w = p->small_w;
    nd.self_re = nt.self_value.real();
    nd.self_im = nt.self_value.imag();
    const bool cval = kernel.kind == SBD_HELMHOLTZ;
    rc = o.form == SBD_FORM_FP32 ? build_far<float>(p, s) : build_far<double>(p, s);
    if (rc) return fail(rc);
    // D over the internal orders (the point records' tile order): the points of a row's
    // columns are neighbours in that order too, so D f reads f locally.  Rows are the
    // targets, columns the sources (the same set for a plan of one point set).
    {
        double *zs = nullptr, *zq = nullptr;
        SBD_CUDA_TRY(cudaMallocAsync(&zs, sizeof(double) * 2 * p->n, s));
        if ((rc = near_gather(p->z, true, p->n, 1, p->pt_perm, zs, s))) return fail(rc);
        if (separate) {
            SBD_CUDA_TRY(cudaMallocAsync(&zq, sizeof(double) * 2 * p->n_tgt, s));
            if ((rc = near_gather(p->zt, true, p->n_tgt, 1, p->tpt_perm, zq, s))) return fail(rc);
        }
        rc = near_build(zs, p->n, delta_min, bb[0], bb[1], bb[2], bb[3], nd, cval, &p->rowptr, &p->col, &p->val,
                        &p->nnz, &p->n_coinc, s, zq, p->n_tgt);
        cudaFreeAsync(zs, s);
        if (zq) cudaFreeAsync(zq, s);
        if (rc) return fail(rc);
    }
    // D f stays FP64 in both forms (the near correction is where G - G_approx cancels);
    // SBD_FLAG_NEAR_FP32 keeps D and the gathered f in FP32 instead (FP32 form only)
    p->d32 = (o.flags & SBD_FLAG_NEAR_FP32) != 0;
    if (p->d32 && (rc = near_values_to_f32(&p->val, p->nnz, cval, s))) return fail(rc);
    const size_t dvb = (cval ? 2 : 1) * (p->d32 ? sizeof(float) : sizeof(double));
    p->device_bytes += static_cast<long long>(sizeof(long long) * (p->n_tgt + 1) + (sizeof(int) + dvb) * p->nnz);
    if (!separate) p->n_coinc /= 2;   // each coincident pair was met from both of its points
    {
        const size_t vb = (cval ? 16 : 8) * static_cast<size_t>(p->n_tgt) * p->max_nrhs;
        if ((rc = dev_alloc(p, &p->f_int, dvb * static_cast<size_t>(p->n) * p->max_nrhs))) return fail(rc);
        if ((rc = dev_alloc(p, &p->q_int, vb))) return fail(rc);
    }
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(&p->sumf), sizeof(double2) * p->max_nrhs))) return fail(rc);
    if ((rc = dev_alloc(p, reinterpret_cast<void**>(&p->zero2), sizeof(double2)))) return fail(rc);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error(std::string("sbd_plan: ") + cudaGetErrorString(cudaGetLastError()));
        return fail(SBD_ECUDA);
    }
    p->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SBD_OK;
}

}  // namespace

extern "C" {

int sbd_plan(const double* points, int64_t n, sbd_kernel kernel, double delta_min, double eps,
             const sbd_options* opt, void* cuda_stream, sbd_plan_t* out) {
    return plan_impl(nullptr, 0, points, n, kernel, delta_min, eps, opt, cuda_stream, out);
}

int sbd_plan_radial(const double* points, int64_t n, const sbd_radial_kernel* kernel, double delta_min,
                    double eps, const sbd_options* opt, void* cuda_stream, sbd_plan_t* out) {
    if (!kernel) {
        set_error("sbd_plan_radial: null kernel");
        return SBD_EINVAL;
    }
    const RadialKernel rk = radial_of(*kernel);
    sbd_kernel k{};
    k.kind = SBD_RADIAL;
    return plan_impl(nullptr, 0, points, n, k, delta_min, eps, opt, cuda_stream, out, &rk);
}

int sbd_plan_st(const double* targets, int64_t n_targets, const double* sources, int64_t n_sources,
                sbd_kernel kernel, double delta_min, double eps, const sbd_options* opt, void* cuda_stream,
                sbd_plan_t* out) {
    if (!targets) {
        set_error("sbd_plan_st: null targets");
        return SBD_EINVAL;
    }
    return plan_impl(targets, n_targets, sources, n_sources, kernel, delta_min, eps, opt, cuda_stream, out);
}

int sbd_far(sbd_plan_t p, const void* f, void* q, int32_t nrhs, void* cuda_stream) {
    int rc = check_plan_call(p, f, q);
    if (rc) return rc;
    if (nrhs < 1 || nrhs > p->max_nrhs) {
        set_error("nrhs outside [1, max_nrhs]");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return p->form == SBD_FORM_FP32 ? far_apply<float>(p, f, q, nrhs, s, nullptr)
                                    : far_apply<double>(p, f, q, nrhs, s, nullptr);
}

namespace {
// q_int = D f in the internal order (f gathered into f_int first)
int close_internal(sbd_plan_s* p, const void* f, int nrhs, cudaStream_t s) {
    const bool c = p->kind == SBD_HELMHOLTZ;
    int rc = near_gather(f, c, p->n, nrhs, p->pt_perm, p->f_int, s, p->d32);
    if (rc) return rc;
    return near_spmv_internal(p->rowptr, p->col, p->val, c, p->n_tgt, nrhs, p->f_int, p->q_int, s, p->d32);
}
}  // namespace

int sbd_close(sbd_plan_t p, const void* f, void* q, int32_t nrhs, void* cuda_stream) {
    int rc = check_plan_call(p, f, q);
    if (rc) return rc;
    if (nrhs < 1 || nrhs > p->max_nrhs) {
        set_error("nrhs outside [1, max_nrhs]");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if ((rc = close_internal(p, f, nrhs, s))) return rc;
    return near_scatter(p->q_int, p->kind == SBD_HELMHOLTZ, p->n_tgt, nrhs, p->tpt_perm, q, s);
}

int sbd_matvec(sbd_plan_t p, const void* f, void* q, int32_t nrhs, void* cuda_stream) {
    int rc = check_plan_call(p, f, q);
    if (rc) return rc;
    if (nrhs < 1 || nrhs > p->max_nrhs) {
        set_error("nrhs outside [1, max_nrhs]");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (p->profile) {
        // step timing: D f first, alone, then the far part (the interpolation adds D f)
        StepTimer t(p, s, SBD_STAGE_SPMV);
        if ((rc = close_internal(p, f, nrhs, s))) return rc;
        t.end();
        return p->form == SBD_FORM_FP32 ? far_apply<float>(p, f, q, nrhs, s, p->q_int)
                                        : far_apply<double>(p, f, q, nrhs, s, p->q_int);
    }
    // D f (memory-bound) on the near stream while the far part's first steps (bound by
    // arithmetic and shared memory) run on s; s waits for it before the interpolation
    SBD_CUDA_TRY(cudaEventRecord(p->ev_fork, s));
    SBD_CUDA_TRY(cudaStreamWaitEvent(p->near_stream, p->ev_fork, 0));
    if ((rc = close_internal(p, f, nrhs, p->near_stream))) return rc;
    SBD_CUDA_TRY(cudaEventRecord(p->ev_join, p->near_stream));
    return p->form == SBD_FORM_FP32 ? far_apply<float>(p, f, q, nrhs, s, p->q_int, p->ev_join)
                                    : far_apply<double>(p, f, q, nrhs, s, p->q_int, p->ev_join);
}

int sbd_matvec_graph(sbd_plan_t p, const void* f, void* q, int32_t nrhs, void* cuda_stream) {
    int rc = check_plan_call(p, f, q);
    if (rc) return rc;
    if (nrhs < 1 || nrhs > p->max_nrhs) {
        set_error("nrhs outside [1, max_nrhs]");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t esz = p->kind == SBD_HELMHOLTZ ? 16 : 8;
    const size_t bytes = esz * static_cast<size_t>(p->n) * nrhs, out_bytes = esz * static_cast<size_t>(p->n_tgt) * nrhs;
    if (!p->g_stream) {
        SBD_CUDA_TRY(cudaStreamCreateWithFlags(&p->g_stream, cudaStreamNonBlocking));
        SBD_CUDA_TRY(cudaEventCreateWithFlags(&p->g_ev_in, cudaEventDisableTiming));
        SBD_CUDA_TRY(cudaEventCreateWithFlags(&p->g_ev_out, cudaEventDisableTiming));
        p->alloc_stream = p->g_stream;
        if ((rc = dev_alloc(p, &p->g_in, esz * static_cast<size_t>(p->n) * p->max_nrhs)) ||
            (rc = dev_alloc(p, &p->g_out, esz * static_cast<size_t>(p->n_tgt) * p->max_nrhs))) return rc;
        p->g_exec.assign(p->max_nrhs + 1, nullptr);
    }
    cudaStream_t g = p->g_stream;
    // order after the caller's prior work, run on the graph stream, order the caller after it
    SBD_CUDA_TRY(cudaEventRecord(p->g_ev_in, s));
    SBD_CUDA_TRY(cudaStreamWaitEvent(g, p->g_ev_in, 0));
    if (!p->g_exec[nrhs]) {
        // one plain matvec first (creates every table the kernels use), then the capture;
        // step timing stays off while capturing
        SBD_CUDA_TRY(cudaMemsetAsync(p->g_in, 0, bytes, g));
        if ((rc = sbd_matvec(p, p->g_in, p->g_out, nrhs, g))) return rc;
        const bool prof = p->profile;
        p->profile = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e;
        {
            std::shared_lock<std::shared_mutex> lock(capture_mutex());
            SBD_CUDA_TRY(cudaStreamBeginCapture(g, cudaStreamCaptureModeThreadLocal));
            rc = sbd_matvec(p, p->g_in, p->g_out, nrhs, g);
            e = cudaStreamEndCapture(g, &graph);
        }
        p->profile = prof;
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) {
            set_error(std::string("sbd_matvec_graph: capture failed: ") + cudaGetErrorString(e));
            return SBD_ECUDA;
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            set_error(std::string("sbd_matvec_graph: instantiate failed: ") + cudaGetErrorString(ei));
            return SBD_ECUDA;
        }
        p->g_exec[nrhs] = exec;
    }
    SBD_CUDA_TRY(cudaMemcpyAsync(p->g_in, f, bytes, cudaMemcpyDeviceToDevice, g));
    SBD_CUDA_TRY(cudaGraphLaunch(p->g_exec[nrhs], g));
    SBD_CUDA_TRY(cudaMemcpyAsync(q, p->g_out, out_bytes, cudaMemcpyDeviceToDevice, g));
    SBD_CUDA_TRY(cudaEventRecord(p->g_ev_out, g));
    SBD_CUDA_TRY(cudaStreamWaitEvent(s, p->g_ev_out, 0));
    return SBD_OK;
}

int sbd_profile(sbd_plan_t p, int32_t enable) {
    if (!p) {
        set_error("null plan");
        return SBD_EINVAL;
    }
    std::unique_lock<std::shared_mutex> sync_lock(capture_mutex());
    SBD_CUDA_TRY(cudaDeviceSynchronize());
    collect_marks(p);
    for (int i = 0; i < SBD_N_STAGES; ++i) {
        p->stage_ms[i] = 0.0;
        p->stage_count[i] = 0;
    }
    p->profile = enable != 0;
    return SBD_OK;
}

int sbd_profile_read(sbd_plan_t p, double* ms, int64_t* count) {
    if (!p || !ms || !count) {
        set_error("null plan or output");
        return SBD_EINVAL;
    }
    collect_marks(p);
    for (int i = 0; i < SBD_N_STAGES; ++i) {
        ms[i] = p->stage_ms[i];
        count[i] = p->stage_count[i];
    }
    return SBD_OK;
}

int sbd_nufft_minus(sbd_plan_t p, const void* f, void* fhat, void* cuda_stream) {
    int rc = check_plan_call(p, f, fhat);
    if (rc) return rc;
    if (p->uniform) {
        set_error("sbd_nufft_minus: a uniform-grid plan has no quadrature nodes");
        return SBD_ENOTSUP;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return p->form == SBD_FORM_FP32 ? nufft_minus_impl<float>(p, f, fhat, s) : nufft_minus_impl<double>(p, f, fhat, s);
}

int sbd_nufft_plus(sbd_plan_t p, const void* ghat, void* q, void* cuda_stream) {
    int rc = check_plan_call(p, ghat, q);
    if (rc) return rc;
    if (p->uniform) {
        set_error("sbd_nufft_plus: a uniform-grid plan has no quadrature nodes");
        return SBD_ENOTSUP;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return p->form == SBD_FORM_FP32 ? nufft_plus_impl<float>(p, ghat, q, s) : nufft_plus_impl<double>(p, ghat, q, s);
}

int sbd_plan_info(sbd_plan_t p, sbd_plan_stats* o) {
    if (!p || !o) {
        set_error("null plan or output");
        return SBD_EINVAL;
    }
    std::memset(o, 0, sizeof *o);
    o->n_points = p->n;
    o->n_targets = p->n_tgt;
    o->separate_targets = p->separate ? 1 : 0;
    o->uniform_grid = p->uniform ? 1 : 0;
    o->point_chunk = p->pt_chunk;
    o->tuned = p->tuned;
    o->robin = p->fit.robin ? 1 : 0;
    o->P = p->fit.P;
    o->n_circles = p->fit.n_circles;
    o->n_xi = p->fit.n_xi;
    o->nnz = p->nnz;
    o->n_coincident = p->n_coinc;
    o->grid_x = p->np.m;
    o->grid_k = p->np.nk;
    o->fft_n = p->np.n;
    o->stencil_x = p->np.Ps;
    o->stencil_k = p->np.Pk;
    o->form = p->form;
    o->kind = p->kind;
    o->delta_max = p->fit.delta_max;
    o->delta_min = p->fit.delta_min;
    o->scale_R = p->fit.scale_R;
    o->a = p->fit.a;
    o->fit_err = p->fit.fit_err;
    o->nufft_tol = p->np.tol;
    o->w0_re = p->w0.real();
    o->w0_im = p->w0.imag();
    o->device_bytes = p->device_bytes;
    o->plan_seconds = p->plan_seconds;
    o->n_records = p->n_rec;
    o->node_acc = p->tuning.acc;
    o->node_sched = p->tuning.sched;
    o->fft_split = p->fft_split;
    o->node_binned = p->node_binned ? 1 : 0;
    return SBD_OK;
}

int sbd_set_tuning(sbd_plan_t p, int32_t acc, int32_t sched, int32_t fft_split) {
    if (!p || acc < 0 || acc > 4 || sched < 0 || sched > 1 || (acc >= 1 && p->form != SBD_FORM_FP32) ||
        (acc >= 3 && !p->node_binned) || (fft_split != 0 && fft_split != 2)) {
        set_error("sbd_set_tuning: invalid plan or variant");
        return SBD_EINVAL;
    }
    p->tuning.acc = acc;
    p->tuning.sched = sched;
    p->fft_split = fft_split;
    return SBD_OK;
}

}  // extern "C"

namespace {

// Tuning cache: the tuner's choice per plan class, so that plans of the same class (a
// server's repeated geometries, a bench's reruns) skip the timing.  Process-wide, thread safe;
// sbd_tune_cache_save / _load persist it as a JSON object {"key": [acc, sched, fft_split, chunk]}.
struct TuneChoice {
    int acc, sched, fft_split, chunk;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;
long long g_tune_hits = 0, g_tune_misses = 0;

std::string tune_key(const sbd_plan_s* p) {
    // form, kind, separate targets, uniform grid, binned node kernel, float32 near field, the grid
    // sizes and N to a half octave
    const int nclass = static_cast<int>(std::lround(2.0 * std::log2(std::max(1.0, static_cast<double>(p->n)))));
    char buf[160];
    std::snprintf(buf, sizeof buf, "f%d_k%d_s%d_u%d_b%d_d%d_m%d_nk%d_n%d_N%d", p->form, p->kind, p->separate ? 1 : 0,
                  p->uniform ? 1 : 0, p->node_binned ? 1 : 0, p->d32 ? 1 : 0, p->np.m, p->np.nk, p->np.n, nclass);
    return buf;
}

int set_chunk(sbd_plan_s* p, int chunk, cudaStream_t s) {
    p->pt_chunk = chunk;
    int rc = fill_work(p->pt_ts, chunk, &p->pt_work, s);
    if (rc) return rc;
    if (p->separate) return fill_work(p->tpt_ts, chunk, &p->tpt_work, s);
    p->tpt_work = p->pt_work;
    return SBD_OK;
}

// Times spreading plus interpolation (reps launches each, after one warm-up, on a constant
// non-zero f) for every chunk of kPointChunks; keeps the fastest.  ms: kNumPointChunks entries.
template <typename T>
int tune_chunks(sbd_plan_s* p, int reps, double* ms, cudaStream_t s) {
    const bool cplx = p->kind == SBD_HELMHOLTZ;
    const size_t esz = cplx ? 16 : 8;
    void *f = nullptr, *q = nullptr;
    if (cudaMallocAsync(&f, esz * p->n, s) != cudaSuccess || cudaMallocAsync(&q, esz * p->n_tgt, s) != cudaSuccess) {
        cudaGetLastError();
        if (f) cudaFreeAsync(f, s);
        set_error("sbd_tune: cannot allocate the timing vectors");
        return SBD_ENOMEM;
    }
    SBD_CUDA_TRY(cudaMemsetAsync(f, 0x3f, esz * p->n, s));
    SBD_CUDA_TRY(cudaMemsetAsync(p->sumf, 0, sizeof(double2), s));
    cudaEvent_t a = nullptr, b = nullptr;
    SBD_CUDA_TRY(cudaEventCreate(&a));
    SBD_CUDA_TRY(cudaEventCreate(&b));
    auto* X = static_cast<cx_t<T>*>(p->wsX);
    const bool real = p->half_nodes;
    auto pass = [&]() {
        int r = spread_tiled<T>(static_cast<const PointRec<T>*>(p->pts), p->pt_perm, p->pt_work, p->geom, f, cplx, X, s,
                                real, 1, p->n);
        if (!r) r = interp_tiled<T>(static_cast<const PointRec<T>*>(p->tpts), p->tpt_perm, p->tpt_work, p->geom, X,
                                    make_double2(0, 0), p->sumf, q, cplx, s, real, nullptr, 1, 1, p->n_tgt);
        return r;
    };
    double best = 1e300;
    int pick = p->pt_chunk, rc = SBD_OK;
    for (int c = 0; c < kNumPointChunks && !rc; ++c) {
        if ((rc = set_chunk(p, kPointChunks[c], s)) || (rc = pass())) break;
        SBD_CUDA_TRY(cudaEventRecord(a, s));
        for (int r = 0; r < reps && !rc; ++r) rc = pass();
        if (rc) break;
        float t_ms = 0.f;
        SBD_CUDA_TRY(cudaEventRecord(b, s));
        SBD_CUDA_TRY(cudaEventSynchronize(b));
        SBD_CUDA_TRY(cudaEventElapsedTime(&t_ms, a, b));
        const double per = static_cast<double>(t_ms) / reps;
        if (ms) ms[c] = per;
        if (per < best) {
            best = per;
            pick = kPointChunks[c];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(f, s);
    cudaFreeAsync(q, s);
    if (rc) return rc;
    return set_chunk(p, pick, s);
}

// The last step of sbd_tune: the point chunk, then the class's choice into the cache.
int finish_tune(sbd_plan_s* p, int reps, const std::string& key, cudaStream_t s) {
    int rc = p->form == SBD_FORM_FP32 ? tune_chunks<float>(p, reps, nullptr, s) : tune_chunks<double>(p, reps, nullptr, s);
    if (rc) return rc;
    p->tuned = 1;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = TuneChoice{p->tuning.acc, p->tuning.sched, p->fft_split, p->pt_chunk};
    return SBD_OK;
}

}  // namespace

extern "C" {

int sbd_tune_points(sbd_plan_t p, int32_t reps, double* ms, void* cuda_stream) {
    if (!p || reps < 1) {
        set_error("sbd_tune_points: null plan or reps < 1");
        return SBD_EINVAL;
    }
    if (ms)
        for (int c = 0; c < kNumPointChunks; ++c) ms[c] = -1.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return p->form == SBD_FORM_FP32 ? tune_chunks<float>(p, reps, ms, s) : tune_chunks<double>(p, reps, ms, s);
}

int sbd_set_point_chunk(sbd_plan_t p, int32_t chunk) {
    if (!p || chunk < kPointChunks[0] || chunk > (1 << 20)) {
        set_error("sbd_set_point_chunk: null plan or chunk outside [128, 2^20]");
        return SBD_EINVAL;
    }
    return set_chunk(p, chunk, p->alloc_stream);
}

int sbd_tune_cache_stats(int64_t* hits, int64_t* misses, int64_t* entries) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (hits) *hits = g_tune_hits;
    if (misses) *misses = g_tune_misses;
    if (entries) *entries = static_cast<int64_t>(g_tune.size());
    return SBD_OK;
}

int sbd_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
    g_tune_hits = g_tune_misses = 0;
    return SBD_OK;
}

int sbd_tune_cache_save(const char* path) {
    if (!path) {
        set_error("sbd_tune_cache_save: null path");
        return SBD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE* fp = std::fopen(path, "w");
    if (!fp) {
        set_error(std::string("sbd_tune_cache_save: cannot open ") + path);
        return SBD_EINVAL;
    }
    std::fprintf(fp, "{");
    bool first = true;
    for (const auto& kv : g_tune) {
        std::fprintf(fp, "%s\n  \"%s\": [%d, %d, %d, %d]", first ? "" : ",", kv.first.c_str(), kv.second.acc,
                     kv.second.sched, kv.second.fft_split, kv.second.chunk);
        first = false;
    }
    std::fprintf(fp, "\n}\n");
    std::fclose(fp);
    return SBD_OK;
}

int sbd_tune_cache_load(const char* path) {
    if (!path) {
        set_error("sbd_tune_cache_load: null path");
        return SBD_EINVAL;
    }
    FILE* fp = std::fopen(path, "r");
    if (!fp) {
        set_error(std::string("sbd_tune_cache_load: cannot open ") + path);
        return SBD_EINVAL;
    }
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, fp)) > 0) text.append(buf, got);
    std::fclose(fp);
    // a flat object of "key": [acc, sched, fft_split, chunk] entries
    std::map<std::string, TuneChoice> read;
    size_t i = text.find('{');
    if (i == std::string::npos) {
        set_error("sbd_tune_cache_load: not a JSON object");
        return SBD_EINVAL;
    }
    for (;;) {
        const size_t k0 = text.find('"', i + 1);
        if (k0 == std::string::npos) break;
        const size_t k1 = text.find('"', k0 + 1);
        const size_t l0 = text.find('[', k1 == std::string::npos ? k0 : k1);
        const size_t l1 = text.find(']', l0 == std::string::npos ? k0 : l0);
        TuneChoice c{};
        if (k1 == std::string::npos || l0 == std::string::npos || l1 == std::string::npos ||
            std::sscanf(text.c_str() + l0 + 1, "%d , %d , %d , %d", &c.acc, &c.sched, &c.fft_split, &c.chunk) != 4 ||
            c.acc < 0 || c.acc > 4 || c.sched < 0 || c.sched > 1 || (c.fft_split != 0 && c.fft_split != 2) ||
            c.chunk < kPointChunks[0] || c.chunk > (1 << 20)) {
            set_error("sbd_tune_cache_load: malformed entry");
            return SBD_EINVAL;
        }
        read[text.substr(k0 + 1, k1 - k0 - 1)] = c;
        i = l1;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : read) g_tune[kv.first] = kv.second;
    return SBD_OK;
}

int sbd_tune(sbd_plan_t p, int32_t reps, double* ms, void* cuda_stream) {
    if (!p || reps < 1) {
        set_error("sbd_tune: null plan or reps < 1");
        return SBD_EINVAL;
    }
    if (ms)
        for (int v = 0; v < 12; ++v) ms[v] = -1.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const std::string key = tune_key(p);
    {
        TuneChoice c{};
        bool hit = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                c = it->second;
                hit = true;
                ++g_tune_hits;
            } else {
                ++g_tune_misses;
            }
        }
        if (hit) {   // the class was tuned before: apply its choice without timing
            p->tuning.acc = c.acc;
            p->tuning.sched = c.sched;
            p->fft_split = c.fft_split;
            p->tuned = 2;
            return set_chunk(p, c.chunk, s);
        }
    }
    // row-FFT phases: time the forward transform with split 0 and 2, keep the faster
    {
        cudaEvent_t a, b;
        SBD_CUDA_TRY(cudaEventCreate(&a));
        SBD_CUDA_TRY(cudaEventCreate(&b));
        double best = 1e300;
        int pick = 0, rc = SBD_OK;
        for (int sp : {0, 2}) {
            p->fft_split = sp;
            auto fwd = [&]() {
                if (p->form == SBD_FORM_FP32) {
                    auto* X = static_cast<cx_t<float>*>(p->wsX);
                    auto* B = static_cast<cx_t<float>*>(p->wsB);
                    auto* C = static_cast<cx_t<float>*>(p->wsC);
                    return p->half_nodes ? forward_fft_real<float>(p, X, C, B, s) : forward_fft<float>(p, X, C, B, s);
                }
                auto* X = static_cast<cx_t<double>*>(p->wsX);
                auto* B = static_cast<cx_t<double>*>(p->wsB);
                auto* C = static_cast<cx_t<double>*>(p->wsC);
                return p->half_nodes ? forward_fft_real<double>(p, X, C, B, s) : forward_fft<double>(p, X, C, B, s);
            };
            if ((rc = fwd())) break;
            cudaEventRecord(a, s);
            for (int r = 0; r < reps && !rc; ++r) rc = fwd();
            if (rc) break;
            float t_ms = 0.f;
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&t_ms, a, b);
            const double per = static_cast<double>(t_ms) / reps;
            if (ms) ms[sp == 0 ? 8 : 9] = per;
            if (per < best) {
                best = per;
                pick = sp;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        p->fft_split = pick;
        if (rc) return rc;
    }
    if (!p->node_fused) return finish_tune(p, reps, key, s);
    // non-zero input: with zeros every compare-and-swap would succeed at once, which
    // hides the retries that concurrent adds to one cell cost with real data
    const long cells = static_cast<long>(p->np.nk) * p->np.nk;
    int frc = p->form == SBD_FORM_FP32 ? fill_grid<float>(static_cast<cx_t<float>*>(p->wsB), cells, 1.f, 0.5f, s)
                                       : fill_grid<double>(static_cast<cx_t<double>*>(p->wsB), cells, 1.0, 0.5, s);
    if (frc) return frc;
    cudaEvent_t a, b;
    SBD_CUDA_TRY(cudaEventCreate(&a));
    SBD_CUDA_TRY(cudaEventCreate(&b));
    double best = 1e300;
    NodeTuning pick = p->tuning;
    int rc = SBD_OK;
    const bool fp32 = p->form == SBD_FORM_FP32;
    const int row0 = p->half_nodes ? kx_low<float>(p) : 0;   // as in the matvec
    for (int acc = 0; acc <= (fp32 ? 4 : 0) && !rc; ++acc) {
        if (acc == 2 && node_fused_smem<float>(p->np.Pk, 2) > 227 * 1024) continue;
        if (acc >= 3 && !p->node_binned) continue;
        for (int sched = 0; sched <= 1 && !rc; ++sched) {
            const NodeTuning t{acc, sched, p->tuning.wbound};
            auto step = [&]() {
                return p->form == SBD_FORM_FP32
                           ? node_step_fused<float>(static_cast<const NodeRec<float>*>(p->nodes), p->node_tile_start,
                                                    p->geom, static_cast<const cx_t<float>*>(p->wsB),
                                                    static_cast<cx_t<float>*>(p->wsC), t, s, 1, row0)
                           : node_step_fused<double>(static_cast<const NodeRec<double>*>(p->nodes),
                                                     p->node_tile_start, p->geom,
                                                     static_cast<const cx_t<double>*>(p->wsB),
                                                     static_cast<cx_t<double>*>(p->wsC), t, s, 1, row0);
            };
            if ((rc = step())) break;
            if (cudaEventRecord(a, s) != cudaSuccess) { rc = SBD_ECUDA; break; }
            for (int r = 0; r < reps && !rc; ++r) rc = step();
            if (rc) break;
            float t_ms = 0.f;
            if (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                cudaEventElapsedTime(&t_ms, a, b) != cudaSuccess) {
                set_error("sbd_tune: event timing failed");
                rc = SBD_ECUDA;
                break;
            }
            const double per = static_cast<double>(t_ms) / reps;
            if (ms) ms[acc < 4 ? acc * 2 + sched : 10 + sched] = per;   // 8, 9: the row FFT's phases
            if (per < best) {
                best = per;
                pick = t;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    p->tuning = pick;
    return finish_tune(p, reps, key, s);
}

// delta_min by measurement: Theorem 1 leaves alpha in [0, 1/6] free and the Introduction asks
// that delta_min balance the far and the close parts, whose costs on this device are known only
// by running them.  One plan per candidate, timed on the caller's stream, the fastest kept.
int sbd_plan_balanced(const double* points, int64_t n, sbd_kernel kernel, double eps, const double* alphas,
                      int32_t count, int32_t nrhs, int32_t reps, const sbd_options* opt, void* cuda_stream,
                      sbd_plan_t* out, double* ms, int32_t* chosen) {
    if (!points || !out || !alphas || n < 1 || count < 1 || count > 16 || nrhs < 1 || reps < 1 ||
        !(eps >= 1e-10 && eps <= 0.1)) {
        set_error("sbd_plan_balanced: null pointer, n < 1, count outside [1, 16], nrhs or reps < 1, "
                  "or eps outside [1e-10, 0.1]");
        return SBD_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (!(alphas[i] >= 0.0 && alphas[i] <= 1.0 / 6.0 + 1e-12)) {
            set_error("sbd_plan_balanced: alpha outside [0, 1/6] (Theorem 1)");
            return SBD_EINVAL;
        }
    sbd_options o{};
    o.form = SBD_FORM_FP64;
    if (opt) o = *opt;
    o.max_nrhs = std::max(o.max_nrhs, nrhs);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double bb[4], md2 = 0.0;
    int rc = points_bbox(points, static_cast<long>(n), bb, s);
    if (!rc) rc = points_max_dist2(points, static_cast<long>(n), 0.5 * (bb[0] + bb[2]), 0.5 * (bb[1] + bb[3]), &md2, s);
    if (rc) return rc;
    const double delta_max = std::max(2.0 * std::sqrt(md2), o.delta_max);
    const size_t vbytes = (kernel.kind == SBD_HELMHOLTZ ? 16 : 8) * static_cast<size_t>(n) * nrhs;
    void *f = nullptr, *q = nullptr;
    if (cudaMallocAsync(&f, vbytes, s) != cudaSuccess || cudaMallocAsync(&q, vbytes, s) != cudaSuccess) {
        cudaGetLastError();
        if (f) cudaFreeAsync(f, s);
        set_error("sbd_plan_balanced: cannot allocate the timing vectors");
        return SBD_ENOMEM;
    }
    cudaMemsetAsync(f, 0x3f, vbytes, s);   // every float64 = 4.8e-4: non-zero, finite
    cudaEvent_t ea = nullptr, eb = nullptr;
    cudaEventCreate(&ea);
    cudaEventCreate(&eb);
    if (ms)
        for (int i = 0; i < count; ++i) ms[i] = -1.0;
    sbd_plan_t best = nullptr;
    double best_ms = 1e300;
    int best_i = -1, last_rc = SBD_OK;
    std::string last_err;
    const double lg = std::pow(std::abs(std::log(eps)), 2.0 / 3.0);
    for (int i = 0; i < count; ++i) {
        const double a = lg / std::pow(static_cast<double>(n), 2.0 / 3.0 - alphas[i]);
        const double dmin = a * delta_max;
        if (!(dmin < delta_max)) {
            last_rc = SBD_EINVAL;
            last_err = "sbd_plan_balanced: delta_min reaches delta_max for alpha " + std::to_string(alphas[i]);
            continue;
        }
        sbd_plan_t p = nullptr;
        int r = sbd_plan(points, n, kernel, dmin, eps, &o, cuda_stream, &p);
        if (!r) r = sbd_tune(p, 3, nullptr, cuda_stream);
        if (!r) r = sbd_matvec(p, f, q, nrhs, cuda_stream);
        float t_ms = 0.f;
        if (!r && cudaEventRecord(ea, s) != cudaSuccess) r = SBD_ECUDA;
        for (int k = 0; k < reps && !r; ++k) r = sbd_matvec(p, f, q, nrhs, cuda_stream);
        if (!r && (cudaEventRecord(eb, s) != cudaSuccess || cudaEventSynchronize(eb) != cudaSuccess ||
                   cudaEventElapsedTime(&t_ms, ea, eb) != cudaSuccess)) {
            set_error("sbd_plan_balanced: event timing failed");
            r = SBD_ECUDA;
        }
        if (r) {
            last_rc = r;
            last_err = g_last_error;
            if (p) sbd_destroy_async(p, cuda_stream);
            continue;
        }
        const double per = static_cast<double>(t_ms) / reps;
        if (ms) ms[i] = per;
        if (per < best_ms) {
            if (best) sbd_destroy_async(best, cuda_stream);
            best = p;
            best_ms = per;
            best_i = i;
        } else {
            sbd_destroy_async(p, cuda_stream);
        }
    }
    cudaFreeAsync(f, s);
    cudaFreeAsync(q, s);
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (cudaStreamSynchronize(s) != cudaSuccess && best) {
        set_error(std::string("sbd_plan_balanced: ") + cudaGetErrorString(cudaGetLastError()));
        sbd_destroy(best);
        return SBD_ECUDA;
    }
    if (!best) {
        set_error(last_err);
        return last_rc ? last_rc : SBD_ECUDA;
    }
    *out = best;
    if (chosen) *chosen = best_i;
    return SBD_OK;
}

int sbd_plan_export(sbd_plan_t p, int64_t cap, double* rho, double* alpha, int32_t* M, double* radius,
                    double* weight_re, double* weight_im) {
    if (!p) {
        set_error("null plan");
        return SBD_EINVAL;
    }
    const SbdFit& f = p->fit;
    if (cap < f.n_circles) {
        set_error("capacity below the number of circles");
        return SBD_EINVAL;
    }
    for (int c = 0; c < f.n_circles; ++c) {
        if (rho) rho[c] = c < f.P ? f.rho[c] : 0.0;
        if (alpha) alpha[c] = c < f.P ? f.alpha[c] : 0.0;
        if (M) M[c] = f.M[c];
        if (radius) radius[c] = f.radius[c];
        if (weight_re) weight_re[c] = f.weight[c].real();
        if (weight_im) weight_im[c] = f.weight[c].imag();
    }
    return SBD_OK;
}

int sbd_close_export(sbd_plan_t p, int64_t* rowptr, int32_t* col, double* val) {
    if (!p || !rowptr || !col || !val) {
        set_error("null plan or buffer");
        return SBD_EINVAL;
    }
    std::unique_lock<std::shared_mutex> sync_lock(capture_mutex());
    SBD_CUDA_TRY(cudaDeviceSynchronize());
    // the plan holds D over the internal orders; map rows (targets) and columns (sources) back
    // to the caller's order (row k = internal row inv[k]), diagonal first, then by column
    const long n = p->n, nr = p->n_tgt;
    const size_t vb = p->kind == SBD_HELMHOLTZ ? 16 : 8;
    std::vector<long long> rp(nr + 1);
    std::vector<int> cl(p->nnz), perm(n), tperm(nr);
    std::vector<unsigned char> vl(vb * p->nnz);
    SBD_CUDA_TRY(cudaMemcpy(rp.data(), p->rowptr, sizeof(long long) * (nr + 1), cudaMemcpyDeviceToHost));
    SBD_CUDA_TRY(cudaMemcpy(cl.data(), p->col, sizeof(int) * p->nnz, cudaMemcpyDeviceToHost));
    if (p->d32) {   // stored in FP32: widen
        std::vector<float> v32(vb / 8 * p->nnz);
        SBD_CUDA_TRY(cudaMemcpy(v32.data(), p->val, sizeof(float) * v32.size(), cudaMemcpyDeviceToHost));
        double* vd = reinterpret_cast<double*>(vl.data());
        for (size_t i = 0; i < v32.size(); ++i) vd[i] = v32[i];
    } else {
        SBD_CUDA_TRY(cudaMemcpy(vl.data(), p->val, vb * p->nnz, cudaMemcpyDeviceToHost));
    }
    SBD_CUDA_TRY(cudaMemcpy(perm.data(), p->pt_perm, sizeof(int) * n, cudaMemcpyDeviceToHost));
    SBD_CUDA_TRY(cudaMemcpy(tperm.data(), p->tpt_perm, sizeof(int) * nr, cudaMemcpyDeviceToHost));
    std::vector<long> inv(nr);
    for (long i = 0; i < nr; ++i) inv[tperm[i]] = i;
    rowptr[0] = 0;
    for (long k = 0; k < nr; ++k) rowptr[k + 1] = rowptr[k] + (rp[inv[k] + 1] - rp[inv[k]]);
    const long diag = p->separate ? -1 : 0;   // a plan of one point set puts each row's diagonal first
    std::vector<std::pair<int, long long>> ent;
    for (long k = 0; k < nr; ++k) {
        const long i = inv[k];
        const long kd = diag < 0 ? -1 : k;
        ent.clear();
        for (long long j = rp[i]; j < rp[i + 1]; ++j) ent.emplace_back(perm[cl[j]], j);
        std::sort(ent.begin(), ent.end(), [kd](const std::pair<int, long long>& a, const std::pair<int, long long>& b) {
            if ((a.first == kd) != (b.first == kd)) return a.first == kd;
            return a.first < b.first;
        });
        long long o = rowptr[k];
        for (const auto& e : ent) {
            col[o] = e.first;
            std::memcpy(reinterpret_cast<unsigned char*>(val) + vb * o, vl.data() + vb * e.second, vb);
            ++o;
        }
    }
    return SBD_OK;
}

int sbd_destroy(sbd_plan_t p) {
    free_plan(p, true, nullptr);
    return SBD_OK;
}

int sbd_destroy_async(sbd_plan_t p, void* cuda_stream) {
    free_plan(p, false, static_cast<cudaStream_t>(cuda_stream));
    return SBD_OK;
}

// A batch: one CUDA graph holding the matvecs of several plans, each on its own branch
// (forked from the launch stream with events, joined at the end), so one launch runs
// instances of uneven size side by side on the device.
struct sbd_batch_s {
    cudaGraphExec_t exec = nullptr;
    int count = 0;
};

int sbd_batch_create(const sbd_plan_t* plans, const int32_t* nrhs, int32_t count, const void* const* f,
                     void* const* q, sbd_batch_t* out) {
    if (!plans || !nrhs || !f || !q || !out || count < 1) {
        set_error("sbd_batch_create: null argument or count < 1");
        return SBD_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !f[i] || !q[i] || nrhs[i] < 1 || nrhs[i] > plans[i]->max_nrhs) {
            set_error("sbd_batch_create: invalid entry " + std::to_string(i));
            return SBD_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                set_error("sbd_batch_create: a plan appears twice (its workspace is shared)");
                return SBD_EINVAL;
            }
    }
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> br(count, nullptr);
    std::vector<cudaEvent_t> ev(count + 1, nullptr);
    auto cleanup = [&]() {
        for (cudaStream_t x : br)
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (origin) cudaStreamDestroy(origin);
    };
    int rc = SBD_OK;
    SBD_CUDA_TRY(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
    for (int i = 0; i < count; ++i) {
        if (cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            set_error("sbd_batch_create: stream or event creation failed");
            return SBD_ECUDA;
        }
    }
    if (cudaEventCreateWithFlags(&ev[count], cudaEventDisableTiming) != cudaSuccess) {
        cleanup();
        set_error("sbd_batch_create: event creation failed");
        return SBD_ECUDA;
    }
    // one plain matvec per plan first: creates every table the kernels use
    for (int i = 0; i < count && !rc; ++i) rc = sbd_matvec(plans[i], f[i], q[i], nrhs[i], br[i]);
    for (int i = 0; i < count; ++i) cudaStreamSynchronize(br[i]);
    if (rc) {
        cleanup();
        return rc;
    }
    std::vector<bool> prof(count);
    for (int i = 0; i < count; ++i) {
        prof[i] = plans[i]->profile;
        plans[i]->profile = false;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaSuccess;
    {
        std::shared_lock<std::shared_mutex> lock(capture_mutex());
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaEventRecord(ev[count], origin);
        for (int i = 0; i < count && e == cudaSuccess && !rc; ++i) {
            e = cudaStreamWaitEvent(br[i], ev[count], 0);               // fork
            if (e == cudaSuccess) rc = sbd_matvec(plans[i], f[i], q[i], nrhs[i], br[i]);
            if (e == cudaSuccess && !rc) e = cudaEventRecord(ev[i], br[i]);
            if (e == cudaSuccess && !rc) e = cudaStreamWaitEvent(origin, ev[i], 0);   // join
        }
        const cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
        if (e == cudaSuccess) e = e2;
    }
    for (int i = 0; i < count; ++i) plans[i]->profile = prof[i];
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cleanup();
        if (!rc) {
            set_error(std::string("sbd_batch_create: capture failed: ") + cudaGetErrorString(e));
            rc = SBD_ECUDA;
        }
        return rc;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    cleanup();
    if (e != cudaSuccess) {
        set_error(std::string("sbd_batch_create: instantiate failed: ") + cudaGetErrorString(e));
        return SBD_ECUDA;
    }
    auto* b = new sbd_batch_s();
    b->exec = exec;
    b->count = count;
    *out = b;
    return SBD_OK;
}

int sbd_batch_launch(sbd_batch_t b, void* cuda_stream) {
    if (!b) {
        set_error("sbd_batch_launch: null batch");
        return SBD_EINVAL;
    }
    SBD_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)));
    return SBD_OK;
}

int sbd_batch_destroy(sbd_batch_t b) {
    if (!b) return SBD_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
    return SBD_OK;
}

}  // extern "C"

namespace {

// Bounded device waits (the grid barriers of the batched launches): the limit, the phantom
// arrivals of a fault-injection test, and the process-wide status word they report to (host
// memory mapped into the device's address space, so the host reads it after a sync).
std::mutex g_wait_mu;
double g_wait_limit_s = 2.0;
unsigned g_wait_phantom = 0;
volatile int* g_status = nullptr;   // host view
int* g_status_dev = nullptr;        // device view

int status_word() {
    std::lock_guard<std::mutex> lock(g_wait_mu);
    if (g_status) return SBD_OK;
    void* h = nullptr;
    {
        std::unique_lock<std::shared_mutex> cap(capture_mutex());
        SBD_CUDA_TRY(cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable));
    }
    *static_cast<volatile int*>(h) = SBD_OK;
    void* d = nullptr;
    SBD_CUDA_TRY(cudaHostGetDevicePointer(&d, h, 0));
    g_status_dev = static_cast<int*>(d);
    g_status = static_cast<volatile int*>(h);
    return SBD_OK;
}

int lane_group(int P) { return P <= 8 ? 8 : P <= 16 ? 16 : 32; }

template <typename T>
int batched_impl(const sbd_plan_t* plans, const void* const* f, void* const* q, const int32_t* nrhs, int count,
                 cudaStream_t s) {
    int rc = status_word();
    if (rc) return rc;
    unsigned phantom;
    unsigned long long limit_ns;
    {
        std::lock_guard<std::mutex> lock(g_wait_mu);
        phantom = g_wait_phantom;
        limit_ns = static_cast<unsigned long long>(g_wait_limit_s * 1e9);
    }
    for (int i = 0; i < count; ++i) {
        sbd_plan_s* p = plans[i];
        if (!p->b_stream) {
            SBD_CUDA_TRY(cudaStreamCreateWithFlags(&p->b_stream, cudaStreamNonBlocking));
            SBD_CUDA_TRY(cudaEventCreateWithFlags(&p->b_ev, cudaEventDisableTiming));
        }
    }
    constexpr int kSync = 8;
    BatchSync* sync = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&sync, sizeof(BatchSync) * kSync, s));
    SBD_CUDA_TRY(cudaMemsetAsync(sync, 0, sizeof(BatchSync) * kSync, s));
    int used = 0;
    auto next_sync = [&]() { return sync + std::min(used++, kSync - 1); };
    // near parts on the plans' near streams, the sums of f on s
    for (int i = 0; i < count; ++i) {
        sbd_plan_s* p = plans[i];
        SBD_CUDA_TRY(cudaEventRecord(p->ev_fork, s));
        SBD_CUDA_TRY(cudaStreamWaitEvent(p->near_stream, p->ev_fork, 0));
        if ((rc = close_internal(p, f[i], nrhs[i], p->near_stream))) return rc;
        SBD_CUDA_TRY(cudaEventRecord(p->ev_join, p->near_stream));
        if ((rc = far_sum(f[i], p->kind == SBD_HELMHOLTZ, p->n, nrhs[i], p->sumf, s))) return rc;
    }
    // spreading: one cooperative launch per lane-group class (clear, barrier, work items)
    for (int G : {8, 16, 32}) {
        PointJobs J{};
        for (int i = 0; i < count; ++i) {
            sbd_plan_s* p = plans[i];
            if (lane_group(p->np.Ps) != G || p->pt_work.count <= 0) continue;
            PointJob& jb = J.job[J.count];
            const bool packed = p->half_nodes, cplx = p->kind == SBD_HELMHOLTZ;
            jb.rec = p->pts;
            jb.perm = p->pt_perm;
            jb.work = p->pt_work;
            jb.m = p->np.m;
            jb.ntx = (jb.m + kNodeTile - 1) / kNodeTile;
            jb.P = p->np.Ps;
            jb.win_kind = p->np.swin;
            jb.win_beta = p->np.beta_s;
            jb.win_poly = p->geom.spoly;
            jb.win_poly64 = p->geom.spoly64;
            jb.f = f[i];
            jb.n_pts = p->n;
            jb.grid = p->wsX;
            jb.gstride = static_cast<long>(jb.m) * jb.m / (packed ? 2 : 1);
            jb.clear_elems = 2 * jb.gstride * nrhs[i];
            jb.nrhs = nrhs[i];
            jb.rg = point_rhs_group<T>(jb.P, cplx && !packed, nrhs[i]);
            jb.packed = packed;
            jb.complex_io = cplx;
            J.first[J.count] = J.total;
            J.total += jb.work.count * ((jb.nrhs + jb.rg - 1) / jb.rg);
            ++J.count;
        }
        if (J.count && (rc = spread_batch<T>(J, G, next_sync(), phantom, limit_ns, g_status_dev, s))) return rc;
    }
    // a plan with no point records spreads nothing: its grids are cleared here
    for (int i = 0; i < count; ++i) {
        sbd_plan_s* p = plans[i];
        if (p->pt_work.count <= 0) {
            const long g = static_cast<long>(p->np.m) * p->np.m;
            SBD_CUDA_TRY(cudaMemsetAsync(p->wsX, 0, sizeof(cx_t<T>) * g * nrhs[i], s));
        }
    }
    // forward transforms, each plan on its own stream
    auto fork_join = [&](auto body) -> int {
        cudaEvent_t e = plans[0]->b_ev;   // fork point: recorded on s, then reused as plan 0's join
        SBD_CUDA_TRY(cudaEventRecord(e, s));
        for (int i = 0; i < count; ++i) SBD_CUDA_TRY(cudaStreamWaitEvent(plans[i]->b_stream, e, 0));
        for (int i = 0; i < count; ++i) {
            sbd_plan_s* p = plans[i];
            const int r = body(p, i);
            if (r) return r;
            SBD_CUDA_TRY(cudaEventRecord(p->b_ev, p->b_stream));
        }
        for (int i = 0; i < count; ++i) SBD_CUDA_TRY(cudaStreamWaitEvent(s, plans[i]->b_ev, 0));
        return SBD_OK;
    };
    rc = fork_join([&](sbd_plan_s* p, int i) {
        auto* X = static_cast<cx_t<T>*>(p->wsX);
        auto* B = static_cast<cx_t<T>*>(p->wsB);
        auto* C = static_cast<cx_t<T>*>(p->wsC);
        int r = p->half_nodes ? forward_fft_real<T>(p, X, C, B, p->b_stream, nrhs[i])
                              : forward_fft<T>(p, X, C, B, p->b_stream, nrhs[i]);
        if (!r && p->uniform) {   // the uniform-grid plans' node step: the multiplication, on their stream
            const int nk = p->np.nk;
            r = uniform_multiply<T>(B, p->ucoef, p->kind == SBD_HELMHOLTZ, C, nk, p->half_nodes ? nk / 2 : 0,
                                    nrhs[i], static_cast<long>(nk) * nk, p->b_stream);
        }
        return r;
    });
    if (rc) return rc;
    // node step: one cooperative launch per kernel family; the two-kernel fallback per plan
    for (int fam = 0; fam < 2; ++fam) {   // 0: binned, 1: fused
        NodeJobs J{};
        for (int i = 0; i < count; ++i) {
            sbd_plan_s* p = plans[i];
            const bool binned = sizeof(T) == 4 && p->node_binned && p->tuning.acc >= 3;
            if (p->uniform || !p->node_fused || binned != (fam == 0)) continue;
            NodeJob& jb = J.job[J.count];
            jb.rec = p->nodes;
            jb.tile_start = p->node_tile_start;
            jb.nk = p->np.nk;
            jb.ntx = (jb.nk + kNodeTile - 1) / kNodeTile;
            jb.ntiles = jb.ntx * jb.ntx;
            jb.P = p->np.Pk;
            jb.Ws = node_fused_stride(jb.P);
            jb.win_kind = p->np.kwin;
            jb.win_beta = p->np.beta_k;
            jb.win_poly = p->geom.kpoly;
            jb.win_poly64 = p->geom.kpoly64;
            jb.bins = p->geom.node_bins;
            jb.kin = p->wsB;
            jb.kout = p->wsC;
            jb.kbatch = static_cast<long>(jb.nk) * jb.nk;
            jb.nrhs = nrhs[i];
            J.first[J.count] = J.total;
            J.total += jb.ntiles * nrhs[i];
            ++J.count;
        }
        if (J.count && (rc = node_batch<T>(J, fam == 0, next_sync(), phantom, limit_ns, g_status_dev, s))) return rc;
    }
    for (int i = 0; i < count; ++i) {
        sbd_plan_s* p = plans[i];
        if (!p->node_fused && !p->uniform &&
            (rc = node_step_tiled<T>(static_cast<const NodeRec<T>*>(p->nodes), p->node_tile_start, p->geom,
                                     static_cast<const cx_t<T>*>(p->wsB), static_cast<cx_t<T>*>(p->ghat),
                                     static_cast<cx_t<T>*>(p->wsC), s, nrhs[i]))) return rc;
    }
    // inverse transforms, each plan on its own stream
    rc = fork_join([&](sbd_plan_s* p, int i) {
        auto* X = static_cast<cx_t<T>*>(p->wsX);
        auto* B = static_cast<cx_t<T>*>(p->wsB);
        auto* C = static_cast<cx_t<T>*>(p->wsC);
        return p->half_nodes ? inverse_fft_real<T>(p, C, B, X, p->b_stream, nrhs[i])
                             : inverse_fft<T>(p, C, B, X, p->b_stream, false, nrhs[i]);
    });
    if (rc) return rc;
    for (int i = 0; i < count; ++i) SBD_CUDA_TRY(cudaStreamWaitEvent(s, plans[i]->ev_join, 0));   // D f ready
    // interpolation at every plan's targets (+ xi = 0 term + D f): persistent CTAs per class
    for (int G : {8, 16, 32}) {
        PointJobs J{};
        for (int i = 0; i < count; ++i) {
            sbd_plan_s* p = plans[i];
            if (lane_group(p->np.Ps) != G || p->tpt_work.count <= 0) continue;
            PointJob& jb = J.job[J.count];
            const bool packed = p->half_nodes, cplx = p->kind == SBD_HELMHOLTZ;
            jb.rec = p->tpts;
            jb.perm = p->tpt_perm;
            jb.work = p->tpt_work;
            jb.m = p->np.m;
            jb.ntx = (jb.m + kNodeTile - 1) / kNodeTile;
            jb.P = p->np.Ps;
            jb.win_kind = p->np.swin;
            jb.win_beta = p->np.beta_s;
            jb.win_poly = nullptr;   // FP32: the gather evaluates the window directly, as launch_interp_chunks
            jb.win_poly64 = p->geom.spoly64;
            jb.q = q[i];
            jb.n_pts = p->n_tgt;
            jb.grid = p->wsX;
            jb.gstride = static_cast<long>(jb.m) * jb.m / (packed ? 2 : 1);
            jb.nrhs = nrhs[i];
            jb.rg = point_rhs_group<T>(jb.P, !packed, nrhs[i]);
            jb.packed = packed;
            jb.complex_io = cplx;
            jb.w0 = make_double2(p->w0.real(), p->w0.imag());
            jb.sumf = p->sumf;
            jb.add = p->q_int;
            J.first[J.count] = J.total;
            J.total += jb.work.count * ((jb.nrhs + jb.rg - 1) / jb.rg);
            ++J.count;
        }
        if (J.count && (rc = interp_batch<T>(J, G, next_sync(), s))) return rc;
    }
    SBD_CUDA_TRY(cudaFreeAsync(sync, s));
    return SBD_OK;
}

}  // namespace

extern "C" {

int sbd_matvec_batched(const sbd_plan_t* plans, const void* const* f, void* const* q, const int32_t* nrhs,
                       int32_t count, void* cuda_stream) {
    if (!plans || !f || !q || !nrhs || count < 1 || count > kMaxBatch) {
        set_error("sbd_matvec_batched: null argument or count outside [1, " + std::to_string(kMaxBatch) + "]");
        return SBD_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !f[i] || !q[i] || nrhs[i] < 1 || nrhs[i] > plans[i]->max_nrhs) {
            set_error("sbd_matvec_batched: invalid entry " + std::to_string(i));
            return SBD_EINVAL;
        }
        if (plans[i]->form != plans[0]->form) {
            set_error("sbd_matvec_batched: the plans of one call must share the form");
            return SBD_ENOTSUP;
        }
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                set_error("sbd_matvec_batched: a plan appears twice (its workspace is shared)");
                return SBD_EINVAL;
            }
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return plans[0]->form == SBD_FORM_FP32 ? batched_impl<float>(plans, f, q, nrhs, count, s)
                                           : batched_impl<double>(plans, f, q, nrhs, count, s);
}

int sbd_set_device_wait(double limit_seconds, int32_t phantom_arrivals) {
    if (!(limit_seconds > 0) || limit_seconds > 600 || phantom_arrivals < 0 || phantom_arrivals > 1024) {
        set_error("sbd_set_device_wait: limit outside (0, 600] s or phantom arrivals outside [0, 1024]");
        return SBD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_wait_mu);
    g_wait_limit_s = limit_seconds;
    g_wait_phantom = static_cast<unsigned>(phantom_arrivals);
    return SBD_OK;
}

int sbd_device_status(void* cuda_stream) {
    SBD_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    std::lock_guard<std::mutex> lock(g_wait_mu);
    if (!g_status) return SBD_OK;
    const int v = *g_status;
    *g_status = SBD_OK;
    if (v != SBD_OK) set_error("a bounded device wait of a batched launch ran out");
    return v;
}

int sbd_fft2(const void* in, void* out, int32_t n0, int32_t n1, int32_t sign, int32_t form, void* cuda_stream) {
    if (!in || !out || n0 < 2 || n1 < 2 || n0 > 65536 || n1 > 65536 || (sign != 1 && sign != -1) ||
        (form != SBD_FORM_FP32 && form != SBD_FORM_FP64)) {
        set_error("sbd_fft2: invalid argument");
        return SBD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t esz = form == SBD_FORM_FP32 ? 8 : 16;
    void* tmp = nullptr;
    SBD_CUDA_TRY(cudaMallocAsync(&tmp, esz * static_cast<size_t>(n0) * n1, s));
    int rc;
    if (form == SBD_FORM_FP32) {
        auto* I = static_cast<const float2*>(in);
        auto* O = static_cast<float2*>(out);
        auto* Tm = static_cast<float2*>(tmp);
        if (!(rc = fft_rows<float>(I, n1, n1, 0, Tm, n1, n1, 0, n0, n1, sign, nullptr, nullptr, nullptr, nullptr, s)) &&
            !(rc = transpose<float>(Tm, n1, 0, O, n0, 0, n0, n1, 1, s)) &&
            !(rc = fft_rows<float>(O, n0, n0, 0, Tm, n0, n0, 0, n1, n0, sign, nullptr, nullptr, nullptr, nullptr, s)))
            rc = transpose<float>(Tm, n0, 0, O, n1, 0, n1, n0, 1, s);
    } else {
        auto* I = static_cast<const double2*>(in);
        auto* O = static_cast<double2*>(out);
        auto* Tm = static_cast<double2*>(tmp);
        if (!(rc = fft_rows<double>(I, n1, n1, 0, Tm, n1, n1, 0, n0, n1, sign, nullptr, nullptr, nullptr, nullptr, s)) &&
            !(rc = transpose<double>(Tm, n1, 0, O, n0, 0, n0, n1, 1, s)) &&
            !(rc = fft_rows<double>(O, n0, n0, 0, Tm, n0, n0, 0, n1, n0, sign, nullptr, nullptr, nullptr, nullptr, s)))
            rc = transpose<double>(Tm, n0, 0, O, n1, 0, n1, n0, 1, s);
    }
    cudaFreeAsync(tmp, s);
    return rc;
}

}  // extern "C"
