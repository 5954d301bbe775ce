// Tiled gather / scatter with separable stencil windows (spreading, node step,
// interpolation); see node.cu.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "far.cuh"
#include "window.cuh"

namespace sbd {

constexpr int kNodeTile = 64;   // grid tile side (cells); must be >= stencil width - 1
constexpr int kBinSide = 8;     // bin side (cells) of the binned node kernel: >= stencil width

// Sort records by the tile of their stencil start on an n x n grid; perm[sorted] =
// original index; tile_start has ceil(n/64)^2 + 1 entries.  Inside a tile of at most
// kTileSortMax records: by original index, or with by_bin by (8 x 8 bin of the stencil
// start, original index).
constexpr int kTileSortMax = 4096;
template <typename Rec>
int tile_sort(const Rec* in, long n_rec, int n, Rec* sorted, int* perm, long long* tile_start, cudaStream_t s,
              bool by_bin = false);

// kout (nk x nk, fully written) = scatter(omega' * gather(kin)); ghat is n_xi scratch.
// nb grids (right-hand sides), nk^2 elements apart, one after the other.
template <typename T>
int node_step_tiled(const NodeRec<T>* nodes, const long long* tile_start, const FarGeom& g,
                    const cx_t<T>* kin, cx_t<T>* ghat, cx_t<T>* kout, cudaStream_t s, int nb = 1);

// Variant of the fused node kernel (see node.cu): acc 0 = two float planes with
// atomicAdd, 1 = one float2 plane with a 64-bit compare-and-swap (FP32 only), 2 = int64
// fixed point (FP32 only), 3 = binned, no atomics in shared memory (FP32 only; records
// sorted by tile_sort with by_bin, every tile within kTileSortMax records, stencil <= 8).
// acc 0-2: sched 0 = records dealt to the lane groups in turn, 1 = one contiguous run per
// group; acc 3: sched 0 = 512 threads per CTA, 1 = 1024.  acc 4: acc 3's bins two per warp,
// one per half-warp, one record per half-warp at a time (see node_binned_body); sched as acc 3.
struct NodeTuning {
    int acc = 0;
    int sched = 0;
    float wbound = 0.f;   // max |omega'| component x P_k^2 (the fixed-point scale bound)
};

// x[i] = re + i im for i < n.
template <typename T>
int fill_grid(cx_t<T>* x, long n, T re, T im, cudaStream_t s);

// The same in one kernel per tile: gather, weight and scatter into a shared accumulator,
// whose overlap band is added atomically into kout (cleared here).  nb grids (right-hand
// sides, nk^2 elements apart) in one launch: blockIdx.y is the right-hand side.
template <typename T>
size_t node_fused_smem(int Pk, int acc = 0);   // dynamic shared memory of the fused kernel
template <typename T>
int node_step_fused(const NodeRec<T>* nodes, const long long* tile_start, const FarGeom& g,
                    const cx_t<T>* kin, cx_t<T>* kout, const NodeTuning& t, cudaStream_t s, int nb = 1,
                    int row0 = 0);

// Work list of the point kernels (spreading, interpolation): item w is the records
// [begin[w], begin[w + 1]) of the 64 x 64 tile tile[w], at most `chunk` of them; the
// records of a tile (sorted by tile_sort) are split into consecutive chunks, so that a tile
// where many points crowd becomes several CTAs instead of one long one.  The chunk is a
// plan parameter chosen by sbd_tune among kPointChunks (default kPointChunk).
constexpr int kPointChunk = 512;
constexpr int kPointChunks[] = {128, 256, 512, 1024, 2048};
constexpr int kNumPointChunks = 5;
struct PointWork {
    const long long* begin;   // count + 1 entries (device)
    const int* tile;          // count entries (device)
    int count;
};
// Host: the chunk list of a tile_start table (ntiles + 1 prefix offsets).
void point_work_list(const std::vector<long long>& tile_start, int chunk, std::vector<long long>& begin,
                     std::vector<int>& tile);

// grid (m x m, fully written) = spreading of f (float64 or complex128, original order).
// packed: real f into a real grid stored as packed row pairs (m / 2 x m complex,
// cell (R, c) = component R & 1 of element (R >> 1, c)).  The grid is cleared, then each
// work item accumulates its chunk in shared memory and adds the cells it reached into the
// grid with global atomics.  nrhs right-hand sides in one launch: f[r * n_pts + l] goes to
// grid r at grid + r m^2; a CTA takes a group of them (window weights evaluated once per
// record for the group).
template <typename T>
int spread_tiled(const PointRec<T>* pts, const int* perm, const PointWork& work, const FarGeom& g,
                 const void* f, bool f_complex, cx_t<T>* grid, cudaStream_t s, bool packed = false, int nrhs = 1,
                 long n_pts = 0);

// q[r * n_pts + perm[i]] = interpolation of grid r (at grid + r m^2) at point i
// + w0 * sumf[r] (float64 or complex128 out) + add[i * add_stride + r] when add is given
// (same type as q, record order), for r < nrhs, in one launch.
template <typename T>
int interp_tiled(const PointRec<T>* pts, const int* perm, const PointWork& work, const FarGeom& g,
                 const cx_t<T>* grid, double2 w0, const double2* sumf, void* q, bool q_complex, cudaStream_t s,
                 bool packed = false, const void* add = nullptr, int add_stride = 1, int nrhs = 1, long n_pts = 0);

// --- batches of instances (sbd_matvec_batched) ------------------------------------------------

constexpr int kMaxBatch = 64;      // instances per batched launch (the job tables ride in kernel parameters)

// Synchronisation word of a batched launch: work-item counter and the generation barrier.
struct BatchSync {
    unsigned items;
    unsigned arrive;
    unsigned gen;
    unsigned pad;
};

// One instance of a batched spreading or interpolation launch.
struct PointJob {
    const void* rec;        // PointRec<T> records of the instance (sources or targets), tile sorted
    const int* perm;        // record -> point index
    PointWork work;         // chunks of the records
    int ntx, m, P, win_kind;
    double win_beta;
    const float4* win_poly; // FP32: the window's polynomial table, or null
    const double* win_poly64; // FP64: the same (the single-plan launches' table, so both give the same sums)
    const void* f;          // spreading: values (float64 / complex128), point l of rhs r at r * n_pts + l
    void* q;                // interpolation: output, same layout
    long n_pts;
    void* grid;             // nrhs grids gstride complex elements apart
    long gstride;
    long clear_elems;       // spreading: T elements of the grids cleared before spreading
    int nrhs, rg;           // right-hand sides and right-hand sides per CTA
    int packed, complex_io; // packed real grid (Laplace); complex values (Helmholtz)
    double2 w0;             // interpolation: weight of the xi = 0 term, its sums sum_l f_l per rhs,
    const double2* sumf;
    const void* add;        // and the near term add[i * nrhs + r] in the record order
};
struct PointJobs {
    int count, total;       // instances, work items of all of them
    int first[kMaxBatch];   // first item of each instance (items: chunk fastest, then rhs group)
    PointJob job[kMaxBatch];
};

// One instance of a batched node-step launch: items are (tile, rhs), tile fastest.
struct NodeJob {
    const void* rec;
    const long long* tile_start;
    int ntx, nk, P, Ws, ntiles, win_kind;
    double win_beta;
    const float4* win_poly; // FP32: the window's polynomial table, or null
    const double* win_poly64; // FP64: the same
    const void* bins;       // binned: the per-tile bin table (BinTable)
    const void* kin;
    void* kout;             // cleared by the launch before the node step
    long kbatch;            // complex elements between the right-hand sides' grids
    int nrhs, pad;
};
struct NodeJobs {
    int count, total;
    int first[kMaxBatch];
    NodeJob job[kMaxBatch];
};

// The job tables travel as kernel parameters (at most 32764 bytes per launch).
static_assert(sizeof(PointJobs) + 64 <= 32764, "point job table too large for kernel parameters");
static_assert(sizeof(NodeJobs) + 64 <= 32764, "node job table too large for kernel parameters");

// Host side of a batched launch.  spread_batch: clears every job's grids and spreads all of
// them in one cooperative launch of persistent CTAs; the barrier between the two phases waits
// at most limit_ns and then writes SBD_ETIMEOUT to *status (phantom: arrivals the barrier
// waits for beyond the launched CTAs, for fault-injection tests; 0 in use).  sync: a
// zeroed BatchSync of this launch.  interp_batch: persistent CTAs over all jobs' items
// (sync zeroed).  node_batch: like spread_batch, clearing every job's output grids before
// the barrier; binned (FP32, every job binned) or the fused kernel with two float planes.
// G (8, 16 or 32): lane group of the point kernels, >= every job's stencil (the caller
// launches one group of jobs per class).
template <typename T>
int spread_batch(const PointJobs& J, int G, BatchSync* sync, unsigned phantom, unsigned long long limit_ns,
                 volatile int* status, cudaStream_t s);
template <typename T>
int interp_batch(const PointJobs& J, int G, BatchSync* sync, cudaStream_t s);
template <typename T>
int node_batch(const NodeJobs& J, bool binned, BatchSync* sync, unsigned phantom, unsigned long long limit_ns,
               volatile int* status, cudaStream_t s);
// Right-hand sides per CTA of the point kernels for stencil width P (complex or packed / real grid).
template <typename T>
int point_rhs_group(int P, bool two_planes, int nrhs);
// Dynamic shared memory of the fused node kernel's stride for stencil P.
int node_fused_stride(int Pk);
// Bin table of one 64 x 64 tile for the binned node kernels (records sorted by the 8 x 8 bin of
// their stencil start): start[k] = first record of bin k relative to the tile's first record
// (start[64] = the tile's record count), order = the 64 bins largest first (ties by bin index).
// Built once per plan (node_bin_tables) instead of by every node-step launch.
constexpr int kNodeBins = (kNodeTile / kBinSide) * (kNodeTile / kBinSide);
struct BinTable {
    unsigned short start[kNodeBins + 1];
    unsigned char order[kNodeBins];
    unsigned char pad[256 - 2 * (kNodeBins + 1) - kNodeBins];
};
static_assert(sizeof(BinTable) == 256, "bin table entry: 16 x 16 bytes");
// One table entry per tile (ntiles = tiles per side squared) from bin-sorted FP32 records.
int node_bin_tables(const NodeRec<float>* rec, const long long* tile_start, int ntiles, BinTable* out,
                    cudaStream_t s);
// Polynomial table of a window for the FP32 stencil kernels (layout: window.cuh), kWinPolyEntries
// entries for a stencil of P <= 16 cells, fitted in FP64.  Returns false (the kernels then
// evaluate the window directly) where P > 16 or where the table, evaluated in FP32 as the kernels
// do, departs from the window by more than max(1.2e-7, tol / 100) at a fraction in (0, 1).
bool window_poly(int kind, double beta, int P, double tol, float4* table);
// The FP64 kernels' table (kWinPolyEntries64 doubles, degree kWinPolyDeg64), accepted where its FP64
// evaluation stays within tol / 4 of the window at fractions in (0, 1); false: evaluated directly.
bool window_poly64(int kind, double beta, int P, double tol, double* table);

}  // namespace sbd
