// Tiled gather / scatter with separable stencil windows on a square grid.
//
// Used for the three stencil operations of the far part (Sec. 1 steps (i)-(iii)):
//   spreading      points -> spreading grid          (scatter, values f)
//   node step      frequency grid -> nodes -> frequency grid
//                  (gather, weight by omega'_p of the node's circle, scatter)
//   interpolation  spreading grid -> points          (gather)
// Records (points or nodes) carry the first cell (cx, cy) of their P x P stencil and
// the fractional position; they are sorted by the 64 x 64 tile holding that cell.
//   gather:  one CTA per tile copies the tile plus a (P-1) halo into shared memory;
//            a group of 16 (or 32) lanes handles one record at a time, lane = stencil
//            column, rows summed in registers, columns reduced by shuffles.
//   scatter: one CTA per output tile accumulates, in shared memory, the clipped
//            stencils of every record whose stencil meets the tile (records of the
//            tile and of the three tiles before it), then stores the tile once.
// No global atomics, and the output grid needs no clearing.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "near.cuh"
#include "node.cuh"
#include "sbd.h"
#include "window.cuh"

namespace sbd {

namespace {

template <typename Rec>
__global__ void tile_count_kernel(const Rec* __restrict__ rec, long n, int ntx, long long* __restrict__ count) {
    const long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const int2 c = rec[i].cell;
    const int t = (c.x / kNodeTile) * ntx + (c.y / kNodeTile);
    atomicAdd(reinterpret_cast<unsigned long long*>(&count[t]), 1ULL);
}

template <typename Rec>
__global__ void tile_scatter_kernel(const Rec* __restrict__ in, long n, int ntx, const long long* __restrict__ start,
                                    int* __restrict__ cursor, Rec* __restrict__ out, int* __restrict__ perm) {
    const long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const Rec r = in[i];
    const int t = (r.cell.x / kNodeTile) * ntx + (r.cell.y / kNodeTile);
    const long long pos = start[t] + atomicAdd(&cursor[t], 1);
    out[pos] = r;
    perm[pos] = static_cast<int>(i);
}

// Deterministic order inside each tile: the records of a tile (in the nondeterministic
// order of the scatter above) sorted by their original index with a bitonic sort in
// shared memory, so that a plan's records, and therefore its FP32 sums, are the same on
// every run, and consecutive records of a tile run along a circle.  BIN puts the key
// (bin of the stencil start, original index) first: the 8 x 8 bins of kBinSide cells,
// row-major in the tile, that the binned node kernel walks.  Tiles with more than
// kTileSortCap records keep the scatter order.
constexpr int kTileSortCap = kTileSortMax;

__device__ __forceinline__ int bin_in_tile(int2 cell) {
    return ((cell.x % kNodeTile) / kBinSide) * (kNodeTile / kBinSide) + (cell.y % kNodeTile) / kBinSide;
}

template <typename Rec, bool BIN>
__global__ void __launch_bounds__(256) tile_order_kernel(const Rec* __restrict__ tmp, const int* __restrict__ tmp_perm,
                                                         const long long* __restrict__ start, Rec* __restrict__ out,
                                                         int* __restrict__ perm) {
    using Key = typename std::conditional<BIN, long long, int>::type;
    __shared__ Key key[kTileSortCap];
    __shared__ short idx[kTileSortCap];
    const long long b = start[blockIdx.x], e = start[blockIdx.x + 1];
    const int c = static_cast<int>(e - b);
    if (c == 0) return;                                   // uniform per block
    if (c > kTileSortCap) {                               // uniform per block
        for (long long i = b + threadIdx.x; i < e; i += blockDim.x) {
            out[i] = tmp[i];
            perm[i] = tmp_perm[i];
        }
        return;
    }
    int L = 1;
    while (L < c) L <<= 1;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        Key k = BIN ? static_cast<Key>(0x7fffffffffffffffLL) : static_cast<Key>(0x7fffffff);
        if (i < c) {
            k = tmp_perm[b + i];
            if constexpr (BIN) k |= static_cast<long long>(bin_in_tile(tmp[b + i].cell)) << 32;
        }
        key[i] = k;
        idx[i] = static_cast<short>(i);
    }
    __syncthreads();
    for (int k = 2; k <= L; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < L; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    if ((key[i] > key[ixj]) == up) {
                        const Key tk = key[i];
                        key[i] = key[ixj];
                        key[ixj] = tk;
                        const short ti = idx[i];
                        idx[i] = idx[ixj];
                        idx[ixj] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        out[b + i] = tmp[b + idx[i]];
        perm[b + i] = static_cast<int>(key[i] & 0x7fffffff);
    }
}

// Stencil weights of the group's lane: w(sub - P/2 + 1 - frac) along both dimensions.
template <typename T>
__device__ __forceinline__ void lane_weights(int sub, int P, const Window<T>& win, T fx, T fy, T& wx, T& wy) {
    wx = 0;
    wy = 0;
    if (sub < P) {
        wx = win(static_cast<T>(sub - P / 2 + 1) - fx);
        wy = win(static_cast<T>(sub - P / 2 + 1) - fy);
    }
}

// The same weights, for the point kernels: in FP32 with a polynomial table (window.cuh), copied
// to shared memory by the caller (tab), each record's weights are two Horner chains on the
// lane's offset instead of the window's square root, division and exponential.
template <typename T>
struct LaneWin {
    Window<T> win;
    int sub, P;
    __device__ __forceinline__ LaneWin(const Window<T>& w, int sub_, int P_, const float4*) : win(w), sub(sub_), P(P_) {}
    __device__ __forceinline__ void operator()(T fx, T fy, T& wx, T& wy) const {
        if constexpr (sizeof(T) == 8) {
            // FP64 table: a Horner chain per axis instead of the FP64 square root, division and exponential
            if (win.poly64 != nullptr) {
                wx = 0;
                wy = 0;
                if (sub < kWinPolyOffsets) poly_weights64(win.poly64, sub, fx, fy, wx, wy);
                return;
            }
        }
        lane_weights<T>(sub, P, win, fx, fy, wx, wy);
    }
};

template <>
struct LaneWin<float> {
    Window<float> win;
    int sub, P;
    const float4* tab;   // shared copy of win.poly, or null
    __device__ __forceinline__ LaneWin(const Window<float>& w, int sub_, int P_, const float4* tab_)
        : win(w), sub(sub_), P(P_), tab(w.poly != nullptr && sub_ < kWinPolyOffsets ? tab_ : nullptr) {}
    __device__ __forceinline__ void operator()(float fx, float fy, float& wx, float& wy) const {
        if (win.poly != nullptr) {
            wx = 0.f;
            wy = 0.f;
            if (tab != nullptr)
                poly_weights(tab[sub], tab[kWinPolyOffsets + sub], tab[2 * kWinPolyOffsets + sub], fx, fy, wx, wy);
        } else {
            lane_weights<float>(sub, P, win, fx, fy, wx, wy);
        }
    }
};

// Shared copy of a window's polynomial table (FP32 kernels; nothing otherwise), made before
// the caller's next __syncthreads.
template <typename T>
__device__ __forceinline__ void copy_poly(const Window<T>& win, float4* tab) {
    if constexpr (sizeof(T) == 4) {
        if (win.poly != nullptr)
            for (int e = threadIdx.x; e < kWinPolyEntries; e += blockDim.x) tab[e] = win.poly[e];
    }
}

// --- value sources / sinks -------------------------------------------------------------------

template <typename T> struct NodeIO {       // node step: gather -> * omega' -> ghat[i]
    cx_t<T>* ghat;
    __device__ __forceinline__ void put(long i, const NodeRec<T>& r, cx_t<T> v) const {
        ghat[i] = cmul(v, r.omega);
    }
};
template <typename T> struct NodeVal {      // node step scatter values
    const cx_t<T>* ghat;
    __device__ __forceinline__ cx_t<T> get(long i) const { return ghat[i]; }
};
template <typename T> struct PointVal {     // spreading values f[r * stride + perm[i]] (float64 or complex128)
    const void* f;
    const int* perm;
    bool fc;
    long stride;          // elements between right-hand sides
    __device__ __forceinline__ cx_t<T> get(long i, int r = 0) const {
        const long j = perm[i] + r * stride;
        if (fc) {
            const double2 v = static_cast<const double2*>(f)[j];
            return mk<T>(static_cast<T>(v.x), static_cast<T>(v.y));
        }
        return mk<T>(static_cast<T>(static_cast<const double*>(f)[j]), static_cast<T>(0));
    }
};
template <typename T> struct PointOut {     // interpolation: q[r][perm[i]] = v + w0 * sumf[r] (+ add)
    void* q;
    const int* perm;
    bool qc;
    double2 w0;
    const double2* sumf;
    const void* add;      // optional FP64 term per record (internal order): add[i * add_stride + add_off + r]
    int add_stride, add_off;
    long stride;          // elements of q between right-hand sides
    __device__ __forceinline__ void put(long i, const PointRec<T>&, cx_t<T> v, int r = 0) const {
        const long j = perm[i] + r * stride;
        const double2 sf = sumf[r];
        double re = static_cast<double>(v.x) + w0.x * sf.x - w0.y * sf.y;
        double im = static_cast<double>(v.y) + w0.x * sf.y + w0.y * sf.x;
        if (add) {
            const long k = i * add_stride + add_off + r;
            if (qc) {
                const double2 a = static_cast<const double2*>(add)[k];
                re += a.x;
                im += a.y;
            } else {
                re += static_cast<const double*>(add)[k];
            }
        }
        if (qc) static_cast<double2*>(q)[j] = make_double2(re, im);
        else static_cast<double*>(q)[j] = re;
    }
};

// --- kernels ----------------------------------------------------------------------------------------

// Real grid stored as packed row pairs: cell (R, c) is component R & 1 of complex
// element (R >> 1, c), i.e. float index ((R >> 1) n + c) 2 + (R & 1).
__device__ __forceinline__ long packed_index(long R, long c, long n) { return ((R >> 1) * n + c) * 2 + (R & 1); }

template <typename T, int G, typename Rec, typename Out, bool PK>
__global__ void __launch_bounds__(256) gather_tiles_kernel(
    const Rec* __restrict__ rec, const long long* __restrict__ tile_start, int ntx, int n, int P, Window<T> win,
    const cx_t<T>* __restrict__ grid, Out out) {
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int tile = blockIdx.x;
    const long long b0 = tile_start[tile], b1 = tile_start[tile + 1];
    if (b0 == b1) return;
    const int ox = (tile / ntx) * kNodeTile, oy = (tile % ntx) * kNodeTile;
    const int W = kNodeTile + P - 1;
    const int rows = min(W, n - ox), cols = min(W, n - oy);
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
        const int r = idx / W, c = idx - r * W;
        C v = mk<T>(0, 0);
        if (r < rows && c < cols) {
            if (PK) v = mk<T>(reinterpret_cast<const T*>(grid)[packed_index(ox + r, oy + c, n)], static_cast<T>(0));
            else v = grid[static_cast<long>(ox + r) * n + oy + c];
        }
        s[idx] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int group = threadIdx.x / G, ngroups = blockDim.x / G;
    for (long long i = b0 + group; i < b1; i += ngroups) {
        const Rec q = rec[i];
        const int rx = q.cell.x - ox, ry = q.cell.y - oy;
        T wx, wy;
        lane_weights<T>(sub, P, win, q.frac.x, q.frac.y, wx, wy);
        T sr = 0, si = 0;
        const C* col = s + static_cast<long>(rx) * W + ry + sub;
        for (int a = 0; a < P; ++a) {
            const T w = __shfl_sync(gmask, wx, a, G);
            if (sub < P) {
                const C v = col[a * W];
                sr += w * v.x;
                si += w * v.y;
            }
        }
        sr *= wy;
        si *= wy;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(gmask, sr, o, G);
            si += __shfl_xor_sync(gmask, si, o, G);
        }
        if (sub == 0) out.put(i, q, mk<T>(sr, si));
    }
}

// (re, im) += (a, b) on a shared-memory float2 with one 64-bit compare-and-swap per
// attempt: sm_103a has no native shared-memory float add (atomicAdd on a shared float
// is itself a compare-and-swap loop), so one loop for both halves halves the loops.
// Lock-free: a failed swap means another thread's succeeded.
__device__ __forceinline__ void shared_add_f2(float2* addr, float a, float b) {
    auto* p = reinterpret_cast<unsigned long long*>(addr);
    unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(p);
    for (;;) {
        const float x = __uint_as_float(static_cast<unsigned>(old)) + a;
        const float y = __uint_as_float(static_cast<unsigned>(old >> 32)) + b;
        const unsigned long long nw =
            (static_cast<unsigned long long>(__float_as_uint(y)) << 32) | __float_as_uint(x);
        const unsigned long long prev = atomicCAS(p, old, nw);
        if (prev == old) return;
        old = prev;
    }
}

// RV: the values are real (Laplace spreading): one accumulator plane and one atomic per
// cell; otherwise re and im interleaved, one atomicAdd each (on this GPU a shared-memory
// float atomicAdd is a compare-and-swap loop; two of them measured faster than one
// 64-bit compare-and-swap of the pair under contention).
template <typename T, int G, typename Rec, typename Val, bool PK, bool RV>
__global__ void __launch_bounds__(256) scatter_tiles_kernel(
    const Rec* __restrict__ rec, const long long* __restrict__ tile_start, int ntx, int n, int P, Window<T> win,
    Val val, cx_t<T>* __restrict__ grid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);          // [kNodeTile][kNodeTile][RV ? 1 : 2]
    constexpr int kC = RV ? 1 : 2;
    const int tile = blockIdx.x;
    const int tx = tile / ntx, ty = tile % ntx;
    const int ox = tx * kNodeTile, oy = ty * kNodeTile;
    for (int idx = threadIdx.x; idx < kC * kNodeTile * kNodeTile; idx += blockDim.x) acc[idx] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int group = threadIdx.x / G, ngroups = blockDim.x / G;
    for (int sx = max(tx - 1, 0); sx <= tx; ++sx) {
        for (int sy = max(ty - 1, 0); sy <= ty; ++sy) {
            const int st = sx * ntx + sy;
            const long long b0 = tile_start[st], b1 = tile_start[st + 1];
            for (long long i = b0 + group; i < b1; i += ngroups) {
                const Rec q = rec[i];
                const int rx = q.cell.x - ox, ry = q.cell.y - oy;   // stencil start relative to this tile
                if (rx + P <= 0 || ry + P <= 0) continue;           // uniform across the group
                T wx, wy;
                lane_weights<T>(sub, P, win, q.frac.x, q.frac.y, wx, wy);
                const cx_t<T> g = val.get(i);
                const int c = ry + sub;
                const bool col_ok = sub < P && c >= 0 && c < kNodeTile;
                const T gr = g.x * wy, gi = g.y * wy;
                for (int a = 0; a < P; ++a) {
                    const T w = __shfl_sync(gmask, wx, a, G);
                    const int r = rx + a;
                    if (col_ok && r >= 0 && r < kNodeTile) {
                        T* cell = acc + kC * (r * kNodeTile + c);
                        atomicAdd(cell, gr * w);
                        if (!RV) atomicAdd(cell + 1, gi * w);
                    }
                }
            }
        }
    }
    __syncthreads();
    const int rows = min(kNodeTile, n - ox), cols = min(kNodeTile, n - oy);
    for (int idx = threadIdx.x; idx < kNodeTile * kNodeTile; idx += blockDim.x) {
        const int r = idx / kNodeTile, c = idx - r * kNodeTile;
        if (r < rows && c < cols) {
            if (PK) reinterpret_cast<T*>(grid)[packed_index(ox + r, oy + c, n)] = acc[kC * idx];
            else grid[static_cast<long>(ox + r) * n + oy + c] = mk<T>(acc[kC * idx], RV ? 0 : acc[kC * idx + 1]);
        }
    }
}

// Interpolation by work item (PointWork): the CTA loads its tile plus the (P-1) halo of the
// grid into shared memory and takes the records of its chunk, a group of G lanes per record
// (lane = stencil column, rows accumulated in registers, columns reduced with shuffles).
// Right-hand sides: a CTA takes rg of them (grids gstride elements apart), whose tiles sit in
// shared memory side by side (kC = 1 plane for a packed real grid, else re / im), so each
// record's window weights are evaluated once for the rg values it produces.  The body serves
// the single-plan kernel (item = blockIdx.x, group = blockIdx.y) and the batched one.
template <typename T, int G, bool PK>
__device__ __forceinline__ void interp_chunk_body(const PointRec<T>* __restrict__ rec, const PointWork& work, int item,
                                                  int ntx, int n, int P, const Window<T>& win,
                                                  const cx_t<T>* __restrict__ grid, const PointOut<T>& out, int nrhs,
                                                  int rg, int grp, long gstride) {
    constexpr int kC = PK ? 1 : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);                    // [rg][W][W][kC]
    const int tile = work.tile[item];
    const long long b0 = work.begin[item], b1 = work.begin[item + 1];
    const int r0 = grp * rg, nr = min(rg, nrhs - r0);
    const int ox = (tile / ntx) * kNodeTile, oy = (tile % ntx) * kNodeTile;
    const int W = kNodeTile + P - 1;
    const int rows = min(W, n - ox), cols = min(W, n - oy);
    for (int rr = 0; rr < nr; ++rr) {
        const cx_t<T>* gr = grid + (r0 + rr) * gstride;
        T* sr = s + static_cast<long>(rr) * kC * W * W;
        for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
            const int r = idx / W, c = idx - r * W;
            if (PK) {
                sr[idx] = r < rows && c < cols ? reinterpret_cast<const T*>(gr)[packed_index(ox + r, oy + c, n)]
                                               : static_cast<T>(0);
            } else {
                const cx_t<T> v = r < rows && c < cols ? gr[static_cast<long>(ox + r) * n + oy + c] : mk<T>(0, 0);
                sr[2 * idx] = v.x;
                sr[2 * idx + 1] = v.y;
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int group = threadIdx.x / G, ngroups = blockDim.x / G;
    const LaneWin<T> lw(win, sub, P, nullptr);
    for (long long i = b0 + group; i < b1; i += ngroups) {
        const PointRec<T> q = rec[i];
        const int rx = q.cell.x - ox, ry = q.cell.y - oy;   // in [0, 64): the record's own tile
        T wx, wy;
        lw(q.frac.x, q.frac.y, wx, wy);
        for (int rr = 0; rr < nr; ++rr) {
            T sr = 0, si = 0;
            const T* col = s + static_cast<long>(rr) * kC * W * W + kC * (static_cast<long>(rx) * W + ry + sub);
            for (int a = 0; a < P; ++a) {
                const T w = __shfl_sync(gmask, wx, a, G);
                if (sub < P) {
                    sr += w * col[kC * a * W];
                    if (!PK) si += w * col[kC * a * W + 1];
                }
            }
            sr *= wy;
            si *= wy;
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(gmask, sr, o, G);
                if (!PK) si += __shfl_xor_sync(gmask, si, o, G);
            }
            if (sub == 0) out.put(i, q, mk<T>(sr, si), r0 + rr);
        }
    }
}

template <typename T, int G, bool PK>
__global__ void __launch_bounds__(256) interp_chunks_kernel(
    const PointRec<T>* __restrict__ rec, PointWork work, int ntx, int n, int P, Window<T> win,
    const cx_t<T>* __restrict__ grid, PointOut<T> out, int nrhs, int rg, long gstride) {
    interp_chunk_body<T, G, PK>(rec, work, blockIdx.x, ntx, n, P, win, grid, out, nrhs, rg, blockIdx.y, gstride);
}

// Spreading by work item (PointWork): the CTA accumulates the stencils of its chunk's records
// into a shared (64 + P - 1)^2 window with shared-memory atomics, then adds every cell it
// reached into the (cleared) grid with global atomics.  RV: real values, one plane.
// Right-hand sides: a CTA takes rg of them (one window each, grids gstride elements apart);
// each record's window weights are evaluated once for its rg values.
template <typename T, int G, bool PK, bool RV>
__device__ __forceinline__ void spread_chunk_body(const PointRec<T>* __restrict__ rec, const PointWork& work,
                                                  int item, int ntx, int n, int P, const Window<T>& win,
                                                  const PointVal<T>& val, cx_t<T>* __restrict__ grid, int nrhs,
                                                  int rg, int grp, long gstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);          // [rg][W][W][RV ? 1 : 2]
    __shared__ float4 wtab[kWinPolyEntries];
    copy_poly(win, wtab);
    constexpr int kC = RV ? 1 : 2;
    const int W = kNodeTile + P - 1;
    const long plane = static_cast<long>(kC) * W * W;
    const int tile = work.tile[item];
    const long long b0 = work.begin[item], b1 = work.begin[item + 1];
    const int r0 = grp * rg, nr = min(rg, nrhs - r0);
    const int ox = (tile / ntx) * kNodeTile, oy = (tile % ntx) * kNodeTile;
    for (long idx = threadIdx.x; idx < nr * plane; idx += blockDim.x) acc[idx] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int group = threadIdx.x / G, ngroups = blockDim.x / G;
    const LaneWin<T> lw(win, sub, P, wtab);
    // each group a contiguous share of the chunk: the records in flight at once lie far apart along
    // the tile's curves, so their shared-memory atomics collide less (0.348 -> 0.337 ms at N = 10^6)
    const long long per = (b1 - b0 + ngroups - 1) / ngroups;
    const long long i0 = b0 + group * per, i1 = min(b1, i0 + per);
    for (long long i = i0; i < i1; ++i) {
        const PointRec<T> q = rec[i];
        const int rx = q.cell.x - ox, ry = q.cell.y - oy;   // in [0, 64): the record's own tile
        T wx, wy;
        lw(q.frac.x, q.frac.y, wx, wy);
        for (int rr = 0; rr < nr; ++rr) {
            const cx_t<T> g = val.get(i, r0 + rr);
            const T gr = g.x * wy, gi = g.y * wy;
            T* cell = acc + rr * plane + kC * (rx * W + ry + sub);
            for (int a = 0; a < P; ++a) {
                const T w = __shfl_sync(gmask, wx, a, G);
                if (sub < P) {
                    atomicAdd(cell + kC * a * W, gr * w);
                    if (!RV) atomicAdd(cell + kC * a * W + 1, gi * w);
                }
            }
        }
    }
    __syncthreads();
    const int rows = min(W, n - ox), cols = min(W, n - oy);
    for (int rr = 0; rr < nr; ++rr) {
        cx_t<T>* gr = grid + (r0 + rr) * gstride;
        const T* ar = acc + rr * plane;
        for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
            const int r = idx / W, c = idx - r * W;
            if (r >= rows || c >= cols) continue;
            const T vr = ar[kC * idx];
            if (PK) {
                if (vr != static_cast<T>(0)) atomicAdd(reinterpret_cast<T*>(gr) + packed_index(ox + r, oy + c, n), vr);
            } else {
                T* g = reinterpret_cast<T*>(gr + static_cast<long>(ox + r) * n + oy + c);
                if (vr != static_cast<T>(0)) atomicAdd(g, vr);
                if (!RV) {
                    const T vi = ar[kC * idx + 1];
                    if (vi != static_cast<T>(0)) atomicAdd(g + 1, vi);
                }
            }
        }
    }
}

template <typename T, int G, bool PK, bool RV>
__global__ void __launch_bounds__(256) spread_chunks_kernel(
    const PointRec<T>* __restrict__ rec, PointWork work, int ntx, int n, int P, Window<T> win, PointVal<T> val,
    cx_t<T>* __restrict__ grid, int nrhs, int rg, long gstride) {
    spread_chunk_body<T, G, PK, RV>(rec, work, blockIdx.x, ntx, n, P, win, val, grid, nrhs, rg, blockIdx.y, gstride);
}

// --- batched point kernels (sbd_matvec_batched): persistent CTAs over the work items of every
// instance of the batch ----------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (every CTA resident), by generation: a CTA reads
// the generation, arrives, and the last of `expected` arrivals opens the next generation.  The
// wait is bounded: past limit_ns the CTA gives up, writes SBD_ETIMEOUT to the status word and
// returns false (its caller then skips the rest of its work and returns).  expected is
// gridDim.x plus any phantom arrivals of a fault-injection test, which then never complete.
__device__ bool grid_barrier(BatchSync* st, unsigned expected, unsigned long long limit_ns, volatile int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &st->gen;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned a = atomicAdd(&st->arrive, 1u);
        ok = 1;
        if (a == expected - 1) {
            st->arrive = 0;
            __threadfence();
            atomicAdd(&st->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g0) {
                if (global_ns() - t0 > limit_ns) {
                    ok = 0;
                    *status = SBD_ETIMEOUT;
                    __threadfence_system();
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Item `it` of the batch: the job whose item range holds it (jobs sorted by first item).
template <typename Jobs>
__device__ __forceinline__ int find_job(const Jobs& J, int it) {
    int j = 0;
    while (j + 1 < J.count && J.first[j + 1] <= it) ++j;
    return j;
}

template <typename T>
__device__ __forceinline__ Window<T> job_window(const PointJob& jb) {
    return Window<T>{jb.win_kind, static_cast<T>(jb.win_beta), static_cast<T>(2.0 / jb.P),
                     sizeof(T) == 4 ? jb.win_poly : nullptr, sizeof(T) == 8 ? jb.win_poly64 : nullptr};
}

// Spreading of the whole batch in one cooperative launch: every CTA first clears its share of
// all the instances' grids, then (after the bounded grid barrier) takes work items (instance,
// chunk, right-hand-side group) from a counter until none are left.
template <typename T, int G>
__global__ void __launch_bounds__(256) spread_batch_kernel(PointJobs J, BatchSync* st, unsigned phantom,
                                                           unsigned long long limit_ns, volatile int* status) {
    for (int j = 0; j < J.count; ++j) {
        const PointJob& jb = J.job[j];
        T* g = static_cast<T*>(jb.grid);
        for (long e = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; e < jb.clear_elems;
             e += static_cast<long>(gridDim.x) * blockDim.x)
            g[e] = static_cast<T>(0);
    }
    if (!grid_barrier(st, gridDim.x + phantom, limit_ns, status)) return;
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = static_cast<int>(atomicAdd(&st->items, 1u));
        __syncthreads();
        const int it = item;
        if (it >= J.total) break;
        const int j = find_job(J, it);
        const PointJob& jb = J.job[j];
        const int local = it - J.first[j];
        const int chunk = local % jb.work.count, grp = local / jb.work.count;
        const Window<T> win = job_window<T>(jb);
        const PointVal<T> val{jb.f, jb.perm, jb.complex_io != 0 && jb.packed == 0, jb.n_pts};
        const auto* rec = static_cast<const PointRec<T>*>(jb.rec);
        auto* grid = static_cast<cx_t<T>*>(jb.grid);
        if (jb.packed)
            spread_chunk_body<T, G, true, true>(rec, jb.work, chunk, jb.ntx, jb.m, jb.P, win, val, grid, jb.nrhs,
                                                jb.rg, grp, jb.gstride);
        else if (!jb.complex_io)
            spread_chunk_body<T, G, false, true>(rec, jb.work, chunk, jb.ntx, jb.m, jb.P, win, val, grid, jb.nrhs,
                                                 jb.rg, grp, jb.gstride);
        else
            spread_chunk_body<T, G, false, false>(rec, jb.work, chunk, jb.ntx, jb.m, jb.P, win, val, grid, jb.nrhs,
                                                  jb.rg, grp, jb.gstride);
    }
}

// Interpolation of the whole batch: persistent CTAs take work items from a counter.
template <typename T, int G>
__global__ void __launch_bounds__(256) interp_batch_kernel(PointJobs J, BatchSync* st) {
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = static_cast<int>(atomicAdd(&st->items, 1u));
        __syncthreads();
        const int it = item;
        if (it >= J.total) break;
        const int j = find_job(J, it);
        const PointJob& jb = J.job[j];
        const int local = it - J.first[j];
        const int chunk = local % jb.work.count, grp = local / jb.work.count;
        const Window<T> win = job_window<T>(jb);
        const PointOut<T> out{jb.q, jb.perm, jb.complex_io != 0, jb.w0, jb.sumf, jb.add, jb.nrhs, 0, jb.n_pts};
        const auto* rec = static_cast<const PointRec<T>*>(jb.rec);
        const auto* grid = static_cast<const cx_t<T>*>(jb.grid);
        if (jb.packed)
            interp_chunk_body<T, G, true>(rec, jb.work, chunk, jb.ntx, jb.m, jb.P, win, grid, out, jb.nrhs, jb.rg,
                                          grp, jb.gstride);
        else
            interp_chunk_body<T, G, false>(rec, jb.work, chunk, jb.ntx, jb.m, jb.P, win, grid, out, jb.nrhs, jb.rg,
                                           grp, jb.gstride);
    }
}

// Threads of a fused node-step CTA: 16 warps, so that the two CTAs that fit an SM's
// shared memory (FP32 form) keep 32 warps in flight for the shared-memory latency.
constexpr int kNodeThreads = 512;

// Fused node step: one CTA per 64 x 64 tile of the frequency grid.  The tile plus a
// (P-1) halo of K sits in shared memory with an accumulator of the same size
// (interleaved float2 in FP32, two planes re / im in FP64).  A group of G lanes (G = 8, 16 or 32 >= P; 32 / G nodes per warp) takes
// one node at a time, lane = stencil column: rows are accumulated in registers and the
// columns reduced with shuffles (gather), the value is weighted by the node's omega'
// and added back with shared atomics (scatter), with the weights computed once.  The
// next record is loaded while the current one is processed.  Cells that only this
// tile's stencils reach (local rows and columns in [P-1, 64)) are stored, the overlap
// band is added atomically into kout, which the caller clears.
//
// Variants (chosen per plan by sbd_tune): ACC = 0 accumulates re and im in two float
// planes with one atomicAdd each, ACC = 1 (FP32 only) in one float2 plane with one
// 64-bit compare-and-swap; SCHED = 0 deals the tile's records to the lane groups in
// turn, SCHED = 1 gives each group one contiguous run of records (the groups of a warp
// then work on records far apart in the sorted order, which collide less).
//
// ACC = 2 (FP32 only): fixed-point accumulation in two int64 planes with native integer
// atomics.  Every contribution g w_a w_b is at most max|K tile| wbound =: B in
// each component (window values <= 1), so scaling by 2^e with B 2^e <= 2^50 leaves room
// for 2^13 contributions of the largest possible size per cell; the quantum is 2^-50 B,
// far below FP32 rounding.  wbound = 2 max|omega'| P^2 (the 2 of the complex product),
// taken from the plan's records, whose weights include the spreading deconvolution.
template <typename T, int G, int NT, int ACC, int SCHED>
__device__ __forceinline__ void node_fused_body(
    const NodeRec<T>* __restrict__ rec, const long long* __restrict__ tile_start, int ntx, int n, int P, int Ws,
    const Window<T>& win, const cx_t<T>* __restrict__ kin, cx_t<T>* __restrict__ kout, float wbound, int tile) {
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[NT / 32];
    __shared__ float4 wtab[kWinPolyEntries];
    const long long b0 = tile_start[tile], b1 = tile_start[tile + 1];
    if (b0 == b1) return;
    copy_poly(win, wtab);
    const int W = kNodeTile + P - 1;
    constexpr bool kF2 = sizeof(T) == 4 && ACC == 1;
    constexpr bool kI64 = sizeof(T) == 4 && ACC == 2;
    C* s = reinterpret_cast<C*>(smem_raw);
    T* acc_re = reinterpret_cast<T*>(s + W * Ws);
    T* acc_im = acc_re + W * Ws;
    float2* acc2 = reinterpret_cast<float2*>(s + W * Ws);
    unsigned long long* acc64_re = reinterpret_cast<unsigned long long*>(s + W * Ws);
    unsigned long long* acc64_im = acc64_re + W * Ws;
    const int ox = (tile / ntx) * kNodeTile, oy = (tile % ntx) * kNodeTile;
    const int rows = min(W, n - ox), cols = min(W, n - oy);
    float kmax = 0.f;
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
        const int r = idx / W, c = idx - r * W;
        C v = mk<T>(0, 0);
        if (r < rows && c < cols) v = kin[static_cast<long>(ox + r) * n + oy + c];
        s[r * Ws + c] = v;
        if constexpr (kF2) {
            acc2[r * Ws + c] = make_float2(0.f, 0.f);
        } else if constexpr (kI64) {
            acc64_re[r * Ws + c] = 0ull;
            acc64_im[r * Ws + c] = 0ull;
            kmax = fmaxf(kmax, fmaxf(fabsf(static_cast<float>(v.x)), fabsf(static_cast<float>(v.y))));
        } else {
            acc_re[r * Ws + c] = 0;
            acc_im[r * Ws + c] = 0;
        }
    }
    float up = 1.f;
    double down = 1.0;
    if constexpr (kI64) {
        for (int o = 16; o > 0; o >>= 1) kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = kmax;
        __syncthreads();
        kmax = 0.f;
        for (int w = 0; w < NT / 32; ++w) kmax = fmaxf(kmax, red[w]);
        const float B = kmax * wbound;
        int e = 0;
        if (B > 0.f) {
            int ex;
            frexpf(B, &ex);                      // B < 2^ex
            e = min(120, max(-120, 50 - ex));
        }
        up = ldexpf(1.f, e);
        down = ldexp(1.0, -e);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - sub));
    const int group = threadIdx.x / G, ngroups = NT / G;
    long long i, iend, istep;
    if (SCHED == 0) {
        i = b0 + group;
        iend = b1;
        istep = ngroups;
    } else {
        const long long len = (b1 - b0 + ngroups - 1) / ngroups;
        i = b0 + group * len;
        iend = min(b1, i + len);
        istep = 1;
    }
    const LaneWin<T> lw(win, sub, P, wtab);
    NodeRec<T> nxt;
    if (i < iend) nxt = rec[i];
    for (; i < iend; i += istep) {
        const NodeRec<T> q = nxt;
        if (i + istep < iend) nxt = rec[i + istep];          // prefetch
        const int rx = q.cell.x - ox, ry = q.cell.y - oy;
        T wx, wy;
        lw(q.frac.x, q.frac.y, wx, wy);
        const int base = rx * Ws + ry + sub;
        T sr = 0, si = 0;
#pragma unroll
        for (int a = 0; a < G; ++a) {
            if (a < P) {
                const T w = __shfl_sync(gmask, wx, a, G);
                if (sub < P) {
                    const C v = s[base + a * Ws];
                    sr += w * v.x;
                    si += w * v.y;
                }
            }
        }
        sr *= wy;
        si *= wy;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(gmask, sr, o, G);
            si += __shfl_xor_sync(gmask, si, o, G);
        }
        const C g = cmul(mk<T>(sr, si), q.omega);
        const T gr = g.x * wy, gi = g.y * wy;
#pragma unroll
        for (int a = 0; a < G; ++a) {
            if (a < P) {
                const T w = __shfl_sync(gmask, wx, a, G);
                if (sub < P) {
                    if constexpr (kF2) {
                        shared_add_f2(acc2 + base + a * Ws, gr * w, gi * w);
                    } else if constexpr (kI64) {
                        atomicAdd(acc64_re + base + a * Ws,
                                  static_cast<unsigned long long>(__float2ll_rn(gr * w * up)));
                        atomicAdd(acc64_im + base + a * Ws,
                                  static_cast<unsigned long long>(__float2ll_rn(gi * w * up)));
                    } else {
                        atomicAdd(acc_re + base + a * Ws, gr * w);
                        atomicAdd(acc_im + base + a * Ws, gi * w);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
        const int r = idx / W, c = idx - r * W;
        if (r >= rows || c >= cols) continue;
        T vr, vi;
        if constexpr (kF2) {
            const float2 v = acc2[r * Ws + c];
            vr = v.x;
            vi = v.y;
        } else if constexpr (kI64) {
            vr = static_cast<T>(static_cast<double>(static_cast<long long>(acc64_re[r * Ws + c])) * down);
            vi = static_cast<T>(static_cast<double>(static_cast<long long>(acc64_im[r * Ws + c])) * down);
        } else {
            vr = acc_re[r * Ws + c];
            vi = acc_im[r * Ws + c];
        }
        C* dst = kout + static_cast<long>(ox + r) * n + oy + c;
        if (r >= P - 1 && c >= P - 1 && r < kNodeTile && c < kNodeTile) {
            *dst = mk<T>(vr, vi);
        } else if (vr != 0 || vi != 0) {
            atomicAdd(&dst->x, vr);
            atomicAdd(&dst->y, vi);
        }
    }
}

template <typename T, int G, int NT, int ACC, int SCHED>
__global__ void __launch_bounds__(NT) node_fused_kernel(
    const NodeRec<T>* __restrict__ rec, const long long* __restrict__ tile_start, int ntx, int n, int P, int Ws,
    Window<T> win, const cx_t<T>* __restrict__ kin, cx_t<T>* __restrict__ kout, float wbound, long kbatch) {
    // tile blockIdx.x of right-hand side blockIdx.y
    node_fused_body<T, G, NT, ACC, SCHED>(rec, tile_start, ntx, n, P, Ws, win, kin + blockIdx.y * kbatch,
                                          kout + blockIdx.y * kbatch, wbound, blockIdx.x);
}

// Binned node step (FP32, stencils of at most kBinSide cells): no atomics in shared
// memory.  The records of a tile are sorted by the 8 x 8 bin of their stencil start
// (tile_sort with by_bin); a record of bin (bx, by) writes only cells
// [8 bx, 8 bx + 15) x [8 by, 8 by + 15), so two bins of the same colour
// (bx & 1, by & 1) never write the same cell.  Each colour adds into its own shared
// accumulator; a warp takes whole bins (from a shared counter) and walks a bin's records
// four at a time:
//   window  lanes 8k..8k+7 evaluate w(j - P/2 + 1 - frac) for record k of the four;
//   gather  lane l covers cells (l / 4, l % 4) and (l / 4, l % 4 + 4) of every record's
//           stencil (weights fetched by shuffles), and a butterfly reduce-scatter leaves
//           record k's sum in lanes 8k..8k+7, which multiply it by omega'_k;
//   scatter one record after the other (a warp barrier between them, the stencils of one
//           bin overlap), plain loads and stores into the colour's accumulator.
// Bins go out largest first, which shortens the tail of the tile.
// Every accumulator cell thus receives the records of one bin, in a fixed order, and
// the four colours are summed in a fixed order: the result is the same on every run.
constexpr int kBinW = kNodeTile + kBinSide - 1;                 // 71: rows / cols any stencil reaches
constexpr int kBins = (kNodeTile / kBinSide) * (kNodeTile / kBinSide);

// Shared row stride of the binned kernel (float2 units): >= kBinW and = 12 (mod 16), so
// that the 4 x 8-word row pieces of one 16-lane phase of a 64-bit access fill the 32
// banks once.
constexpr int kBinWs = 76;
static_assert(kBinWs >= kBinW && kBinWs % 16 == 12, "binned stride");

// HALF (the tuner's acc 4): each half-warp carries records of its own bin, the warp taking two
// bins at a time and walking them in step (the half-warp of the shorter bin idles at its end).
// Lane (rh, c) of a half covers column c of the 8 x 8 stencil in rows {0, 1, 4, 5} + 2 rh, so
// that the two row sets of one access sit 2 rows = 152 float2 apart, i.e. in the other 8 of
// the 16 64-bit bank pairs: every 64-bit access of a half-warp is free of bank conflicts for
// any stencil start.  Per record: 4 gather and 8 scatter accesses per lane, 4 shuffles for the
// row weights and 8 for the sum over the half, and no serialisation between the records of a
// quad (the two bins never share a cell: same-colour bins are disjoint, the others write other
// planes).
// Record loop of the binned kernels: the CTA's input tile in s, the four colour accumulators in
// acc (zero on entry), the tile's bin table in tab and next_bin = 0 (all visible to every thread);
// warps take bins from next_bin until none are left.
template <int NT, bool HALF>
__device__ __forceinline__ void binned_records(const NodeRec<float>* __restrict__ rec, long long b0, int cnt,
                                               const BinTable& tab, int& next_bin, int ox, int oy, int P,
                                               const Window<float>& win, const float2* s, float2* acc) {
    constexpr int plane = kBinW * kBinWs;
    const int tid = threadIdx.x;
    const bool poly = win.poly != nullptr;   // window weights from the polynomial table (registers)
    const unsigned full = 0xffffffffu;
    const int lane = tid & 31;
    if constexpr (HALF) {
        const int half = lane >> 4, hl = lane & 15;
        const int cb = hl & 7, rh = hl >> 3;
        const float offw = static_cast<float>(cb - P / 2 + 1);
        float4 pc0 = make_float4(0.f, 0.f, 0.f, 0.f), pc1 = pc0, pc2 = pc0;
        if (poly) {
            pc0 = __ldg(win.poly + cb);
            pc1 = __ldg(win.poly + kWinPolyOffsets + cb);
            pc2 = __ldg(win.poly + 2 * kWinPolyOffsets + cb);
        }
        int rowk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) rowk[k] = (k & 1) + 4 * (k >> 1) + 2 * rh;
        for (;;) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(&next_bin, 2);
            slot = __shfl_sync(full, slot, 0);
            if (slot >= kBins) break;
            const int mine = slot + half;
            const bool has_bin = mine < kBins;
            const int bin = has_bin ? tab.order[mine] : 0;
            float2* ac = acc + (((bin / (kNodeTile / kBinSide)) & 1) * 2 + (bin & 1)) * plane;
            const int e0 = has_bin ? min(static_cast<int>(tab.start[bin]), cnt) : 0;
            const int e1 = has_bin ? min(max(static_cast<int>(tab.start[bin + 1]), e0), cnt) : 0;
            const int len = e1 - e0;
            const int steps = max(len, __shfl_xor_sync(full, len, 16));
            NodeRec<float> nxt;
            if (len > 0) nxt = rec[b0 + e0];
            for (int j = 0; j < steps; ++j) {
                const bool act = j < len;
                int base = 0;
                float wx = 0.f, wy = 0.f;
                float2 om = make_float2(0.f, 0.f);
                if (act) {
                    const NodeRec<float> q = nxt;
                    if (j + 1 < len) nxt = rec[b0 + e0 + j + 1];
                    base = (q.cell.x - ox) * kBinWs + (q.cell.y - oy);
                    if (poly) {
                        poly_weights(pc0, pc1, pc2, q.frac.x, q.frac.y, wx, wy);
                    } else if (cb < P) {
                        wx = win(offw - q.frac.x);
                        wy = win(offw - q.frac.y);
                    }
                    om = q.omega;
                }
                float wr[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) wr[k] = wy * __shfl_sync(full, wx, (half << 4) + rowk[k]);
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 v = s[base + rowk[k] * kBinWs + cb];
                    sr += wr[k] * v.x;
                    si += wr[k] * v.y;
                }
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) {            // the sum over the half-warp
                    sr += __shfl_xor_sync(full, sr, o);
                    si += __shfl_xor_sync(full, si, o);
                }
                const float gr = sr * om.x - si * om.y, gi = sr * om.y + si * om.x;
                if (act) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float2* pc = ac + base + rowk[k] * kBinWs + cb;
                        float2 t = *pc;
                        t.x += gr * wr[k];
                        t.y += gi * wr[k];
                        *pc = t;
                    }
                }
                __syncwarp();
            }
        }
    }
    const int kown = lane >> 3, sub = lane & 7;                     // window lane: record, offset
    const int ca = lane >> 2, cb = lane & 3;                        // cells (ca, cb), (ca, cb + 4)
    const float offw = static_cast<float>(sub - P / 2 + 1);
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float4 pc0 = make_float4(0.f, 0.f, 0.f, 0.f), pc1 = pc0, pc2 = pc0;
    if (poly) {
        pc0 = __ldg(win.poly + sub);
        pc1 = __ldg(win.poly + kWinPolyOffsets + sub);
        pc2 = __ldg(win.poly + 2 * kWinPolyOffsets + sub);
    }
    for (; !HALF;) {
        int slot = 0;
        if (lane == 0) slot = atomicAdd(&next_bin, 1);
        slot = __shfl_sync(full, slot, 0);
        if (slot >= kBins) break;
        const int bin = tab.order[slot];
        float2* ac = acc + (((bin / (kNodeTile / kBinSide)) & 1) * 2 + (bin & 1)) * plane;
        const int e0 = min(static_cast<int>(tab.start[bin]), cnt);
        const int e1 = min(max(static_cast<int>(tab.start[bin + 1]), e0), cnt);
        NodeRec<float> nxt;                                         // record of the next quad
        if (e0 + kown < e1) nxt = rec[b0 + e0 + kown];
        for (int j = e0; j < e1; j += 4) {
            const int jr = j + kown;
            int base = 0;
            float wx = 0.f, wy = 0.f;
            float2 om = make_float2(0.f, 0.f);
            if (jr < e1) {
                const NodeRec<float> q = nxt;
                if (jr + 4 < e1) nxt = rec[b0 + jr + 4];
                base = (q.cell.x - ox) * kBinWs + (q.cell.y - oy);
                if (poly) {
                    poly_weights(pc0, pc1, pc2, q.frac.x, q.frac.y, wx, wy);
                } else if (sub < P) {
                    wx = win(offw - q.frac.x);
                    wy = win(offw - q.frac.y);
                }
                om = q.omega;
            }
            float x[8], w1[4], w2[4];
            int bk[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bk[k] = __shfl_sync(full, base, 8 * k) + ca * kBinWs + cb;
                const float wa = __shfl_sync(full, wx, 8 * k + ca);
                w1[k] = wa * __shfl_sync(full, wy, 8 * k + cb);
                w2[k] = wa * __shfl_sync(full, wy, 8 * k + cb + 4);
                const float2 s1 = s[bk[k]], s2 = s[bk[k] + 4];
                x[2 * k] = w1[k] * s1.x + w2[k] * s2.x;
                x[2 * k + 1] = w1[k] * s1.y + w2[k] * s2.y;
            }
            // reduce-scatter: afterwards lane l holds x[(l >> 2) & 7] summed over the warp,
            // i.e. part (l >> 2) & 1 (re, im) of record (l >> 3)
            float y[4], z[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float send = b4 ? x[i] : x[4 + i], keep = b4 ? x[4 + i] : x[i];
                y[i] = keep + __shfl_xor_sync(full, send, 16);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float send = b3 ? y[i] : y[2 + i], keep = b3 ? y[2 + i] : y[i];
                z[i] = keep + __shfl_xor_sync(full, send, 8);
            }
            float u = (b2 ? z[1] : z[0]) + __shfl_xor_sync(full, b2 ? z[0] : z[1], 4);
            u += __shfl_xor_sync(full, u, 2);
            u += __shfl_xor_sync(full, u, 1);
            const float o = __shfl_xor_sync(full, u, 4);
            const float sr = b2 ? o : u, si = b2 ? u : o;
            const float gr = sr * om.x - si * om.y, gi = sr * om.y + si * om.x;
            const int nl = min(4, e1 - j);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k < nl) {                                       // uniform per warp
                    const float hr = __shfl_sync(full, gr, 8 * k), hi = __shfl_sync(full, gi, 8 * k);
                    float2* p1 = ac + bk[k];
                    float2 t1 = p1[0], t2 = p1[4];
                    t1.x += hr * w1[k];
                    t1.y += hi * w1[k];
                    t2.x += hr * w2[k];
                    t2.y += hi * w2[k];
                    p1[0] = t1;
                    p1[4] = t2;
                    __syncwarp();
                }
            }
        }
    }
}

// Flush of a binned tile: the four planes summed into the tile's window of kout (cells only this
// tile reaches stored, the overlap band added atomically; kout cleared beforehand).  FUSED (the
// persistent kernel): the planes are cleared for the next tile, and the next tile's input
// (kin_next, origin (nox, noy), extent nrows x ncols; kin_next null: none) is loaded into s in
// the same pass, so its loads overlap the flush's stores.
template <int NT, bool FUSED>
__device__ __forceinline__ void binned_flush(float2* acc, float2* __restrict__ kout, int ox, int oy, int rows,
                                             int cols, int n, int P, float2* s = nullptr,
                                             const float2* __restrict__ kin_next = nullptr, int nox = 0,
                                             int noy = 0, int nrows = 0, int ncols = 0) {
    constexpr int plane = kBinW * kBinWs;
    const int W = kNodeTile + P - 1;
    const int span = FUSED ? kBinW : W;
    for (int idx = threadIdx.x; idx < span * span; idx += NT) {
        const int r = idx / span, c = idx - r * span;
        const int o = r * kBinWs + c;
        float2 v = make_float2(0.f, 0.f);
        if (FUSED && kin_next != nullptr && r < nrows && c < ncols)
            v = kin_next[static_cast<long>(nox + r) * n + noy + c];
        if (r < W && c < W) {
            float vr = acc[o].x, vi = acc[o].y;
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                vr += acc[k * plane + o].x;
                vi += acc[k * plane + o].y;
            }
            if (FUSED) {
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k * plane + o] = make_float2(0.f, 0.f);
            }
            if (r < rows && c < cols) {
                float2* dst = kout + static_cast<long>(ox + r) * n + oy + c;
                if (r >= P - 1 && c >= P - 1 && r < kNodeTile && c < kNodeTile) {
                    *dst = make_float2(vr, vi);
                } else if (vr != 0.f || vi != 0.f) {
                    atomicAdd(&dst->x, vr);
                    atomicAdd(&dst->y, vi);
                }
            }
        }
        if (FUSED) s[o] = v;
    }
}

template <int NT, bool HALF = false>
__device__ __forceinline__ void node_binned_body(
    const NodeRec<float>* __restrict__ rec, const long long* __restrict__ tile_start,
    const BinTable* __restrict__ bins, int ntx, int n, int P, const Window<float>& win,
    const float2* __restrict__ kin, float2* __restrict__ kout, int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) BinTable tab;                          // bin starts, bins largest first
    __shared__ int next_bin;
    const long long b0 = tile_start[tile], b1 = tile_start[tile + 1];
    if (b0 == b1) return;                                           // uniform per block
    const int cnt = static_cast<int>(b1 - b0);
    constexpr int plane = kBinW * kBinWs;
    float2* s = reinterpret_cast<float2*>(smem_raw);                 // input tile
    float2* acc = s + plane;                                        // four colour accumulators
    const int ox = (tile / ntx) * kNodeTile, oy = (tile % ntx) * kNodeTile;
    const int W = kNodeTile + P - 1;
    const int rows = min(W, n - ox), cols = min(W, n - oy);
    const int tid = threadIdx.x;
    constexpr int kTabVec = sizeof(BinTable) / sizeof(int4);
    if (tid < kTabVec) reinterpret_cast<int4*>(&tab)[tid] = reinterpret_cast<const int4*>(bins + tile)[tid];
    for (int idx = tid; idx < kBinW * kBinW; idx += NT) {
        const int r = idx / kBinW, c = idx - r * kBinW;
        float2 v = make_float2(0.f, 0.f);
        if (r < rows && c < cols) v = kin[static_cast<long>(ox + r) * n + oy + c];
        const int o = r * kBinWs + c;
        s[o] = v;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k * plane + o] = make_float2(0.f, 0.f);
    }
    if (tid == 0) next_bin = 0;
    __syncthreads();
    binned_records<NT, HALF>(rec, b0, cnt, tab, next_bin, ox, oy, P, win, s, acc);
    __syncthreads();
    binned_flush<NT, false>(acc, kout, ox, oy, rows, cols, n, P);
}

// Persistent binned node step: one CTA per SM walks the items (tile, right-hand side), the tiles
// of the plan's non-empty list (largest first) fastest, taking items blockIdx.x + k gridDim.x; the
// flush of each tile clears the planes and loads the next item's input in the same pass
// (binned_flush), so no CTA starts cold and the next tile's loads overlap this tile's stores.
template <int NT, bool HALF>
__global__ void __launch_bounds__(NT, 1) node_binned_persistent_kernel(
    const NodeRec<float>* __restrict__ rec, const long long* __restrict__ tile_start,
    const BinTable* __restrict__ bins, const int* __restrict__ order, int ntl, int ntx, int n, int P,
    Window<float> win, const float2* __restrict__ kin, float2* __restrict__ kout, long kbatch, int nb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) BinTable tab;
    __shared__ int next_bin;
    constexpr int plane = kBinW * kBinWs;
    constexpr int kTabVec = sizeof(BinTable) / sizeof(int4);
    float2* s = reinterpret_cast<float2*>(smem_raw);                 // input tile
    float2* acc = s + plane;                                        // four colour accumulators
    const int items = ntl * nb;
    int it = blockIdx.x;
    if (it >= items) return;                                        // uniform per block
    const int W = kNodeTile + P - 1;
    const int tid = threadIdx.x;
    // item i: tile order[i mod ntl] of right-hand side i / ntl (grid offset returned)
    auto where = [&](int i, int& tile, int& ox, int& oy, int& rows, int& cols) -> long {
        tile = order[i % ntl];
        ox = (tile / ntx) * kNodeTile;
        oy = (tile % ntx) * kNodeTile;
        rows = min(W, n - ox);
        cols = min(W, n - oy);
        return static_cast<long>(i / ntl) * kbatch;
    };
    int tile, ox, oy, rows, cols;
    long off = where(it, tile, ox, oy, rows, cols);
    for (int idx = tid; idx < 4 * plane; idx += NT) acc[idx] = make_float2(0.f, 0.f);
    for (int idx = tid; idx < kBinW * kBinW; idx += NT) {
        const int r = idx / kBinW, c = idx - r * kBinW;
        float2 v = make_float2(0.f, 0.f);
        if (r < rows && c < cols) v = kin[off + static_cast<long>(ox + r) * n + oy + c];
        s[r * kBinWs + c] = v;
    }
    if (tid < kTabVec) reinterpret_cast<int4*>(&tab)[tid] = reinterpret_cast<const int4*>(bins + tile)[tid];
    if (tid == 0) next_bin = 0;
    __syncthreads();
    for (;;) {
        const long long b0 = tile_start[tile];
        const int cnt = static_cast<int>(tile_start[tile + 1] - b0);
        binned_records<NT, HALF>(rec, b0, cnt, tab, next_bin, ox, oy, P, win, s, acc);
        __syncthreads();
        const int nx = it + static_cast<int>(gridDim.x);
        const bool more = nx < items;                               // uniform per block
        int ntile = 0, nox = 0, noy = 0, nrows = 0, ncols = 0;
        long noff = 0;
        if (more) noff = where(nx, ntile, nox, noy, nrows, ncols);
        binned_flush<NT, true>(acc, kout + off, ox, oy, rows, cols, n, P, s, more ? kin + noff : nullptr, nox, noy,
                               nrows, ncols);
        if (!more) break;
        if (tid < kTabVec) reinterpret_cast<int4*>(&tab)[tid] = reinterpret_cast<const int4*>(bins + ntile)[tid];
        if (tid == 0) next_bin = 0;
        __syncthreads();
        it = nx;
        tile = ntile;
        ox = nox;
        oy = noy;
        rows = nrows;
        cols = ncols;
        off = noff;
    }
}

// Plan time: the bin table of tile blockIdx.x (BinTable).  Bin starts: record i opens the bins
// (bin(i - 1), bin(i)] (records sorted by bin); then C threads rank one bin against 64 / C others
// each, larger bins first and ties by bin index.
__global__ void __launch_bounds__(256) bin_table_kernel(const NodeRec<float>* __restrict__ rec,
                                                        const long long* __restrict__ tile_start,
                                                        BinTable* __restrict__ out) {
    constexpr int NT = 256;
    __shared__ int bstart[kBins + 1];
    __shared__ __align__(16) BinTable tab;
    const int tile = blockIdx.x, tid = threadIdx.x;
    const long long b0 = tile_start[tile];
    const int cnt = static_cast<int>(tile_start[tile + 1] - b0);
    for (int k = tid; k <= kBins; k += NT) bstart[k] = cnt;
    __syncthreads();
    for (int i = tid; i < cnt; i += NT) {
        const int bi = bin_in_tile(rec[b0 + i].cell);
        const int bp = i > 0 ? bin_in_tile(rec[b0 + i - 1].cell) : -1;
        for (int k = bp + 1; k <= bi; ++k) bstart[k] = i;
    }
    __syncthreads();
    constexpr int C = NT / kBins;
    static_assert(C >= 1 && C <= 32 && (C & (C - 1)) == 0, "rank split");
    const int t = tid / C, c = tid % C;
    const int nt = bstart[t + 1] - bstart[t];
    int rank = 0;
#pragma unroll
    for (int u = c * (kBins / C); u < (c + 1) * (kBins / C); ++u) {
        const int nu = bstart[u + 1] - bstart[u];
        rank += (nu > nt || (nu == nt && u < t)) ? 1 : 0;
    }
#pragma unroll
    for (int o = C / 2; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o, C);
    if (c == 0) tab.order[rank] = static_cast<unsigned char>(t);
    for (int k = tid; k <= kBins; k += NT) tab.start[k] = static_cast<unsigned short>(bstart[k]);
    for (int k = tid; k < static_cast<int>(sizeof(tab.pad)); k += NT) tab.pad[k] = 0;
    __syncthreads();
    constexpr int kTabVec = sizeof(BinTable) / sizeof(int4);
    if (tid < kTabVec) reinterpret_cast<int4*>(out + tile)[tid] = reinterpret_cast<const int4*>(&tab)[tid];
}

// Node step of a whole batch (sbd_matvec_batched), one cooperative launch of persistent CTAs:
// each CTA clears its share of every instance's output grids, passes the bounded grid barrier
// (see grid_barrier), then takes items (instance, tile, right-hand side; tile fastest) from a
// counter.  BINNED: every instance runs the binned body (FP32, all binned); otherwise the fused
// body with two float planes and records dealt in turn (ACC 0, SCHED 0), G lanes per record.
template <typename T, int G, bool BINNED>
__global__ void __launch_bounds__(kNodeThreads * (BINNED ? 2 : 1), 1) node_batch_kernel(
    NodeJobs J, BatchSync* st, unsigned phantom, unsigned long long limit_ns, volatile int* status) {
    for (int j = 0; j < J.count; ++j) {
        const NodeJob& jb = J.job[j];
        T* g = static_cast<T*>(jb.kout);
        const long elems = 2 * jb.kbatch * jb.nrhs;
        for (long e = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; e < elems;
             e += static_cast<long>(gridDim.x) * blockDim.x)
            g[e] = static_cast<T>(0);
    }
    if (!grid_barrier(st, gridDim.x + phantom, limit_ns, status)) return;
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = static_cast<int>(atomicAdd(&st->items, 1u));
        __syncthreads();
        const int it = item;
        if (it >= J.total) break;
        const int j = find_job(J, it);
        const NodeJob& jb = J.job[j];
        const int local = it - J.first[j];
        const int tile = local % jb.ntiles, r = local / jb.ntiles;
        const auto* kin = static_cast<const cx_t<T>*>(jb.kin) + r * jb.kbatch;
        auto* kout = static_cast<cx_t<T>*>(jb.kout) + r * jb.kbatch;
        const Window<T> win{jb.win_kind, static_cast<T>(jb.win_beta), static_cast<T>(2.0 / jb.P),
                            sizeof(T) == 4 ? jb.win_poly : nullptr, sizeof(T) == 8 ? jb.win_poly64 : nullptr};
        if constexpr (BINNED) {
            if constexpr (sizeof(T) == 4)
                node_binned_body<2 * kNodeThreads>(static_cast<const NodeRec<float>*>(jb.rec), jb.tile_start,
                                                   static_cast<const BinTable*>(jb.bins), jb.ntx, jb.nk, jb.P,
                                                   win, kin, kout, tile);
        } else {
            node_fused_body<T, G, kNodeThreads, 0, 0>(static_cast<const NodeRec<T>*>(jb.rec), jb.tile_start, jb.ntx,
                                                      jb.nk, jb.P, jb.Ws, win, kin, kout, 0.f, tile);
        }
    }
}

// Shared row stride for the fused node kernel: >= W and congruent to P8 modulo 32.
inline int fused_stride(int W, int P8) {
    int ws = W;
    while (ws % 32 != P8 % 32) ++ws;
    return ws;
}

inline int fused_p8(int P) { return P <= 8 ? 8 : (P <= 16 ? 16 : 32); }

inline int tiles_per_side(int n) { return (n + kNodeTile - 1) / kNodeTile; }

template <typename T>
Window<T> make_window(int kind, double beta, int P, const float4* poly = nullptr, const double* poly64 = nullptr) {
    return Window<T>{kind, static_cast<T>(beta), static_cast<T>(2.0 / P), sizeof(T) == 4 ? poly : nullptr,
                     sizeof(T) == 8 ? poly64 : nullptr};
}

template <typename T, typename Rec, typename Out, bool PK = false>
int launch_gather(const Rec* rec, const long long* tile_start, int n, int P, int kind, double beta,
                  const cx_t<T>* grid, Out out, cudaStream_t s) {
    const Window<T> win = make_window<T>(kind, beta, P);
    const int ntx = tiles_per_side(n);
    const size_t W = kNodeTile + P - 1;
    const size_t smem = W * W * sizeof(cx_t<T>);
    const unsigned nt = static_cast<unsigned>(ntx) * ntx;
    if (P <= 8) {
        auto k = gather_tiles_kernel<T, 8, Rec, Out, PK>;
        SBD_TRY(raise_smem_limit(k, smem));
        k<<<nt, 256, smem, s>>>(rec, tile_start, ntx, n, P, win, grid, out);
    } else if (P <= 16) {
        auto k = gather_tiles_kernel<T, 16, Rec, Out, PK>;
        SBD_TRY(raise_smem_limit(k, smem));
        k<<<nt, 256, smem, s>>>(rec, tile_start, ntx, n, P, win, grid, out);
    } else {
        auto k = gather_tiles_kernel<T, 32, Rec, Out, PK>;
        SBD_TRY(raise_smem_limit(k, smem));
        k<<<nt, 256, smem, s>>>(rec, tile_start, ntx, n, P, win, grid, out);
    }
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T, typename Rec, typename Val, bool PK = false, bool RV = false>
int launch_scatter(const Rec* rec, const long long* tile_start, int n, int P, int kind, double beta, Val val,
                   cx_t<T>* grid, cudaStream_t s) {
    const Window<T> win = make_window<T>(kind, beta, P);
    const int ntx = tiles_per_side(n);
    const size_t smem = (RV ? 1 : 2) * sizeof(T) * kNodeTile * kNodeTile;
    const unsigned nt = static_cast<unsigned>(ntx) * ntx;
    if (P <= 8) {
        auto k = scatter_tiles_kernel<T, 8, Rec, Val, PK, RV>;
        SBD_TRY(raise_smem_limit(k, smem));
        k<<<nt, 256, smem, s>>>(rec, tile_start, ntx, n, P, win, val, grid);
    } else if (P <= 16) {
        auto k = scatter_tiles_kernel<T, 16, Rec, Val, PK, RV>;
        SBD_TRY(raise_smem_limit(k, smem));
        k<<<nt, 256, smem, s>>>(rec, tile_start, ntx, n, P, win, val, grid);
    } else {
        auto k = scatter_tiles_kernel<T, 32, Rec, Val, PK, RV>;
        SBD_TRY(raise_smem_limit(k, smem));
        k<<<nt, 256, smem, s>>>(rec, tile_start, ntx, n, P, win, val, grid);
    }
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

}  // namespace

bool window_poly64(int kind, double beta, int P, double tol, double* table) {
    constexpr int K = kWinPolyDeg64 + 1;
    for (int e = 0; e < kWinPolyEntries64; ++e) table[e] = 0.0;
    if (P < 1 || P > kWinPolyOffsets || !(beta > 0.0) || !(tol > 0.0)) return false;
    const double pi = 3.14159265358979323846;
    auto window = [&](double d) {   // the window of window.cuh, in FP64
        if (kind == kWinGauss) return std::exp(-beta * d * d);
        const double z = d * 2.0 / P, r = 1.0 - z * z;
        return r > 0.0 ? std::exp(-beta * z * z / (1.0 + std::sqrt(r))) : 0.0;
    };
    const double bound = 0.25 * tol;
    for (int j = 0; j < P; ++j) {
        const double off = j - P / 2 + 1;
        double y[K], a[K];
        for (int k = 0; k < K; ++k) y[k] = window(off - 0.5 * (std::cos(pi * (k + 0.5) / K) + 1.0));
        for (int i = 0; i < K; ++i) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += y[k] * std::cos(pi * i * (k + 0.5) / K);
            a[i] = (i == 0 ? 1.0 : 2.0) * acc / K;
        }
        double mono[K] = {}, t0[K] = {}, t1[K] = {}, t2[K];
        t0[0] = 1.0;
        t1[1] = 1.0;
        mono[0] = a[0];
        for (int e = 0; e < K; ++e) mono[e] += a[1] * t1[e];
        for (int i = 2; i < K; ++i) {
            for (int e = 0; e < K; ++e) t2[e] = (e > 0 ? 2.0 * t1[e - 1] : 0.0) - t0[e];
            for (int e = 0; e < K; ++e) {
                mono[e] += a[i] * t2[e];
                t0[e] = t1[e];
                t1[e] = t2[e];
            }
        }
        for (int k = 0; k < K; ++k) table[k * kWinPolyOffsets + j] = mono[kWinPolyDeg64 - k];   // highest first
        for (int t = 0; t < 2048; ++t) {
            const double f = (t + 0.5) / 2048.0, sv = std::fma(2.0, f, -1.0);
            double acc = table[j];
            for (int k = 1; k < K; ++k) acc = std::fma(acc, sv, table[k * kWinPolyOffsets + j]);
            if (std::fabs(acc - window(off - f)) > bound) {
                for (int e = 0; e < kWinPolyEntries64; ++e) table[e] = 0.0;
                return false;
            }
        }
    }
    return true;
}

int node_bin_tables(const NodeRec<float>* rec, const long long* tile_start, int ntiles, BinTable* out,
                    cudaStream_t s) {
    if (ntiles <= 0) return SBD_OK;
    bin_table_kernel<<<ntiles, 256, 0, s>>>(rec, tile_start, out);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

bool window_poly(int kind, double beta, int P, double tol, float4* table) {
    constexpr int K = kWinPolyDeg + 1;
    for (int e = 0; e < kWinPolyEntries; ++e) table[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P < 1 || P > kWinPolyOffsets || !(beta > 0.0)) return false;
    const double pi = 3.14159265358979323846;
    auto window = [&](double d) {   // the window of window.cuh, in FP64
        if (kind == kWinGauss) return std::exp(-beta * d * d);
        const double z = d * 2.0 / P, r = 1.0 - z * z;
        return r > 0.0 ? std::exp(-beta * z * z / (1.0 + std::sqrt(r))) : 0.0;
    };
    const double bound = std::max(1.2e-7, 0.01 * tol);
    for (int j = 0; j < P; ++j) {
        const double off = j - P / 2 + 1;
        // Chebyshev interpolation in s = 2 f - 1 at the K Chebyshev points (first kind)
        double y[K], a[K];
        for (int k = 0; k < K; ++k) y[k] = window(off - 0.5 * (std::cos(pi * (k + 0.5) / K) + 1.0));
        for (int i = 0; i < K; ++i) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += y[k] * std::cos(pi * i * (k + 0.5) / K);
            a[i] = (i == 0 ? 1.0 : 2.0) * acc / K;
        }
        // sum_i a_i T_i(s) in powers of s (T_{i+1} = 2 s T_i - T_{i-1})
        double mono[K] = {}, t0[K] = {}, t1[K] = {}, t2[K];
        t0[0] = 1.0;
        t1[1] = 1.0;
        mono[0] = a[0];
        for (int e = 0; e < K; ++e) mono[e] += a[1] * t1[e];
        for (int i = 2; i < K; ++i) {
            for (int e = 0; e < K; ++e) t2[e] = (e > 0 ? 2.0 * t1[e - 1] : 0.0) - t0[e];
            for (int e = 0; e < K; ++e) {
                mono[e] += a[i] * t2[e];
                t0[e] = t1[e];
                t1[e] = t2[e];
            }
        }
        float c[K];
        for (int k = 0; k < K; ++k) c[k] = static_cast<float>(mono[kWinPolyDeg - k]);   // highest first
        for (int q = 0; q < kWinPolyQuads; ++q)
            table[q * kWinPolyOffsets + j] = make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
        // the kernels' FP32 Horner evaluation against the window
        for (int t = 0; t < 1024; ++t) {
            const float f = (t + 0.5f) / 1024.f;
            const float sv = std::fma(2.f, f, -1.f);
            float acc = c[0];
            for (int k = 1; k < K; ++k) acc = std::fma(acc, sv, c[k]);
            if (std::fabs(static_cast<double>(acc) - window(off - static_cast<double>(f))) > bound) {
                for (int e = 0; e < kWinPolyEntries; ++e) table[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                return false;
            }
        }
    }
    return true;
}

template <typename Rec>
int tile_sort(const Rec* in, long n_rec, int n, Rec* sorted, int* perm, long long* tile_start, cudaStream_t s,
              bool by_bin) {
    const int ntx = tiles_per_side(n);
    const long ntiles = static_cast<long>(ntx) * ntx;
    int* cursor = nullptr;
    SBD_CUDA_TRY(cudaMemsetAsync(tile_start, 0, sizeof(long long) * (ntiles + 1), s));
    SBD_CUDA_TRY(cudaMallocAsync(&cursor, sizeof(int) * ntiles, s));
    SBD_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * ntiles, s));
    const unsigned nb = static_cast<unsigned>((n_rec + 255) / 256);
    if (n_rec > 0) {
        tile_count_kernel<Rec><<<nb, 256, 0, s>>>(in, n_rec, ntx, tile_start);
        SBD_LAUNCH_CHECK();
    }
    long long total = 0;
    int rc = scan_exclusive_i64(tile_start, ntiles + 1, &total, s);
    if (rc) return rc;
    if (n_rec > 0) {
        Rec* tmp = nullptr;
        int* tmp_perm = nullptr;
        SBD_CUDA_TRY(cudaMallocAsync(&tmp, sizeof(Rec) * n_rec, s));
        SBD_CUDA_TRY(cudaMallocAsync(&tmp_perm, sizeof(int) * n_rec, s));
        tile_scatter_kernel<Rec><<<nb, 256, 0, s>>>(in, n_rec, ntx, tile_start, cursor, tmp, tmp_perm);
        SBD_LAUNCH_CHECK();
        if (by_bin)
            tile_order_kernel<Rec, true><<<static_cast<unsigned>(ntiles), 256, 0, s>>>(tmp, tmp_perm, tile_start,
                                                                                       sorted, perm);
        else
            tile_order_kernel<Rec, false><<<static_cast<unsigned>(ntiles), 256, 0, s>>>(tmp, tmp_perm, tile_start,
                                                                                        sorted, perm);
        SBD_LAUNCH_CHECK();
        SBD_CUDA_TRY(cudaFreeAsync(tmp, s));
        SBD_CUDA_TRY(cudaFreeAsync(tmp_perm, s));
    }
    SBD_CUDA_TRY(cudaFreeAsync(cursor, s));
    return SBD_OK;
}

template <typename T>
size_t node_fused_smem(int Pk, int acc) {
    if (acc == 3) return static_cast<size_t>(5) * kBinW * kBinWs * sizeof(float2);
    const int W = kNodeTile + Pk - 1;
    const int Ws = fused_stride(W, fused_p8(Pk));
    const size_t accb = acc == 2 ? 2 * sizeof(unsigned long long) : 2 * sizeof(T);
    return static_cast<size_t>(W) * Ws * (sizeof(cx_t<T>) + accb);
}

template <typename T, int G, int ACC, int SCHED>
int launch_fused(const NodeRec<T>* nodes, const long long* tile_start, dim3 nt, int ntx, const FarGeom& g,
                 int Ws, const Window<T>& win, const cx_t<T>* kin, cx_t<T>* kout, float wbound, long kb,
                 cudaStream_t s) {
    // the int64 planes leave room for one CTA per SM: twice the threads keep the warps
    constexpr int NT = ACC == 2 ? 2 * kNodeThreads : kNodeThreads;
    const size_t smem = node_fused_smem<T>(g.Pk, ACC);
    auto k = node_fused_kernel<T, G, NT, ACC, SCHED>;
    SBD_TRY(raise_smem_limit(k, smem));
    k<<<nt, NT, smem, s>>>(nodes, tile_start, ntx, g.nk, g.Pk, Ws, win, kin, kout, wbound, kb);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T, int G>
int launch_fused_g(const NodeRec<T>* nodes, const long long* tile_start, dim3 nt, int ntx, const FarGeom& g,
                   int Ws, const Window<T>& win, const cx_t<T>* kin, cx_t<T>* kout, const NodeTuning& t, long kb,
                   cudaStream_t s) {
    const float wb = t.wbound;
    if (sizeof(T) == 4 && t.acc == 1) {
        return t.sched ? launch_fused<T, G, 1, 1>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, wb, kb, s)
                       : launch_fused<T, G, 1, 0>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, wb, kb, s);
    }
    if (sizeof(T) == 4 && t.acc == 2) {
        return t.sched ? launch_fused<T, G, 2, 1>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, wb, kb, s)
                       : launch_fused<T, G, 2, 0>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, wb, kb, s);
    }
    return t.sched ? launch_fused<T, G, 0, 1>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, wb, kb, s)
                   : launch_fused<T, G, 0, 0>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, wb, kb, s);
}

namespace {
int sm_count();   // SMs of the current device (defined with the batched launches)
}

template <int NT, bool HALF = false>
int launch_binned(const NodeRec<float>* nodes, const long long* tile_start, dim3 nt, int ntx, const FarGeom& g,
                  const Window<float>& win, const float2* kin, float2* kout, long kb, cudaStream_t s) {
    const size_t smem = node_fused_smem<float>(g.Pk, 3);
    if (g.node_bins == nullptr) {
        set_error("node step: the binned kernel needs the plan's bin table");
        return SBD_EINVAL;
    }
    if (g.node_order == nullptr || g.n_node_tiles <= 0) return SBD_OK;   // no records: kout stays cleared
    auto k = node_binned_persistent_kernel<NT, HALF>;
    SBD_TRY(raise_smem_limit(k, smem));
    const int items = g.n_node_tiles * static_cast<int>(nt.y);
    const int grid = std::max(1, std::min(items, sm_count()));
    k<<<grid, NT, smem, s>>>(nodes, tile_start, static_cast<const BinTable*>(g.node_bins), g.node_order,
                             g.n_node_tiles, ntx, g.nk, g.Pk, win, kin, kout, kb, static_cast<int>(nt.y));
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int node_step_fused(const NodeRec<T>* nodes, const long long* tile_start, const FarGeom& g,
                    const cx_t<T>* kin, cx_t<T>* kout, const NodeTuning& t, cudaStream_t s, int nb, int row0) {
    if (nb < 1 || nb > 65535) {
        set_error("node step: 1 to 65535 right-hand sides per launch");
        return SBD_EINVAL;
    }
    if (row0 < 0 || row0 >= g.nk) {
        set_error("node step: first cleared row outside the grid");
        return SBD_EINVAL;
    }
    const long kb = static_cast<long>(g.nk) * g.nk;
    // the stencils add into a cleared grid: rows row0.. (the rows the caller reads) of each grid
    const size_t row_bytes = sizeof(cx_t<T>) * static_cast<size_t>(g.nk);
    if (nb == 1)
        SBD_CUDA_TRY(cudaMemsetAsync(kout + static_cast<long>(row0) * g.nk, 0, row_bytes * (g.nk - row0), s));
    else
        SBD_CUDA_TRY(cudaMemset2DAsync(kout + static_cast<long>(row0) * g.nk, sizeof(cx_t<T>) * kb, 0,
                                       row_bytes * (g.nk - row0), nb, s));
    const int ntx = tiles_per_side(g.nk);
    const dim3 nt(static_cast<unsigned>(ntx) * ntx, static_cast<unsigned>(nb));
    if constexpr (sizeof(T) == 4) {
        if (t.acc == 3 || t.acc == 4) {
            if (g.Pk > kBinSide) {
                set_error("node step: the binned kernel needs a stencil of at most 8 cells");
                return SBD_EINVAL;
            }
            const Window<float> win = make_window<float>(g.kwin, g.beta_k, g.Pk, g.kpoly);
            if (t.acc == 4)
                return t.sched
                           ? launch_binned<2 * kNodeThreads, true>(nodes, tile_start, nt, ntx, g, win, kin, kout, kb, s)
                           : launch_binned<kNodeThreads, true>(nodes, tile_start, nt, ntx, g, win, kin, kout, kb, s);
            return t.sched ? launch_binned<2 * kNodeThreads>(nodes, tile_start, nt, ntx, g, win, kin, kout, kb, s)
                           : launch_binned<kNodeThreads>(nodes, tile_start, nt, ntx, g, win, kin, kout, kb, s);
        }
    }
    const int W = kNodeTile + g.Pk - 1;
    const int P8 = fused_p8(g.Pk);
    const int Ws = fused_stride(W, P8);
    const Window<T> win = make_window<T>(g.kwin, g.beta_k, g.Pk, g.kpoly, g.kpoly64);
    if (P8 == 8) return launch_fused_g<T, 8>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, t, kb, s);
    if (P8 == 16) return launch_fused_g<T, 16>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, t, kb, s);
    return launch_fused_g<T, 32>(nodes, tile_start, nt, ntx, g, Ws, win, kin, kout, t, kb, s);
}

template <typename T>
int node_step_tiled(const NodeRec<T>* nodes, const long long* tile_start, const FarGeom& g,
                    const cx_t<T>* kin, cx_t<T>* ghat, cx_t<T>* kout, cudaStream_t s, int nb) {
    const long kb = static_cast<long>(g.nk) * g.nk;
    for (int r = 0; r < nb; ++r) {   // fallback for stencils too wide for the fused kernel: one grid at a time
        int rc = launch_gather<T>(nodes, tile_start, g.nk, g.Pk, g.kwin, g.beta_k, kin + r * kb, NodeIO<T>{ghat}, s);
        if (rc) return rc;
        rc = launch_scatter<T>(nodes, tile_start, g.nk, g.Pk, g.kwin, g.beta_k, NodeVal<T>{ghat}, kout + r * kb, s);
        if (rc) return rc;
    }
    return SBD_OK;
}

void point_work_list(const std::vector<long long>& tile_start, int chunk, std::vector<long long>& begin,
                     std::vector<int>& tile) {
    begin.clear();
    tile.clear();
    for (size_t t = 0; t + 1 < tile_start.size(); ++t)
        for (long long b = tile_start[t]; b < tile_start[t + 1]; b += chunk) {
            begin.push_back(b);
            tile.push_back(static_cast<int>(t));
        }
    begin.push_back(tile_start.empty() ? 0 : tile_start.back());
}

// Right-hand sides per CTA of the point kernels: as many shared windows of `per` bytes as
// fit a quarter of the SM's shared memory (four 256-thread CTAs stay resident), at most 4.
inline int rhs_group(size_t per, int nrhs) {
    int rg = static_cast<int>((56u * 1024u) / (per > 0 ? per : 1));
    if (rg > 4) rg = 4;
    if (rg > nrhs) rg = nrhs;
    return rg < 1 ? 1 : rg;
}

template <typename T, int G, bool PK, bool RV>
int launch_spread_chunks(const PointRec<T>* pts, const PointWork& work, const FarGeom& g, PointVal<T> val,
                         cx_t<T>* grid, int nrhs, long gstride, cudaStream_t s) {
    const Window<T> win = make_window<T>(g.swin, g.beta_s, g.Ps, g.spoly, g.spoly64);
    const size_t W = kNodeTile + g.Ps - 1;
    const size_t per = (RV ? 1 : 2) * sizeof(T) * W * W;
    const int rg = rhs_group(per, nrhs);
    const size_t smem = per * rg;
    auto k = spread_chunks_kernel<T, G, PK, RV>;
    SBD_TRY(raise_smem_limit(k, smem));
    const dim3 grd(static_cast<unsigned>(work.count), static_cast<unsigned>((nrhs + rg - 1) / rg));
    k<<<grd, 256, smem, s>>>(pts, work, tiles_per_side(g.m), g.m, g.Ps, win, val, grid, nrhs, rg, gstride);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T, int G, bool PK>
int launch_interp_chunks(const PointRec<T>* pts, const PointWork& work, const FarGeom& g, const cx_t<T>* grid,
                         const PointOut<T>& out, int nrhs, long gstride, cudaStream_t s) {
    // FP32: the window evaluated directly, the table's shared-memory reads cost this gather loop more
    // than they save (it is bound by shared-memory wavefronts; 0.26 against 0.33 ms at N = 10^6);
    // FP64: the FP64 table (the FP64 pipe is the bound there)
    const Window<T> win = make_window<T>(g.swin, g.beta_s, g.Ps, nullptr, g.spoly64);
    const size_t W = kNodeTile + g.Ps - 1;
    const size_t per = (PK ? 1 : 2) * sizeof(T) * W * W;
    const int rg = rhs_group(per, nrhs);
    const size_t smem = per * rg;
    auto k = interp_chunks_kernel<T, G, PK>;
    SBD_TRY(raise_smem_limit(k, smem));
    const dim3 grd(static_cast<unsigned>(work.count), static_cast<unsigned>((nrhs + rg - 1) / rg));
    k<<<grd, 256, smem, s>>>(pts, work, tiles_per_side(g.m), g.m, g.Ps, win, grid, out, nrhs, rg, gstride);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int spread_tiled(const PointRec<T>* pts, const int* perm, const PointWork& work, const FarGeom& g,
                 const void* f, bool f_complex, cx_t<T>* grid, cudaStream_t s, bool packed, int nrhs, long n_pts) {
    if (packed && (f_complex || (g.m & 1))) {
        set_error("spread: a packed real grid needs real values and an even side");
        return SBD_EINVAL;
    }
    if (g.Ps > 32) {
        set_error("spread: stencil wider than 32 cells");
        return SBD_ENOTSUP;
    }
    if (nrhs < 1 || nrhs > 65535 * 4) {
        set_error("spread: right-hand sides out of range");
        return SBD_EINVAL;
    }
    // grid b at b * cells complex elements (the packed real grid is half a complex grid)
    const long cells = static_cast<long>(g.m) * g.m / (packed ? 2 : 1);
    SBD_CUDA_TRY(cudaMemsetAsync(grid, 0, sizeof(cx_t<T>) * cells * nrhs, s));
    if (work.count <= 0) return SBD_OK;
    const PointVal<T> val{f, perm, packed ? false : f_complex, n_pts};
    const bool rv = packed || !f_complex;
    if (packed) {
        if (g.Ps <= 8) return launch_spread_chunks<T, 8, true, true>(pts, work, g, val, grid, nrhs, cells, s);
        if (g.Ps <= 16) return launch_spread_chunks<T, 16, true, true>(pts, work, g, val, grid, nrhs, cells, s);
        return launch_spread_chunks<T, 32, true, true>(pts, work, g, val, grid, nrhs, cells, s);
    }
    if (rv) {
        if (g.Ps <= 8) return launch_spread_chunks<T, 8, false, true>(pts, work, g, val, grid, nrhs, cells, s);
        if (g.Ps <= 16) return launch_spread_chunks<T, 16, false, true>(pts, work, g, val, grid, nrhs, cells, s);
        return launch_spread_chunks<T, 32, false, true>(pts, work, g, val, grid, nrhs, cells, s);
    }
    if (g.Ps <= 8) return launch_spread_chunks<T, 8, false, false>(pts, work, g, val, grid, nrhs, cells, s);
    if (g.Ps <= 16) return launch_spread_chunks<T, 16, false, false>(pts, work, g, val, grid, nrhs, cells, s);
    return launch_spread_chunks<T, 32, false, false>(pts, work, g, val, grid, nrhs, cells, s);
}

template <typename T>
int interp_tiled(const PointRec<T>* pts, const int* perm, const PointWork& work, const FarGeom& g,
                 const cx_t<T>* grid, double2 w0, const double2* sumf, void* q, bool q_complex, cudaStream_t s,
                 bool packed, const void* add, int add_stride, int nrhs, long n_pts) {
    if (nrhs < 1 || nrhs > 65535 * 4) {
        set_error("interp: right-hand sides out of range");
        return SBD_EINVAL;
    }
    const PointOut<T> out{q, perm, q_complex, w0, sumf, add, add_stride, 0, n_pts};
    const long cells = static_cast<long>(g.m) * g.m / (packed ? 2 : 1);
    if (packed && (q_complex || (g.m & 1))) {
        set_error("interp: a packed real grid needs real output and an even side");
        return SBD_EINVAL;
    }
    if (g.Ps > 32) {
        set_error("interp: stencil wider than 32 cells");
        return SBD_ENOTSUP;
    }
    if (work.count <= 0) return SBD_OK;
    if (packed) {
        if (g.Ps <= 8) return launch_interp_chunks<T, 8, true>(pts, work, g, grid, out, nrhs, cells, s);
        if (g.Ps <= 16) return launch_interp_chunks<T, 16, true>(pts, work, g, grid, out, nrhs, cells, s);
        return launch_interp_chunks<T, 32, true>(pts, work, g, grid, out, nrhs, cells, s);
    }
    if (g.Ps <= 8) return launch_interp_chunks<T, 8, false>(pts, work, g, grid, out, nrhs, cells, s);
    if (g.Ps <= 16) return launch_interp_chunks<T, 16, false>(pts, work, g, grid, out, nrhs, cells, s);
    return launch_interp_chunks<T, 32, false>(pts, work, g, grid, out, nrhs, cells, s);
}

template <typename T>
__global__ void fill_kernel(cx_t<T>* __restrict__ x, long n, T re, T im) {
    for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long>(gridDim.x) * blockDim.x)
        x[i] = mk<T>(re, im);
}

template <typename T>
int fill_grid(cx_t<T>* x, long n, T re, T im, cudaStream_t s) {
    if (n <= 0) return SBD_OK;
    const unsigned nb = static_cast<unsigned>(std::min<long>((n + 255) / 256, 152L * 64));
    fill_kernel<T><<<nb, 256, 0, s>>>(x, n, re, im);
    SBD_LAUNCH_CHECK();
    return SBD_OK;
}

template <typename T>
int point_rhs_group(int P, bool two_planes, int nrhs) {
    const size_t W = kNodeTile + P - 1;
    return rhs_group((two_planes ? 2 : 1) * sizeof(T) * W * W, nrhs);
}

int node_fused_stride(int Pk) { return fused_stride(kNodeTile + Pk - 1, fused_p8(Pk)); }

namespace {

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 0;
    return sms;
}

// A cooperative launch of the most CTAs that can be resident at once (so the grid barrier can
// complete), at least one.
template <typename K, typename... A>
int launch_cooperative(K kernel, int threads, size_t smem, cudaStream_t s, A... args) {
    SBD_TRY(raise_smem_limit(kernel, smem));
    int per_sm = 0;
    SBD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    const int sms = sm_count();
    if (per_sm < 1 || sms < 1) {
        set_error("batched launch: kernel does not fit an SM");
        return SBD_ENOTSUP;
    }
    void* argv[] = {static_cast<void*>(&args)...};
    SBD_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(per_sm * sms),
                                             dim3(threads), argv, smem, s));
    return SBD_OK;
}

template <typename T>
size_t point_batch_smem(const PointJobs& J, bool interp) {
    size_t smem = 0;
    for (int j = 0; j < J.count; ++j) {
        const PointJob& jb = J.job[j];
        const size_t W = kNodeTile + jb.P - 1;
        const bool two = interp ? !jb.packed : (jb.complex_io && !jb.packed);
        smem = std::max(smem, (two ? 2 : 1) * sizeof(T) * W * W * jb.rg);
    }
    return smem;
}

}  // namespace

template <typename T>
int spread_batch(const PointJobs& J, int G, BatchSync* sync, unsigned phantom, unsigned long long limit_ns,
                 volatile int* status, cudaStream_t s) {
    const size_t smem = point_batch_smem<T>(J, false);
    if (G == 8) return launch_cooperative(spread_batch_kernel<T, 8>, 256, smem, s, J, sync, phantom, limit_ns, status);
    if (G == 16)
        return launch_cooperative(spread_batch_kernel<T, 16>, 256, smem, s, J, sync, phantom, limit_ns, status);
    return launch_cooperative(spread_batch_kernel<T, 32>, 256, smem, s, J, sync, phantom, limit_ns, status);
}

template <typename T>
int interp_batch(const PointJobs& J, int G, BatchSync* sync, cudaStream_t s) {
    const size_t smem = point_batch_smem<T>(J, true);
    auto launch = [&](auto kernel) {
        SBD_TRY(raise_smem_limit(kernel, smem));
        int per_sm = 0;
        SBD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem));
        const int grid = std::max(1, std::min(std::max(per_sm, 1) * std::max(sm_count(), 1), J.total));
        kernel<<<grid, 256, smem, s>>>(J, sync);
        SBD_LAUNCH_CHECK();
        return SBD_OK;
    };
    if (G == 8) return launch(interp_batch_kernel<T, 8>);
    if (G == 16) return launch(interp_batch_kernel<T, 16>);
    return launch(interp_batch_kernel<T, 32>);
}

template <typename T>
int node_batch(const NodeJobs& J, bool binned, BatchSync* sync, unsigned phantom, unsigned long long limit_ns,
               volatile int* status, cudaStream_t s) {
    if (binned) {
        if constexpr (sizeof(T) == 4)
            return launch_cooperative(node_batch_kernel<float, 8, true>, 2 * kNodeThreads,
                                      node_fused_smem<float>(J.job[0].P, 3), s, J, sync, phantom, limit_ns, status);
        set_error("node_batch: the binned kernel is FP32 only");
        return SBD_EINVAL;
    }
    size_t smem = 0;
    int P8 = 8;
    for (int j = 0; j < J.count; ++j) {
        smem = std::max(smem, node_fused_smem<T>(J.job[j].P, 0));
        P8 = std::max(P8, fused_p8(J.job[j].P));
    }
    if (P8 == 8)
        return launch_cooperative(node_batch_kernel<T, 8, false>, kNodeThreads, smem, s, J, sync, phantom, limit_ns,
                                  status);
    if (P8 == 16)
        return launch_cooperative(node_batch_kernel<T, 16, false>, kNodeThreads, smem, s, J, sync, phantom, limit_ns,
                                  status);
    return launch_cooperative(node_batch_kernel<T, 32, false>, kNodeThreads, smem, s, J, sync, phantom, limit_ns,
                              status);
}

#define SBD_NODE_INST(T)                                                                                     \
    template int tile_sort<NodeRec<T>>(const NodeRec<T>*, long, int, NodeRec<T>*, int*, long long*,          \
                                       cudaStream_t, bool);                                                  \
    template int tile_sort<PointRec<T>>(const PointRec<T>*, long, int, PointRec<T>*, int*, long long*,       \
                                        cudaStream_t, bool);                                                 \
    template int node_step_tiled<T>(const NodeRec<T>*, const long long*, const FarGeom&, const cx_t<T>*,     \
                                    cx_t<T>*, cx_t<T>*, cudaStream_t, int);                                  \
    template size_t node_fused_smem<T>(int, int);                                                            \
    template int fill_grid<T>(cx_t<T>*, long, T, T, cudaStream_t);                                          \
    template int node_step_fused<T>(const NodeRec<T>*, const long long*, const FarGeom&, const cx_t<T>*,     \
                                    cx_t<T>*, const NodeTuning&, cudaStream_t, int, int);                    \
    template int spread_tiled<T>(const PointRec<T>*, const int*, const PointWork&, const FarGeom&,           \
                                 const void*, bool, cx_t<T>*, cudaStream_t, bool, int, long);                \
    template int interp_tiled<T>(const PointRec<T>*, const int*, const PointWork&, const FarGeom&,           \
                                 const cx_t<T>*, double2, const double2*, void*, bool, cudaStream_t, bool,   \
                                 const void*, int, int, long);                                          \
    template int point_rhs_group<T>(int, bool, int);                                                         \
    template int spread_batch<T>(const PointJobs&, int, BatchSync*, unsigned, unsigned long long,            \
                                 volatile int*, cudaStream_t);                                              \
    template int interp_batch<T>(const PointJobs&, int, BatchSync*, cudaStream_t);                           \
    template int node_batch<T>(const NodeJobs&, bool, BatchSync*, unsigned, unsigned long long, volatile int*, \
                               cudaStream_t);
SBD_NODE_INST(float)
SBD_NODE_INST(double)

}  // namespace sbd
