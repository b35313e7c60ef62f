// Binned surface-area-heuristic (SAH) topology of a bottom-level BVH, the
// build for trace speed (RG_BLAS_SAH).  The triangles start in Morton order
// (the LBVH's sort); a segment of that order is one subtree.  Level by level,
// every segment of more than kSahSmall triangles is split by the binned SAH
// (kSahBins bins of the centroid bounds on each axis, the split of least
// area(left) * count(left) + area(right) * count(right)), and partitioned
// stably, so each side keeps its Morton order.  Segments of at most kSahSmall
// triangles (a pair: one node), and every segment below kSahMaxLevels levels,
// get the Karras hierarchy of their Morton codes.  (Stopping the SAH at
// segments of 16 or 4 triangles measured 3-4 % and 1 % slower traversal.)  The internal
// nodes of a segment of c triangles whose root is node d are d .. d + c - 2
// (depth-first numbering: left subtree from d + 1, right from d + count(left)),
// so no allocation is needed and the root is node 0, as in the LBVH.  Every
// choice comes from atomic minima, maxima and counts, which do not depend on
// the order of the atomics, and from one thread's fixed-order sweep, so the
// build is deterministic.  The node boxes are computed afterwards by the
// LBVH's bottom-up refit.
#include <algorithm>
#include <climits>
#include <atomic>
#include <string>
#include <vector>

#include "karras.cuh"
#include "rg_internal.cuh"

namespace rg {

namespace {

constexpr int kBinVals = 7;  // per bin: count, box lo (3), box hi (3) as ordered ints
constexpr int kTaskBins = 3 * kSahBins * kBinVals;
constexpr int kTaskAcc = 6 + kTaskBins;  // centroid bounds (lo 3, hi 3), then the bins
static_assert(kTaskAcc == (int)kSahAccInts, "per-task accumulator size");
constexpr int kSahBlock = 256;

__device__ __forceinline__ float centroid_of(const float* __restrict__ lohi, uint32_t prim, int a) {
    return __fmul_rn(0.5f, __fadd_rn(lohi[6 * (size_t)prim + a], lohi[6 * (size_t)prim + 3 + a]));
}

// Bin of a centroid coordinate: floor((c - cmin) * scale) clamped to the
// bins (NaN to bin 0); the binning and the partition use this one function.
__device__ __forceinline__ int bin_of(float c, float cmin, float scale) {
    const float f = __fmul_rn(__fsub_rn(c, cmin), scale);
    if (!(f >= 0.0f)) return 0;
    return f < (float)kSahBins ? (int)f : kSahBins - 1;
}

__device__ __forceinline__ int ord_inf() { return f2ord(__int_as_float(0x7F800000)); }
__device__ __forceinline__ int ord_ninf() { return f2ord(__int_as_float(0xFF800000)); }

// The chunk of positions block b works on: [chunk begin, end).
__device__ __forceinline__ void chunk_of(const SahTask* tasks, const uint2* blk, uint32_t b, uint32_t& t, uint32_t& p0,
                                         uint32_t& p1) {
    const uint2 e = blk[b];
    t = e.x;
    p0 = e.y;
    const uint32_t end = tasks[t].begin + tasks[t].count;
    p1 = min(p0 + kSahChunk, end);
}

__global__ void k_sah_init(int* __restrict__ acc, uint32_t m) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * (uint32_t)kTaskAcc) return;
    const uint32_t v = i % (uint32_t)kTaskAcc;
    int x;
    if (v < 6) {
        x = v < 3 ? ord_inf() : ord_ninf();
    } else {
        const uint32_t w = (v - 6) % kBinVals;
        x = w == 0 ? 0 : (w < 4 ? ord_inf() : ord_ninf());
    }
    acc[i] = x;
}

// Centroid bounds of each task's segment: a block reduces its chunk, then one
// atomic per bound.
__global__ void __launch_bounds__(kSahBlock) k_sah_cbounds(const float* __restrict__ lohi,
                                                           const uint32_t* __restrict__ prim_at,
                                                           const SahTask* __restrict__ tasks,
                                                           const uint2* __restrict__ blk, int* __restrict__ acc) {
    __shared__ int s[6][kSahBlock / 32];
    uint32_t t, p0, p1;
    chunk_of(tasks, blk, blockIdx.x, t, p0, p1);
    int mn[3] = {ord_inf(), ord_inf(), ord_inf()}, mx[3] = {ord_ninf(), ord_ninf(), ord_ninf()};
    for (uint32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const uint32_t prim = prim_at[p];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int c = f2ord(centroid_of(lohi, prim, a));
            mn[a] = min(mn[a], c);
            mx[a] = max(mx[a], c);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], off));
            mx[a] = max(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], off));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s[a][warp] = mn[a];
            s[3 + a][warp] = mx[a];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        int v = s[q][0];
        for (int w = 1; w < kSahBlock / 32; ++w) v = q < 3 ? min(v, s[q][w]) : max(v, s[q][w]);
        int* dst = acc + (size_t)t * kTaskAcc + q;
        if (q < 3)
            atomicMin(dst, v);
        else
            atomicMax(dst, v);
    }
}

// Per task: the binning frame of each axis from its centroid bounds (scale 0,
// every centroid in bin 0, when the bounds are a point on that axis).
__global__ void k_sah_prep(const int* __restrict__ acc, uint32_t m, SahParam* __restrict__ par) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int* a = acc + (size_t)t * kTaskAcc;
    SahParam P{};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = ord2f(a[k]), hi = ord2f(a[3 + k]);
        const float ext = __fsub_rn(hi, lo);
        P.cmin[k] = lo;
        P.scale[k] = ext > 0.0f ? fminf(__fdiv_rn((float)kSahBins, ext), 3.0e38f) : 0.0f;
    }
    P.axis = -1;
    par[t] = P;
}

// Binning: per block in shared memory (count, box of the triangles per bin
// and axis), then merged into the task's bins once per non-empty bin.
__global__ void __launch_bounds__(kSahBlock) k_sah_bin(const float* __restrict__ lohi,
                                                       const uint32_t* __restrict__ prim_at,
                                                       const SahTask* __restrict__ tasks,
                                                       const uint2* __restrict__ blk, const SahParam* __restrict__ par,
                                                       int* __restrict__ acc) {
    __shared__ int sb[kTaskBins];
    for (int v = threadIdx.x; v < kTaskBins; v += blockDim.x) {
        const int w = v % kBinVals;
        sb[v] = w == 0 ? 0 : (w < 4 ? ord_inf() : ord_ninf());
    }
    __syncthreads();
    uint32_t t, p0, p1;
    chunk_of(tasks, blk, blockIdx.x, t, p0, p1);
    const SahParam P = par[t];
    for (uint32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const uint32_t prim = prim_at[p];
        int lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = f2ord(lohi[6 * (size_t)prim + k]);
            hi[k] = f2ord(lohi[6 * (size_t)prim + 3 + k]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int b = bin_of(centroid_of(lohi, prim, a), P.cmin[a], P.scale[a]);
            int* e = sb + (a * kSahBins + b) * kBinVals;
            atomicAdd(e, 1);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                atomicMin(e + 1 + k, lo[k]);
                atomicMax(e + 4 + k, hi[k]);
            }
        }
    }
    __syncthreads();
    int* g = acc + (size_t)t * kTaskAcc + 6;
    for (int v = threadIdx.x; v < kTaskBins; v += blockDim.x) {
        const int w = v % kBinVals;
        if (sb[v - w] == 0) continue;  // empty bin
        if (w == 0)
            atomicAdd(g + v, sb[v]);
        else if (w < 4)
            atomicMin(g + v, sb[v]);
        else
            atomicMax(g + v, sb[v]);
    }
}

__device__ __forceinline__ float half_area(const float* lo, const float* hi) {
    const float dx = __fsub_rn(hi[0], lo[0]), dy = __fsub_rn(hi[1], lo[1]), dz = __fsub_rn(hi[2], lo[2]);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
}

// Per task (one thread): the split of least SAH cost over the kSahBins - 1
// bin boundaries of each axis, in a fixed order (axis, then boundary; the
// first of equal costs wins); without one (every axis' centroids in one bin)
// the segment is halved by position.  Writes the task's node: its children
// (a leaf when one side holds one triangle), their parent entries, its leaf
// range (ranges may be null), and the left count for the host.
__global__ void k_sah_split(const int* __restrict__ acc, const SahTask* __restrict__ tasks, uint32_t m,
                            SahParam* __restrict__ par, uint32_t n_leaves, float4* __restrict__ nodes,
                            uint32_t* __restrict__ parents, uint32_t* __restrict__ ranges,
                            uint32_t* __restrict__ out_nl) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const SahTask T = tasks[t];
    const int* g = acc + (size_t)t * kTaskAcc + 6;
    float best = __int_as_float(0x7F800000);
    int best_axis = -1, best_split = 0;
    uint32_t best_nl = 0;
    for (int a = 0; a < 3; ++a) {
        float rlo[kSahBins][3], rhi[kSahBins][3];
        uint32_t rc[kSahBins];
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        uint32_t c = 0;
        for (int b = kSahBins - 1; b >= 1; --b) {
            const int* e = g + (a * kSahBins + b) * kBinVals;
            c += (uint32_t)e[0];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], ord2f(e[1 + k]));
                hi[k] = fmaxf(hi[k], ord2f(e[4 + k]));
                rlo[b][k] = lo[k];
                rhi[b][k] = hi[k];
            }
            rc[b] = c;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = INFINITY;
            hi[k] = -INFINITY;
        }
        c = 0;
        for (int s = 1; s < kSahBins; ++s) {
            const int* e = g + (a * kSahBins + s - 1) * kBinVals;
            c += (uint32_t)e[0];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] = fminf(lo[k], ord2f(e[1 + k]));
                hi[k] = fmaxf(hi[k], ord2f(e[4 + k]));
            }
            const uint32_t nl = c, nr = rc[s];
            if (nl == 0 || nr == 0) continue;
            const float cost = __fadd_rn(__fmul_rn(half_area(lo, hi), (float)nl),
                                         __fmul_rn(half_area(rlo[s], rhi[s]), (float)nr));
            if (cost < best) {
                best = cost;
                best_axis = a;
                best_split = s;
                best_nl = nl;
            }
        }
    }
    if (best_axis < 0) best_nl = T.count / 2;
    par[t].axis = best_axis;
    par[t].split = best_split;
    par[t].nl = best_nl;
    out_nl[t] = best_nl;
    const uint32_t nl = best_nl, nr = T.count - best_nl;
    const uint32_t left = nl == 1 ? (kLeaf | T.begin) : T.node + 1;
    const uint32_t right = nr == 1 ? (kLeaf | (T.begin + nl)) : T.node + nl;
    uint32_t* ch = reinterpret_cast<uint32_t*>(nodes + 4 * (size_t)T.node + 3);
    ch[0] = left;
    ch[1] = right;
    parents[(left & kLeaf) ? (size_t)(n_leaves - 1) + (left & ~kLeaf) : left] = T.node;
    parents[(right & kLeaf) ? (size_t)(n_leaves - 1) + (right & ~kLeaf) : right] = T.node;
    if (T.node == 0) parents[0] = kNone;
    if (ranges) {
        ranges[2 * (size_t)T.node] = T.begin;
        ranges[2 * (size_t)T.node + 1] = T.begin + T.count - 1;
    }
}

__device__ __forceinline__ bool goes_left(const float* __restrict__ lohi, uint32_t prim, uint32_t p,
                                          const SahTask& T, const SahParam& P) {
    if (P.axis < 0) return p - T.begin < P.nl;
    return bin_of(centroid_of(lohi, prim, P.axis), P.cmin[P.axis], P.scale[P.axis]) < P.split;
}

// Left-side count of each block's chunk.
__global__ void __launch_bounds__(kSahBlock) k_sah_part_count(const float* __restrict__ lohi,
                                                              const uint32_t* __restrict__ prim_at,
                                                              const SahTask* __restrict__ tasks,
                                                              const uint2* __restrict__ blk,
                                                              const SahParam* __restrict__ par,
                                                              uint32_t* __restrict__ blk_left) {
    __shared__ uint32_t s[kSahBlock / 32];
    uint32_t t, p0, p1;
    chunk_of(tasks, blk, blockIdx.x, t, p0, p1);
    const SahTask T = tasks[t];
    const SahParam P = par[t];
    uint32_t cnt = 0;
    for (uint32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) cnt += goes_left(lohi, prim_at[p], p, T, P);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t v = 0;
        for (int w = 0; w < kSahBlock / 32; ++w) v += s[w];
        blk_left[blockIdx.x] = v;
    }
}

// Per task (one thread): the left-side count before each of its blocks.
__global__ void k_sah_part_offsets(const SahTask* __restrict__ tasks, uint32_t m, const uint32_t* __restrict__ blk_left,
                                   uint32_t* __restrict__ blk_off) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const SahTask T = tasks[t];
    uint32_t off = 0;
    for (uint32_t b = T.first_block; b < T.first_block + T.n_blocks; ++b) {
        blk_off[b] = off;
        off += blk_left[b];
    }
}

// Stable partition: a block walks its chunk in order, tile by tile; a left
// triangle goes to begin + (left triangles before it in the segment), a right
// one to begin + count(left) + (right triangles before it).
template <class K>
__global__ void __launch_bounds__(kSahBlock) k_sah_part_scatter(const float* __restrict__ lohi,
                                                                const uint32_t* __restrict__ prim_at,
                                                                const K* __restrict__ key_at,
                                                                const SahTask* __restrict__ tasks,
                                                                const uint2* __restrict__ blk,
                                                                const SahParam* __restrict__ par,
                                                                const uint32_t* __restrict__ blk_off,
                                                                uint32_t* __restrict__ prim_out, K* __restrict__ key_out) {
    __shared__ uint32_t wc[kSahBlock / 32];
    uint32_t t, p0, p1;
    chunk_of(tasks, blk, blockIdx.x, t, p0, p1);
    const SahTask T = tasks[t];
    const SahParam P = par[t];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t run = blk_off[blockIdx.x];
    for (uint32_t tile = p0; tile < p1; tile += kSahBlock) {
        const uint32_t p = tile + threadIdx.x;
        const bool valid = p < p1;
        uint32_t prim = 0;
        K key = 0;
        bool left = false;
        if (valid) {
            prim = prim_at[p];
            key = key_at[p];
            left = goes_left(lohi, prim, p, T, P);
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, left);
        if (lane == 0) wc[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (uint32_t w = 0; w < kSahBlock / 32; ++w) {
            if (w < warp) before += wc[w];
            total += wc[w];
        }
        if (valid) {
            const uint32_t lrank = run + before + __popc(bal & ((1u << lane) - 1u));
            const uint32_t dest = T.begin + (left ? lrank : P.nl + ((p - T.begin) - lrank));
            prim_out[dest] = prim;
            key_out[dest] = key;
        }
        run += total;
        __syncthreads();
    }
}

template <class K>
__global__ void __launch_bounds__(kSahBlock) k_sah_copy_back(const SahTask* __restrict__ tasks,
                                                             const uint2* __restrict__ blk,
                                                             const uint32_t* __restrict__ prim_out,
                                                             const K* __restrict__ key_out,
                                                             uint32_t* __restrict__ prim_at, K* __restrict__ key_at) {
    uint32_t t, p0, p1;
    chunk_of(tasks, blk, blockIdx.x, t, p0, p1);
    for (uint32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        prim_at[p] = prim_out[p];
        key_at[p] = key_out[p];
    }
}

template <class K>
cudaError_t sah_level_t(const SahLevel& L, cudaStream_t s) {
    const uint32_t tg = (L.m + 127u) / 128u;
    k_sah_init<<<(L.m * (uint32_t)kTaskAcc + 255u) / 256u, 256, 0, s>>>(L.acc, L.m);
    k_sah_cbounds<<<L.n_blocks, kSahBlock, 0, s>>>(L.lohi, L.prim_at, L.tasks, L.blk, L.acc);
    k_sah_prep<<<tg, 128, 0, s>>>(L.acc, L.m, L.par);
    k_sah_bin<<<L.n_blocks, kSahBlock, 0, s>>>(L.lohi, L.prim_at, L.tasks, L.blk, L.par, L.acc);
    k_sah_split<<<tg, 128, 0, s>>>(L.acc, L.tasks, L.m, L.par, L.n_leaves, L.nodes, L.parents, L.ranges, L.out_nl);
    k_sah_part_count<<<L.n_blocks, kSahBlock, 0, s>>>(L.lohi, L.prim_at, L.tasks, L.blk, L.par, L.blk_left);
    k_sah_part_offsets<<<tg, 128, 0, s>>>(L.tasks, L.m, L.blk_left, L.blk_off);
    k_sah_part_scatter<K><<<L.n_blocks, kSahBlock, 0, s>>>(L.lohi, L.prim_at, static_cast<const K*>(L.key_at), L.tasks,
                                                           L.blk, L.par, L.blk_off, L.prim_out,
                                                           static_cast<K*>(L.key_out));
    k_sah_copy_back<K><<<L.n_blocks, kSahBlock, 0, s>>>(L.tasks, L.blk, L.prim_out, static_cast<const K*>(L.key_out),
                                                        L.prim_at, static_cast<K*>(L.key_at));
    count_launches(9);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- small builds in blocks
// The same hierarchy for at most kSahOneMax items (a TLAS rebuilt every
// frame) in three launches after the Morton codes, without host round trips.
// Phase 1, one block of 1024 threads: the stable Morton sort (an LSD radix
// sort in shared memory), then levels of splits of the segments of more than
// kSahSubMax items; the children of at most kSahSubMax
// items go to a pending list.  Phase 2, a grid of blocks of kSahSubMax
// threads: each block takes pending segments and builds them to the end.
// Both keep every item's box in shared memory.  Every choice uses the
// functions and the order of the level-by-level build above (centroid_of,
// bin_of, the frames, the bins, the sweep), so the tree is the same.  The
// split's bins also give the exact boxes of both children (the minima and
// maxima of their items' boxes), which are written into the node; only
// position halvings (no valid split) and Karras segments below the depth cap
// leave boxes to the bottom-up refit, which the build then asks for.
constexpr uint32_t kSahSubMax = 128;     // items of a phase-2 segment (= its block's threads)
constexpr uint32_t kSahTopSegs = kSahOneMax / (kSahSubMax + 1) + 1;  // phase-1 segments of a level
constexpr uint32_t kSahSubSegs = kSahSubMax / 3 + 1;                  // phase-2 segments of a level
constexpr uint16_t kSegNone = 0xFFFF;
constexpr int kAcc = (kTaskAcc + 3) & ~3;  // a segment's accumulators in a block, padded to 16 bytes

struct OneSeg {
    uint16_t begin, count, node, pad;    // block-local first position, items, internal node
};
struct OneRes {
    uint16_t nl;                         // items on the left
    int8_t axis, split;                  // the split (axis -1: halving by position)
    float cmin, scale;                   // the axis's binning frame
    uint16_t child[2];                   // next-level segment of each side, or kSegNone
};
struct SahPending {
    uint32_t begin, count, node, level;  // a segment for phase 2 (global positions)
};

// Shared state of a block that builds the segments of NMAX items, at most SEGS
// of them split per level.  Items are named by a block-local index: the box
// of each, its Morton rank, and the local index at each position.
template <int NMAX, int SEGS>
struct BlockSah {
    float box[NMAX][6];                  // (phase 1's sort uses it as scratch first)
    uint16_t gr[NMAX];                   // Morton rank of each local index
    uint16_t idx[2][NMAX];               // local index at each position (two buffers)
    uint16_t seg_of[NMAX];               // this level's segment of each position, or kSegNone
    uint16_t excl[NMAX];                 // left items before each position
    OneSeg seg[2][SEGS];
    OneRes res[SEGS];
    alignas(16) int acc[SEGS * kAcc];    // per segment: centroid bounds and bins
    float par[SEGS * 6];                 // per segment: cmin and scale of each axis
    unsigned long long best[SEGS];       // per segment: least (cost, candidate)
    alignas(16) int pat[kAcc];           // the accumulators' initial values of one segment
    uint32_t m, mnext, npend, wsum[32];
};
using BlockTop = BlockSah<kSahOneMax, kSahTopSegs>;
using BlockSub = BlockSah<kSahSubMax, kSahSubSegs>;
static_assert(sizeof(BlockTop) <= 227 * 1024 && 3 * sizeof(BlockSub) <= 227 * 1024, "shared memory of the SAH blocks");
static_assert(kSahOneMax <= 0xFFFFu && kSahOneMax % 1024 == 0, "16-bit positions and whole positions per thread");
static_assert(kSahOneMax * 6 * sizeof(float) >= kSahOneMax * 6 + 32 * 65 * 4 + 32 * 4, "sort scratch fits the boxes");

// Node `node` over leaves b .. b + c - 1 with nl on the left: its children
// (a leaf when one side holds one item), their parent entries, its range.
__device__ __forceinline__ void emit_sah_node(uint32_t node, uint32_t b, uint32_t c, uint32_t nl, uint32_t n_leaves,
                                              float4* nodes, uint32_t* parents, uint32_t* ranges) {
    const uint32_t nr = c - nl;
    const uint32_t left = nl == 1 ? (kLeaf | b) : node + 1;
    const uint32_t right = nr == 1 ? (kLeaf | (b + nl)) : node + nl;
    uint32_t* ch = reinterpret_cast<uint32_t*>(nodes + 4 * (size_t)node + 3);
    ch[0] = left;
    ch[1] = right;
    parents[(left & kLeaf) ? (size_t)(n_leaves - 1) + (left & ~kLeaf) : left] = node;
    parents[(right & kLeaf) ? (size_t)(n_leaves - 1) + (right & ~kLeaf) : right] = node;
    if (node == 0) parents[0] = kNone;
    if (ranges) {
        ranges[2 * (size_t)node] = b;
        ranges[2 * (size_t)node + 1] = b + c - 1;
    }
}

// The boxes of a node's two children (lo xyz, hi xyz each), in the node's
// layout: floats 0-5 the left child's, 6-11 the right child's.
__device__ __forceinline__ void put_child_boxes(float4* nodes, uint32_t node, const float* l, const float* r) {
    float4* f = nodes + 4 * (size_t)node;
    f[0] = make_float4(l[0], l[1], l[2], l[3]);
    f[1] = make_float4(l[4], l[5], r[0], r[1]);
    f[2] = make_float4(r[2], r[3], r[4], r[5]);
}

// Keys of a segment through its positions' local indices.
template <class K>
struct LocalKeys {
    const K* keys;
    const uint16_t* gr;
    const uint16_t* idx;
    __device__ __forceinline__ K operator[](int64_t i) const { return keys[gr[idx[i]]]; }
};

// Stable sort of n <= NMAX 30-bit Morton codes in shared memory: the sorted
// codes, and the index of each, to keys_out and perm0.  An LSD radix sort, 6
// bits a pass: a warp ranks its items of one digit by ballots, a block-wide
// scan of the (digit, warp) counts places them.  The items are padded to NMAX
// with the largest code (after every real item, which keeps them last).  Item
// j of (warp w, lane l) is position 128 w + 32 j + l, so a warp's items in
// (j, lane) order are in position order, and each pass is stable.
template <int NT, int NMAX>
__device__ void block_sort_codes(unsigned char* scratch, const uint32_t* __restrict__ codes, uint32_t n,
                                 uint32_t* keys_out, uint32_t* perm0) {
    static_assert(NMAX == 4 * NT && NT % 32 == 0, "four items per thread");
    constexpr int D = 6, R = 1 << D, W = NT / 32, CS = R + 1;  // counters [warp][digit], padded rows
    uint32_t* kbuf = reinterpret_cast<uint32_t*>(scratch);
    uint16_t* vbuf = reinterpret_cast<uint16_t*>(kbuf + NMAX);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(vbuf + NMAX);
    uint32_t* wtot = cnt + W * CS;
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t k[4], v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t p = 128u * warp + 32u * j + lane;
        k[j] = p < n ? codes[p] : 0x3FFFFFFFu;
        v[j] = p;
    }
    for (int shift = 0; shift < 30; shift += D) {
        for (uint32_t i = lane; i < (uint32_t)R; i += 32) cnt[warp * CS + i] = 0;
        __syncwarp();
        uint32_t rank[4], dig[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t d = (k[j] >> shift) & (R - 1);
            uint32_t peers = 0xFFFFFFFFu;
#pragma unroll
            for (int bit = 0; bit < D; ++bit) {
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (d >> bit) & 1u);
                peers &= ((d >> bit) & 1u) ? bal : ~bal;
            }
            const uint32_t before = cnt[warp * CS + d];
            dig[j] = d;
            rank[j] = before + __popc(peers & lt);
            __syncwarp();
            if ((peers & lt) == 0) cnt[warp * CS + d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // exclusive scan of the counters in (digit, warp) order, two a thread
        uint32_t e[2], sum = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t i = 2 * t + h, d = i / W, w = i % W;
            e[h] = (i < (uint32_t)(R * W)) ? cnt[w * CS + d] : 0u;
            sum += e[h];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
            if ((int)lane >= off) inc += y;
        }
        if (lane == 31) wtot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t x = lane < (uint32_t)W ? wtot[lane] : 0u;
            uint32_t winc = x;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, winc, off);
                if ((int)lane >= off) winc += y;
            }
            if (lane < (uint32_t)W) wtot[lane] = winc - x;
        }
        __syncthreads();
        uint32_t run = wtot[warp] + inc - sum;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t i = 2 * t + h, d = i / W, w = i % W;
            if (i < (uint32_t)(R * W)) cnt[w * CS + d] = run;
            run += e[h];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t dst = cnt[warp * CS + dig[j]] + rank[j];
            kbuf[dst] = k[j];
            vbuf[dst] = (uint16_t)v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t p = 128u * warp + 32u * j + lane;
            k[j] = kbuf[p];
            v[j] = vbuf[p];
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t p = 128u * warp + 32u * j + lane;
        if (p < n) {
            keys_out[p] = k[j];
            perm0[p] = v[j];
        }
    }
}

// Builds the segment of cnt items at global positions base .. base + cnt - 1,
// rooted at internal node `node` at depth level0.  With stop > 0, children of
// at most `stop` items go to the pending list instead of being split here.
// The Morton rank at position base + i is base + i (phase 1) or rank_g's.
// perm0 and keys may be written earlier in the same launch: no read-only
// loads through them.
template <int NT, int NMAX, int SEGS>
__device__ void sah_block(BlockSah<NMAX, SEGS>& S, const float* __restrict__ lohi, uint32_t n_leaves,
                          const uint32_t* keys, const uint32_t* perm0, uint32_t* rank_g, uint32_t base, uint32_t cnt,
                          uint32_t node, uint32_t level0, uint32_t stop, bool ranks_identity, SahPending* pending,
                          uint32_t* n_pending, float4* nodes, uint32_t* parents, uint32_t* ranges,
                          uint32_t* boxes_done) {
    constexpr uint32_t P = (NMAX + NT - 1) / NT;  // positions per thread in the partition's scan
    constexpr int W = NT / 32;
    constexpr bool kByShuffle = NT >= 512;       // the sweep: 16-lane groups, else a thread per axis
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    for (uint32_t i = t; i < cnt; i += NT) {
        const uint32_t r = ranks_identity ? base + i : rank_g[base + i];
        const uint32_t prim = perm0[r];
        S.gr[i] = (uint16_t)r;
#pragma unroll
        for (int k = 0; k < 6; ++k) S.box[i][k] = lohi[6 * (size_t)prim + k];
        S.idx[0][i] = (uint16_t)i;
        S.seg_of[i] = 0;
    }
    for (uint32_t w = t; w < (uint32_t)kAcc; w += NT) {
        int x;
        if (w >= (uint32_t)kTaskAcc) {
            x = 0;
        } else if (w < 6) {
            x = w < 3 ? ord_inf() : ord_ninf();
        } else {
            const uint32_t u = (w - 6) % kBinVals;
            x = u == 0 ? 0 : (u < 4 ? ord_inf() : ord_ninf());
        }
        S.pat[w] = x;
    }
    if (t == 0) {
        S.seg[0][0] = OneSeg{0, (uint16_t)cnt, (uint16_t)node, 0};
        S.m = 1;
        S.npend = 0;
    }
    __syncthreads();
    int cb = 0;
    for (uint32_t level = level0;; ++level) {
        const uint32_t m = S.m;
        if (m == 0) break;
        OneSeg* cur = S.seg[cb];
        OneSeg* nxt = S.seg[cb ^ 1];
        const uint16_t* ix = S.idx[cb];
        uint16_t* ix2 = S.idx[cb ^ 1];
        __syncthreads();
        if (t == 0) S.mnext = 0;
        for (uint32_t v = t; v < m * (uint32_t)(kAcc / 4); v += NT) {
            const uint32_t q = v / (uint32_t)(kAcc / 4), w = v - q * (uint32_t)(kAcc / 4);
            reinterpret_cast<int4*>(S.acc)[v] = reinterpret_cast<const int4*>(S.pat)[w];
        }
        __syncthreads();
        // centroid bounds: each thread's P consecutive positions merged per run
        // of one segment; one warp reduction when the warp holds one segment
        {
            uint32_t rq = kSegNone;
            bool multi = false;
            int mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
#pragma unroll
            for (uint32_t j = 0; j < P; ++j) {
                const uint32_t p = P * t + j;
                const uint32_t q = p < cnt ? S.seg_of[p] : kSegNone;
                if (q == kSegNone) continue;
                const float* bx = S.box[ix[p]];
                int c[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) c[k] = f2ord(centroid_of(bx, 0, k));
                if (q != rq) {
                    if (rq != kSegNone) {
                        int* ac = S.acc + (size_t)rq * kAcc;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            atomicMin(ac + k, mn[k]);
                            atomicMax(ac + 3 + k, mx[k]);
                        }
                        multi = true;
                    }
                    rq = q;
#pragma unroll
                    for (int k = 0; k < 3; ++k) mn[k] = mx[k] = c[k];
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        mn[k] = min(mn[k], c[k]);
                        mx[k] = max(mx[k], c[k]);
                    }
                }
            }
            const uint32_t q0 = __shfl_sync(0xFFFFFFFFu, rq, 0);
            const bool uni = __all_sync(0xFFFFFFFFu, rq == q0 && !multi);
            if (uni) {
                if (q0 != kSegNone) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        mn[k] = __reduce_min_sync(0xFFFFFFFFu, mn[k]);
                        mx[k] = __reduce_max_sync(0xFFFFFFFFu, mx[k]);
                    }
                    if (lane == 0) {
                        int* ac = S.acc + (size_t)q0 * kAcc;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            atomicMin(ac + k, mn[k]);
                            atomicMax(ac + 3 + k, mx[k]);
                        }
                    }
                }
            } else if (rq != kSegNone) {
                int* ac = S.acc + (size_t)rq * kAcc;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    atomicMin(ac + k, mn[k]);
                    atomicMax(ac + 3 + k, mx[k]);
                }
            }
        }
        __syncthreads();
        for (uint32_t q = t; q < m; q += NT) {
            const int* a = S.acc + (size_t)q * kAcc;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float lo = ord2f(a[k]), hi = ord2f(a[3 + k]);
                const float ext = __fsub_rn(hi, lo);
                S.par[6 * q + k] = lo;
                S.par[6 * q + 3 + k] = ext > 0.0f ? fminf(__fdiv_rn((float)kSahBins, ext), 3.0e38f) : 0.0f;
            }
            S.best[q] = ~0ull;
        }
        __syncthreads();
        // bins: each thread's P consecutive positions merged per run of one
        // segment and bin on each axis, one set of atomics per run
        {
            uint32_t rq = kSegNone;
            int rb[3] = {0, 0, 0};
            int st[3][7];
#pragma unroll
            for (uint32_t j = 0; j < P; ++j) {
                const uint32_t p = P * t + j;
                const uint32_t q = p < cnt ? S.seg_of[p] : kSegNone;
                if (q == kSegNone) continue;
                const float* bx = S.box[ix[p]];
                int v[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] = f2ord(bx[k]);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int b = bin_of(centroid_of(bx, 0, a), S.par[6 * q + a], S.par[6 * q + 3 + a]);
                    if (q == rq && b == rb[a]) {
                        st[a][0] += 1;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            st[a][1 + k] = min(st[a][1 + k], v[k]);
                            st[a][4 + k] = max(st[a][4 + k], v[3 + k]);
                        }
                    } else {
                        if (rq != kSegNone) {
                            int* e = S.acc + (size_t)rq * kAcc + 6 + (a * kSahBins + rb[a]) * kBinVals;
                            atomicAdd(e, st[a][0]);
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                atomicMin(e + 1 + k, st[a][1 + k]);
                                atomicMax(e + 4 + k, st[a][4 + k]);
                            }
                        }
                        rb[a] = b;
                        st[a][0] = 1;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            st[a][1 + k] = v[k];
                            st[a][4 + k] = v[3 + k];
                        }
                    }
                }
                rq = q;
            }
            if (rq != kSegNone) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int* e = S.acc + (size_t)rq * kAcc + 6 + (a * kSahBins + rb[a]) * kBinVals;
                    atomicAdd(e, st[a][0]);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        atomicMin(e + 1 + k, st[a][1 + k]);
                        atomicMax(e + 4 + k, st[a][4 + k]);
                    }
                }
            }
        }
        __syncthreads();
        // the least cost over the candidates (axis a, boundary s) of each
        // segment, first in the candidates' order among equal costs: a packed
        // key (cost bits, then the candidate's index a * 15 + s - 1; -0 taken
        // as +0).  The minima and maxima of each side are exact in any order
        // (a float and an ordered-int fold may differ only in the sign of a
        // zero, which reaches the cost only as the sign of a zero cost), so
        // the choice is the level-by-level sweep's.
        if (kByShuffle) {
            // 16-lane groups, one per (segment, axis): lane s holds bin s; the
            // left side of boundary s is the prefix of bins 0 .. s - 1, the
            // right side the suffix s .. 15, both scanned across the lanes
        for (uint32_t v = t; v < ((m * 48u + 31u) & ~31u); v += NT) {
            const uint32_t g = v >> 4, s = v & 15u;
            const bool valid = g < m * 3u;
            const uint32_t q = valid ? g / 3u : 0u;
            const int a = valid ? (int)(g % 3u) : 0;
            const int* e = S.acc + (size_t)q * kAcc + 6 + (a * kSahBins + (int)s) * kBinVals;
            int pc = valid ? e[0] : 0, sc = pc;
            int pv[6], sv[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) pv[k] = sv[k] = valid ? e[1 + k] : (k < 3 ? ord_inf() : ord_ninf());
#pragma unroll
            for (int d = 1; d < 16; d <<= 1) {
                const int yc = __shfl_up_sync(0xFFFFFFFFu, pc, d, 16);
                const int zc = __shfl_down_sync(0xFFFFFFFFu, sc, d, 16);
                if ((int)s >= d) pc += yc;
                if ((int)s + d < 16) sc += zc;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const int y = __shfl_up_sync(0xFFFFFFFFu, pv[k], d, 16);
                    const int z = __shfl_down_sync(0xFFFFFFFFu, sv[k], d, 16);
                    if ((int)s >= d) pv[k] = k < 3 ? min(pv[k], y) : max(pv[k], y);
                    if ((int)s + d < 16) sv[k] = k < 3 ? min(sv[k], z) : max(sv[k], z);
                }
            }
            const int lc = __shfl_up_sync(0xFFFFFFFFu, pc, 1, 16);
            float lo[3], hi[3], rlo[3], rhi[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] = ord2f(__shfl_up_sync(0xFFFFFFFFu, pv[k], 1, 16));
                hi[k] = ord2f(__shfl_up_sync(0xFFFFFFFFu, pv[3 + k], 1, 16));
                rlo[k] = ord2f(sv[k]);
                rhi[k] = ord2f(sv[3 + k]);
            }
            unsigned long long key = ~0ull;
            if (valid && s >= 1u && lc != 0 && sc != 0) {
                const float cost = __fadd_rn(__fadd_rn(__fmul_rn(half_area(lo, hi), (float)(uint32_t)lc),
                                                       __fmul_rn(half_area(rlo, rhi), (float)(uint32_t)sc)),
                                             0.0f);
                if (cost < INFINITY)
                    key = ((unsigned long long)__float_as_uint(cost) << 32) | (uint32_t)(a * (kSahBins - 1) + (int)s - 1);
            }
#pragma unroll
            for (int d = 8; d > 0; d >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, key, d, 16);
                key = y < key ? y : key;
            }
            if (valid && s == 0u && key != ~0ull) atomicMin(&S.best[q], key);
        }
        } else {
            // a thread per (segment, axis): the sweep's suffix and prefix folds
            for (uint32_t v = t; v < m * 3u; v += NT) {
                const uint32_t q = v / 3u;
                const int a = (int)(v % 3u);
                const int* g = S.acc + (size_t)q * kAcc + 6 + a * kSahBins * kBinVals;
                float rlo[kSahBins][3], rhi[kSahBins][3];
                uint32_t rc[kSahBins];
                float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                uint32_t c = 0;
#pragma unroll
                for (int b = kSahBins - 1; b >= 1; --b) {
                    const int* e = g + b * kBinVals;
                    c += (uint32_t)e[0];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        lo[k] = fminf(lo[k], ord2f(e[1 + k]));
                        hi[k] = fmaxf(hi[k], ord2f(e[4 + k]));
                        rlo[b][k] = lo[k];
                        rhi[b][k] = hi[k];
                    }
                    rc[b] = c;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    lo[k] = INFINITY;
                    hi[k] = -INFINITY;
                }
                c = 0;
                unsigned long long best = ~0ull;
#pragma unroll
                for (int s = 1; s < kSahBins; ++s) {
                    const int* e = g + (s - 1) * kBinVals;
                    c += (uint32_t)e[0];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        lo[k] = fminf(lo[k], ord2f(e[1 + k]));
                        hi[k] = fmaxf(hi[k], ord2f(e[4 + k]));
                    }
                    if (c == 0 || rc[s] == 0) continue;
                    const float cost = __fadd_rn(__fadd_rn(__fmul_rn(half_area(lo, hi), (float)c),
                                                           __fmul_rn(half_area(rlo[s], rhi[s]), (float)rc[s])),
                                                 0.0f);
                    if (!(cost < INFINITY)) continue;
                    const unsigned long long key = ((unsigned long long)__float_as_uint(cost) << 32) |
                                                   (uint32_t)(a * (kSahBins - 1) + s - 1);
                    best = key < best ? key : best;
                }
                if (best != ~0ull) atomicMin(&S.best[q], best);
            }
        }
        __syncthreads();
        // the split of each segment, its node, and its children's boxes from
        // the bins of each side
        for (uint32_t q = t; q < m; q += NT) {
            const unsigned long long key = S.best[q];
            const uint32_t count = cur[q].count;
            OneRes R;
            R.axis = -1;
            R.split = 0;
            R.nl = (uint16_t)(count / 2);
            R.cmin = R.scale = 0.0f;
            if (key != ~0ull) {
                const uint32_t c = (uint32_t)key;
                const int a = (int)(c / (kSahBins - 1)), sp = (int)(c % (kSahBins - 1)) + 1;
                const int* g = S.acc + (size_t)q * kAcc + 6 + a * kSahBins * kBinVals;
                int lb[6], rb[6];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    lb[k] = rb[k] = ord_inf();
                    lb[3 + k] = rb[3 + k] = ord_ninf();
                }
                uint32_t nl = 0;
                for (int b = 0; b < kSahBins; ++b) {
                    const int* e = g + b * kBinVals;
                    int* d = b < sp ? lb : rb;
                    if (b < sp) nl += (uint32_t)e[0];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        d[k] = min(d[k], e[1 + k]);
                        d[3 + k] = max(d[3 + k], e[4 + k]);
                    }
                }
                float l[6], r[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    l[k] = ord2f(lb[k]);
                    r[k] = ord2f(rb[k]);
                }
                put_child_boxes(nodes, cur[q].node, l, r);
                R.axis = (int8_t)a;
                R.split = (int8_t)sp;
                R.nl = (uint16_t)nl;
                R.cmin = S.par[6 * q + a];
                R.scale = S.par[6 * q + 3 + a];
            } else {
                *boxes_done = 0u;  // halved by position: the children's boxes come from the refit
            }
            R.child[0] = R.child[1] = kSegNone;
            S.res[q] = R;
            emit_sah_node(cur[q].node, base + cur[q].begin, count, R.nl, n_leaves, nodes, parents, ranges);
        }
        __syncthreads();
        // stable partition: exclusive left counts over the positions (thread t
        // owns positions P t .. P t + P - 1)
        bool left[P];
        uint32_t mine = 0;
#pragma unroll
        for (uint32_t j = 0; j < P; ++j) {
            const uint32_t p = P * t + j;
            left[j] = false;
            if (p < cnt && S.seg_of[p] != kSegNone) {
                const uint16_t q = S.seg_of[p];
                const OneRes R = S.res[q];
                left[j] = R.axis < 0 ? (p - cur[q].begin < R.nl)
                                     : bin_of(centroid_of(S.box[ix[p]], 0, R.axis), R.cmin, R.scale) < R.split;
            }
            mine += left[j];
        }
        uint32_t inc = mine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
            if ((int)lane >= off) inc += y;
        }
        if (lane == 31) S.wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t x = lane < (uint32_t)W ? S.wsum[lane] : 0u;
            uint32_t winc = x;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, winc, off);
                if ((int)lane >= off) winc += y;
            }
            if (lane < (uint32_t)W) S.wsum[lane] = winc - x;
        }
        __syncthreads();
        uint32_t run = S.wsum[warp] + inc - mine;
#pragma unroll
        for (uint32_t j = 0; j < P; ++j) {
            const uint32_t p = P * t + j;
            if (p < cnt) S.excl[p] = (uint16_t)run;
            run += left[j];
        }
        __syncthreads();
#pragma unroll
        for (uint32_t j = 0; j < P; ++j) {
            const uint32_t p = P * t + j;
            if (p >= cnt) continue;
            const uint16_t q = S.seg_of[p];
            if (q == kSegNone) {
                ix2[p] = ix[p];
                continue;
            }
            const uint32_t b = cur[q].begin;
            const uint32_t lr = (uint32_t)S.excl[p] - (uint32_t)S.excl[b];
            ix2[b + (left[j] ? lr : (uint32_t)S.res[q].nl + ((p - b) - lr))] = ix[p];
        }
        __syncthreads();
        // children: pairs, the Karras hierarchy below the depth cap, pending
        // segments, or the next level
        for (uint32_t q = t; q < m; q += NT) {
            const OneSeg G = cur[q];
            const uint32_t nl = S.res[q].nl;
            for (int side = 0; side < 2; ++side) {
                const uint32_t b = side ? G.begin + nl : G.begin;
                const uint32_t c = side ? G.count - nl : nl;
                const uint32_t nd = side ? G.node + nl : G.node + 1;
                if (c == 2) {
                    emit_sah_node(nd, base + b, 2, 1, n_leaves, nodes, parents, ranges);
                    put_child_boxes(nodes, nd, S.box[ix2[b]], S.box[ix2[b + 1]]);
                } else if (c >= 3 && level + 1 >= kSahMaxLevels) {
                    const LocalKeys<uint32_t> ks{keys, S.gr, ix2 + b};
                    for (uint32_t i = 0; i + 1 < c; ++i)
                        karras_node(ks, c, (int64_t)i, reinterpret_cast<uint32_t*>(nodes) + 12, 16, parents, ranges,
                                    nd, base + b, n_leaves);
                    *boxes_done = 0u;  // the Karras nodes' boxes come from the refit
                } else if (c >= 3 && stop > 0 && c <= stop) {
                    const uint32_t k = atomicAdd(&S.npend, 1u);
                    pending[k] = SahPending{base + b, c, nd, level + 1};
                } else if (c >= 3) {
                    const uint32_t slot = atomicAdd(&S.mnext, 1u);
                    nxt[slot] = OneSeg{(uint16_t)b, (uint16_t)c, (uint16_t)nd, 0};
                    S.res[q].child[side] = (uint16_t)slot;
                }
            }
        }
        __syncthreads();
        for (uint32_t p = t; p < cnt; p += NT) {
            const uint16_t q = S.seg_of[p];
            if (q == kSegNone) continue;
            S.seg_of[p] = S.res[q].child[p - cur[q].begin >= S.res[q].nl ? 1 : 0];
        }
        if (t == 0) S.m = S.mnext;
        cb ^= 1;
        __syncthreads();

    }
    for (uint32_t p = t; p < cnt; p += NT) rank_g[base + p] = S.gr[S.idx[cb][p]];
    if (t == 0 && stop > 0) *n_pending = S.npend;
    __syncthreads();
}

// Phase 1: the Morton sort, then the splits of the segments of more than
// kSahSubMax items.
__global__ void __launch_bounds__(1024, 1) k_sah_top(const float* __restrict__ lohi, uint32_t n,
                                                     const uint32_t* __restrict__ codes, uint32_t* keys,
                                                     uint32_t* perm0, uint32_t* rank_g, SahPending* pending,
                                                     uint32_t* n_pending, float4* nodes, uint32_t* parents,
                                                     uint32_t* ranges, uint32_t* boxes_done) {
    extern __shared__ __align__(16) unsigned char sm[];
    BlockTop& S = *reinterpret_cast<BlockTop*>(sm);
    block_sort_codes<1024, kSahOneMax>(reinterpret_cast<unsigned char*>(&S.box[0][0]), codes, n, keys, perm0);
    for (uint32_t p = threadIdx.x; p < n; p += blockDim.x) rank_g[p] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        *n_pending = 0;
        *boxes_done = 1u;
        if (n == 2) {
            emit_sah_node(0, 0, 2, 1, n, nodes, parents, ranges);
            put_child_boxes(nodes, 0, lohi + 6 * (size_t)perm0[0], lohi + 6 * (size_t)perm0[1]);
        }
        if (n >= 3 && n <= kSahSubMax) {
            pending[0] = SahPending{0u, n, 0u, 0u};
            *n_pending = 1;
        }
    }
    __syncthreads();
    if (n <= kSahSubMax) return;
    sah_block<1024, kSahOneMax, kSahTopSegs>(S, lohi, n, keys, perm0, rank_g, 0, n, 0, 0, kSahSubMax, true, pending,
                                             n_pending, nodes, parents, ranges, boxes_done);
}

// Phase 2: each block builds pending segments to the end.
__global__ void __launch_bounds__(kSahSubMax) k_sah_sub(const float* __restrict__ lohi, uint32_t n,
                                                        const uint32_t* __restrict__ keys,
                                                        const uint32_t* __restrict__ perm0, uint32_t* rank_g,
                                                        const SahPending* __restrict__ pending,
                                                        const uint32_t* __restrict__ n_pending, float4* nodes,
                                                        uint32_t* parents, uint32_t* ranges, uint32_t* boxes_done) {
    extern __shared__ __align__(16) unsigned char sm[];
    BlockSub& S = *reinterpret_cast<BlockSub*>(sm);
    const uint32_t np = *n_pending;
    for (uint32_t k = blockIdx.x; k < np; k += gridDim.x) {
        const SahPending T = pending[k];
        sah_block<kSahSubMax, kSahSubMax, kSahSubSegs>(S, lohi, n, keys, perm0, rank_g, T.begin, T.count, T.node,
                                                       T.level, 0, false, nullptr, nullptr, nodes, parents, ranges,
                                                       boxes_done);
    }
}

__global__ void k_sah_gather(const uint32_t* __restrict__ perm0, const uint32_t* __restrict__ rank_g, uint32_t n,
                             uint32_t* __restrict__ perm_out) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) perm_out[p] = perm0[rank_g[p]];
}

}  // namespace

cudaError_t launch_sah_small(const float* lohi, uint32_t n, const uint32_t* codes, uint32_t* perm_out, float4* nodes,
                             uint32_t* parents, uint32_t* ranges, const SahSmallScratch& w, cudaStream_t s) {
    if (n < 2 || n > kSahOneMax) return cudaErrorInvalidValue;
    static std::atomic<int> attr_set{0};  // per process; concurrent first callers set the same values
    if (!attr_set.load(std::memory_order_acquire)) {
        cudaError_t e = cudaFuncSetAttribute(k_sah_top, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(BlockTop));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sah_sub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BlockSub));
        if (e != cudaSuccess) return e;
        attr_set.store(1, std::memory_order_release);
    }
    SahPending* pending = static_cast<SahPending*>(w.pending);
    k_sah_top<<<1, 1024, sizeof(BlockTop), s>>>(lohi, n, codes, w.keys, w.perm0, w.rank, pending, w.n_pending, nodes,
                                                parents, ranges, w.boxes_done);
    const uint32_t grid = std::min<uint32_t>((uint32_t)device_sm_count(), n / 3 + 1);
    k_sah_sub<<<grid, kSahSubMax, sizeof(BlockSub), s>>>(lohi, n, w.keys, w.perm0, w.rank, pending, w.n_pending,
                                                         nodes, parents, ranges, w.boxes_done);
    k_sah_gather<<<(n + 255) / 256, 256, 0, s>>>(w.perm0, w.rank, n, perm_out);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_sah_level(const SahLevel& L, int key_bits, cudaStream_t s) {
    if (L.m == 0) return cudaSuccess;
    return key_bits == 64 ? sah_level_t<uint64_t>(L, s) : sah_level_t<uint32_t>(L, s);
}

namespace {
rg_status sah_cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky launch error
    return report_error(e == cudaErrorMemoryAllocation ? RG_ERR_OOM : RG_ERR_CUDA,
                        (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}
}  // namespace

#define SAH_CK(call)                                             \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return sah_cuda_fail(e_, #call);  \
    } while (0)

// Binned-SAH topology (RG_BLAS_SAH): the LBVH's Morton sort, then
// levels of SAH splits over the segments of more than kSahSmall triangles
// (one host round trip per level for the left counts), then the Karras
// hierarchy inside every remaining segment.  Same outputs as lbvh_topology.
rg_status sah_topology(const ScratchAlloc& tmp, const float* lohi, uint32_t n, const int* cb_ord, int bits, float4* nodes,
                       uint32_t* perm, uint32_t* parents, cudaStream_t s, uint32_t* ranges) {
    const int key_bits = bits == 21 ? 64 : 32;
    const size_t kb = key_bits / 8;
    void *codes, *sorted, *vals, *scratch;
    rg_status r;
    if ((r = tmp.get(tmp.ctx, &codes, n * kb, "morton codes"))) return r;
    if ((r = tmp.get(tmp.ctx, &sorted, n * kb, "sorted codes"))) return r;
    if ((r = tmp.get(tmp.ctx, &vals, n * 4ull, "sort values"))) return r;
    if ((r = tmp.get(tmp.ctx, &scratch, radix_sort_scratch_bytes(n, key_bits), "sort scratch"))) return r;
    SAH_CK(launch_morton(lohi, n, cb_ord, bits, codes, static_cast<uint32_t*>(vals), nullptr, s));
    SAH_CK(radix_sort_pairs(codes, static_cast<uint32_t*>(vals), n, key_bits, sorted, perm, scratch, s));
    if (n <= kSahSmall) {
        SAH_CK(launch_karras(sorted, n, key_bits, reinterpret_cast<uint32_t*>(nodes) + 12, 16, parents, s, ranges));
        return RG_OK;
    }
    // a level's segments go through the kernels in slices of at most
    // kSahSliceTasks, which bounds the bins' scratch (1,368 B per segment)
    const uint32_t max_tasks = std::min(n / (kSahSmall + 1) + 1, kSahSliceTasks);
    const uint32_t max_blocks = n / kSahChunk + max_tasks;
    void *prim_out, *key_out, *d_tasks, *d_blk, *acc, *par, *blk_left, *blk_off, *out_nl;
    if ((r = tmp.get(tmp.ctx, &prim_out, n * 4ull, "SAH positions")) || (r = tmp.get(tmp.ctx, &key_out, n * kb, "SAH keys")) ||
        (r = tmp.get(tmp.ctx, &d_tasks, (size_t)max_tasks * sizeof(SahTask), "SAH tasks")) ||
        (r = tmp.get(tmp.ctx, &d_blk, (size_t)max_blocks * sizeof(uint2), "SAH blocks")) ||
        (r = tmp.get(tmp.ctx, &acc, (size_t)max_tasks * kSahAccInts * 4, "SAH bins")) ||
        (r = tmp.get(tmp.ctx, &par, (size_t)max_tasks * sizeof(SahParam), "SAH splits")) ||
        (r = tmp.get(tmp.ctx, &blk_left, (size_t)max_blocks * 4, "SAH block counts")) ||
        (r = tmp.get(tmp.ctx, &blk_off, (size_t)max_blocks * 4, "SAH block offsets")) ||
        (r = tmp.get(tmp.ctx, &out_nl, (size_t)max_tasks * 4, "SAH left counts")))
        return r;
    std::vector<SahTask> tasks(1);
    tasks[0] = SahTask{0u, n, 0u, 0u, 0u, {0u, 0u, 0u}};
    std::vector<KarrasSeg> segs;
    uint32_t seg_threads = 0;
    std::vector<uint2> blk;
    std::vector<uint32_t> nl;
    std::vector<SahTask> next;
    for (uint32_t level = 0; !tasks.empty(); ++level) {
        next.clear();
        for (size_t t0 = 0; t0 < tasks.size(); t0 += kSahSliceTasks) {
            const uint32_t m = (uint32_t)std::min(tasks.size() - t0, (size_t)kSahSliceTasks);
            SahTask* slice = tasks.data() + t0;
            blk.clear();
            for (uint32_t t = 0; t < m; ++t) {
                slice[t].first_block = (uint32_t)blk.size();
                for (uint32_t p = slice[t].begin; p < slice[t].begin + slice[t].count; p += kSahChunk)
                    blk.push_back(make_uint2(t, p));
                slice[t].n_blocks = (uint32_t)blk.size() - slice[t].first_block;
            }
            SAH_CK(cudaMemcpyAsync(d_tasks, slice, m * sizeof(SahTask), cudaMemcpyHostToDevice, s));
            SAH_CK(cudaMemcpyAsync(d_blk, blk.data(), blk.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
            SahLevel L{};
            L.lohi = lohi;
            L.n_leaves = n;
            L.m = m;
            L.n_blocks = (uint32_t)blk.size();
            L.tasks = static_cast<const SahTask*>(d_tasks);
            L.blk = static_cast<const uint2*>(d_blk);
            L.acc = static_cast<int*>(acc);
            L.par = static_cast<SahParam*>(par);
            L.prim_at = perm;
            L.key_at = sorted;
            L.prim_out = static_cast<uint32_t*>(prim_out);
            L.key_out = key_out;
            L.blk_left = static_cast<uint32_t*>(blk_left);
            L.blk_off = static_cast<uint32_t*>(blk_off);
            L.out_nl = static_cast<uint32_t*>(out_nl);
            L.nodes = nodes;
            L.parents = parents;
            L.ranges = ranges;
            SAH_CK(launch_sah_level(L, key_bits, s));
            nl.resize(m);
            SAH_CK(cudaMemcpyAsync(nl.data(), out_nl, m * 4ull, cudaMemcpyDeviceToHost, s));
            SAH_CK(cudaStreamSynchronize(s));
            auto child = [&](uint32_t b, uint32_t c, uint32_t node) {
                if (c <= 1) return;
                if (c <= kSahSmall || level + 1 >= kSahMaxLevels) {
                    segs.push_back(KarrasSeg{b, c, node, seg_threads});
                    seg_threads += c - 1;
                } else {
                    next.push_back(SahTask{b, c, node, 0u, 0u, {0u, 0u, 0u}});
                }
            };
            for (uint32_t t = 0; t < m; ++t) {
                const SahTask& T = slice[t];
                child(T.begin, nl[t], T.node + 1);
                child(T.begin + nl[t], T.count - nl[t], T.node + nl[t]);
            }
        }
        tasks.swap(next);
    }
    if (!segs.empty()) {
        void* d_segs;
        if ((r = tmp.get(tmp.ctx, &d_segs, segs.size() * sizeof(KarrasSeg), "Karras segments"))) return r;
        SAH_CK(cudaMemcpyAsync(d_segs, segs.data(), segs.size() * sizeof(KarrasSeg), cudaMemcpyHostToDevice, s));
        SAH_CK(launch_karras_segments(sorted, key_bits, static_cast<const KarrasSeg*>(d_segs), (uint32_t)segs.size(),
                                     seg_threads, n, nodes, parents, ranges, s));
    }
    return RG_OK;
}


rg_status sah_one_topology(const ScratchAlloc& tmp, const float* lohi, uint32_t n, const int* cb_ord, int bits,
                           float4* nodes, uint32_t* perm, uint32_t* parents, cudaStream_t s, uint32_t* ranges,
                           uint32_t* boxes_done) {
    if (bits != 10) return report_error(RG_ERR_INVALID_ARG, "the small SAH build takes 30-bit Morton codes");
    void *codes, *keys, *perm0, *rank, *pending, *n_pending;
    rg_status r;
    if ((r = tmp.get(tmp.ctx, &codes, n * 4ull, "morton codes"))) return r;
    if ((r = tmp.get(tmp.ctx, &keys, n * 4ull, "sorted codes"))) return r;
    if ((r = tmp.get(tmp.ctx, &perm0, n * 4ull, "Morton order"))) return r;
    if ((r = tmp.get(tmp.ctx, &rank, n * 4ull, "SAH ranks"))) return r;
    if ((r = tmp.get(tmp.ctx, &pending, (size_t)(n / 3 + 1) * 16, "SAH pending segments"))) return r;
    if ((r = tmp.get(tmp.ctx, &n_pending, 16, "SAH pending count"))) return r;
    SahSmallScratch w{static_cast<uint32_t*>(keys), static_cast<uint32_t*>(perm0), static_cast<uint32_t*>(rank),
                      pending, static_cast<uint32_t*>(n_pending), boxes_done};
    SAH_CK(launch_morton(lohi, n, cb_ord, bits, codes, nullptr, nullptr, s));
    SAH_CK(launch_sah_small(lohi, n, static_cast<const uint32_t*>(codes), perm, nodes, parents, ranges, w, s));
    return RG_OK;
}

}  // namespace rg
