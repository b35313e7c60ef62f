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
#include <string>
#include <vector>

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

}  // namespace

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


}  // namespace rg
