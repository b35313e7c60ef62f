// LBVH construction of the two-level acceleration structure (paper Sec. 1:
// the two-layered structure built from vertices and transformation matrices).
//
// Bottom level, per mesh: triangle boxes and centroid bounds -> Morton codes
// -> stable LSD radix sort -> Karras (HPG 2012) hierarchy -> bottom-up box
// refit with one atomic flag per node (second arriver proceeds).  Top level:
// float64 inverse of each instance transform, Arvo (Graphics Gems 1990) world
// box with directed rounding, then the same LBVH steps over instance boxes.
//
// Every float32 operation that decides a Morton code or a box is an explicit
// round-to-nearest (or directed) intrinsic, so no FMA contraction can change
// a result: codes, order, topology and boxes are reproducible bit for bit.
#include "karras.cuh"
#include "rg_internal.cuh"

namespace rg {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ uint64_t spread21(uint64_t x) {
    x &= 0x1FFFFFull;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// warp-level min/max of ordered ints, one atomic per warp
__device__ __forceinline__ void reduce_bounds(int* cb_ord, int c0, int c1, int c2, bool valid) {
    int mn[3] = {valid ? c0 : INT_MAX, valid ? c1 : INT_MAX, valid ? c2 : INT_MAX};
    int mx[3] = {valid ? c0 : INT_MIN, valid ? c1 : INT_MIN, valid ? c2 : INT_MIN};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], off));
            mx[a] = max(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], off));
        }
    }
    if ((threadIdx.x & 31) == 0 && mn[0] != INT_MAX) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(cb_ord + a, mn[a]);
            atomicMax(cb_ord + 3 + a, mx[a]);
        }
    }
}

__device__ __forceinline__ float centroid(float lo, float hi) { return __fmul_rn(__fadd_rn(lo, hi), 0.5f); }

__global__ void k_init_bounds(int* cb_ord) {
    int t = threadIdx.x;
    if (t < 3) cb_ord[t] = f2ord(__int_as_float(0x7F800000));        // +inf
    else if (t < 6) cb_ord[t] = f2ord(__int_as_float(0xFF800000));   // -inf
}

__global__ void k_tri_bounds(const float* __restrict__ vtx, uint32_t nv, const uint32_t* __restrict__ idx,
                             uint32_t nt, float* __restrict__ lohi, int* cb_ord, DevStatus* st) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < nt;
    int c[3] = {0, 0, 0};
    if (valid) {
        uint32_t a = idx[3 * (size_t)i], b = idx[3 * (size_t)i + 1], cc = idx[3 * (size_t)i + 2];
        if (a >= nv || b >= nv || cc >= nv) {
            record_error(st, RG_ERR_INVALID_ARG);
            a = b = cc = 0;
        }
        float lo[3], hi[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float x0 = vtx[3 * (size_t)a + ax], x1 = vtx[3 * (size_t)b + ax], x2 = vtx[3 * (size_t)cc + ax];
            lo[ax] = fminf(fminf(x0, x1), x2);
            hi[ax] = fmaxf(fmaxf(x0, x1), x2);
            lohi[6 * (size_t)i + ax] = lo[ax];
            lohi[6 * (size_t)i + 3 + ax] = hi[ax];
            c[ax] = f2ord(centroid(lo[ax], hi[ax]));
        }
    }
    if (cb_ord) reduce_bounds(cb_ord, c[0], c[1], c[2], valid);
}

__global__ void k_centroid_bounds(const float* __restrict__ lohi, uint32_t n, int* cb_ord) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    int c[3] = {0, 0, 0};
    if (valid) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) c[ax] = f2ord(centroid(lohi[6 * (size_t)i + ax], lohi[6 * (size_t)i + 3 + ax]));
    }
    reduce_bounds(cb_ord, c[0], c[1], c[2], valid);
}

// Morton quantisation on one cubic grid over the centroid box: a single scale
// for all axes, so a flat mesh keeps its thin axis thin instead of being
// split across it first.
struct MortonGrid {
    float cmin[3], cmax[3], scale;
};

__device__ __forceinline__ MortonGrid morton_grid(const int* cb_ord, int bits) {
    MortonGrid g;
    const float full = (float)(1u << bits);
    float ext = 0.0f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        g.cmin[ax] = ord2f(cb_ord[ax]);
        g.cmax[ax] = ord2f(cb_ord[3 + ax]);
        if (g.cmax[ax] > g.cmin[ax]) ext = fmaxf(ext, __fsub_rn(g.cmax[ax], g.cmin[ax]));
    }
    g.scale = ext > 0.0f ? __fdiv_rn(full, ext) : 0.0f;
    return g;
}

// Quantised centroid of box b (lo.xyz, hi.xyz).
template <int BITS>
__device__ __forceinline__ void morton_q(const MortonGrid& g, const float* b, uint32_t* q) {
    const float qmax = (float)((1u << BITS) - 1u);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (!(g.cmax[ax] > g.cmin[ax])) {
            q[ax] = 0;
            continue;
        }
        float c = centroid(b[ax], b[3 + ax]);
        float f = floorf(__fmul_rn(__fsub_rn(c, g.cmin[ax]), g.scale));
        f = fminf(fmaxf(f, 0.0f), qmax);
        q[ax] = (uint32_t)f;
    }
}

__device__ __forceinline__ uint32_t morton30(const MortonGrid& g, const float* b) {
    uint32_t q[3];
    morton_q<10>(g, b, q);
    return (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
}

template <int BITS>
__global__ void k_morton(const float* __restrict__ lohi, uint32_t n, const int* __restrict__ cb_ord,
                         void* __restrict__ codes, uint32_t* __restrict__ vals, float* cb_out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const MortonGrid g = morton_grid(cb_ord, BITS);
    if (cb_out && i == 0) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            cb_out[ax] = g.cmin[ax];
            cb_out[3 + ax] = g.cmax[ax];
        }
    }
    if (i >= n) return;
    if (BITS == 10) {
        static_cast<uint32_t*>(codes)[i] = morton30(g, lohi + 6 * (size_t)i);
    } else {
        uint32_t q[3];
        morton_q<21>(g, lohi + 6 * (size_t)i, q);
        static_cast<uint64_t*>(codes)[i] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    }
    if (vals) vals[i] = i;
}

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort, 8-bit digits.  Per pass: (1) per-tile digit counts,
// (2) one exclusive scan over the digit-major count table, (3) a stable
// scatter: ranks inside a tile come from __match_any_sync peer groups per warp
// plus a per-digit prefix over the warps, processed in tile order.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_rs_count(const K* __restrict__ keys, uint32_t n, int shift,
                                                            uint32_t* __restrict__ hist, uint32_t nblocks) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        size_t i = base + (size_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Single-block exclusive scan of m counts, in place.
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ hist, uint32_t m) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (uint32_t base = 0; base < m; base += 1024u * 4u) {
        uint32_t v[4];
        uint32_t i0 = base + threadIdx.x * 4u;
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < m) ? hist[i0 + k] : 0u;
            uint32_t t = v[k];
            v[k] = sum;
            sum += t;
        }
        // inclusive warp scan of per-thread sums
        uint32_t x = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_sums[lane];
            uint32_t z = w;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, off);
                if (lane >= off) z += y;
            }
            warp_sums[lane] = z - w;  // exclusive
        }
        __syncthreads();
        uint32_t carry = carry_s;
        uint32_t excl = carry + warp_sums[warp] + (x - sum);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < m) hist[i0 + k] = excl + v[k];
        __syncthreads();
        if (threadIdx.x == 1023) carry_s = excl + sum;
        __syncthreads();
    }
}

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                              uint32_t n, int shift, const uint32_t* __restrict__ hist,
                                                              uint32_t nblocks, K* __restrict__ keys_out,
                                                              uint32_t* __restrict__ vals_out) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_wc[kWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_off[tid] = hist[(size_t)tid * nblocks + blockIdx.x];
    s_run[tid] = 0;
    const uint32_t lt_mask = (1u << lane) - 1u;
    size_t base = (size_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        size_t i = base + (size_t)r * kSortThreads + tid;
        bool valid = i < n;
        K key = valid ? keys[i] : K(0);
        uint32_t val = valid ? vals[i] : 0u;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & 0xFFu) : 256u;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s_wc[w][tid] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t rank = __popc(peers & lt_mask);
        if (valid && lane == __ffs(peers) - 1) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t sum = s_run[tid];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                uint32_t t = s_wc[w][tid];
                s_wc[w][tid] = sum;
                sum += t;
            }
            s_run[tid] = sum;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_off[d] + s_wc[warp][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- Karras
// (delta, karras_node: karras.cuh)

// One thread per internal node of all segments: the segment by binary search
// over the segments' first thread numbers.
template <class K>
__global__ void k_karras_segments(const K* __restrict__ keys, const KarrasSeg* __restrict__ segs, uint32_t n_segs,
                                  uint32_t n_threads, uint32_t n_leaves, uint32_t* __restrict__ child_base,
                                  uint32_t* __restrict__ parents, uint32_t* __restrict__ ranges) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_threads) return;
    uint32_t lo = 0, hi = n_segs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (segs[mid].first <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    const KarrasSeg S = segs[lo];
    karras_node(keys + S.begin, S.count, (int64_t)(g - S.first), child_base, 16, parents, ranges, S.node, S.begin,
                n_leaves);
}

template <class K>
__global__ void k_karras(const K* __restrict__ keys, uint32_t n, uint32_t* __restrict__ child_base, int stride,
                         uint32_t* __restrict__ parents, uint32_t* __restrict__ ranges) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n - 1) return;
    karras_node(keys, n, i, child_base, stride, parents, ranges);
}

// ---------------------------------------------------------------- refit
// Write one child box into slot `side` of node p (see the node layout).
__device__ __forceinline__ void store_slot(float4* nodes, uint32_t p, int side, const float* b) {
    float* f = reinterpret_cast<float*>(nodes + 4 * (size_t)p);
    if (side == 0) {
        *reinterpret_cast<float4*>(f) = make_float4(b[0], b[1], b[2], b[3]);
        *reinterpret_cast<float2*>(f + 4) = make_float2(b[4], b[5]);
    } else {
        *reinterpret_cast<float2*>(f + 6) = make_float2(b[0], b[1]);
        *reinterpret_cast<float4*>(f + 8) = make_float4(b[2], b[3], b[4], b[5]);
    }
}
__device__ __forceinline__ void load_slot_cg(const float4* nodes, uint32_t p, int side, float* b) {
    const float* f = reinterpret_cast<const float*>(nodes + 4 * (size_t)p);
    if (side == 0) {
        float4 x = __ldcg(reinterpret_cast<const float4*>(f));
        float2 y = __ldcg(reinterpret_cast<const float2*>(f + 4));
        b[0] = x.x; b[1] = x.y; b[2] = x.z; b[3] = x.w; b[4] = y.x; b[5] = y.y;
    } else {
        float2 x = __ldcg(reinterpret_cast<const float2*>(f + 6));
        float4 y = __ldcg(reinterpret_cast<const float4*>(f + 8));
        b[0] = x.x; b[1] = x.y; b[2] = y.x; b[3] = y.y; b[4] = y.z; b[5] = y.w;
    }
}

// Climb from leaf j to the root; the second thread to reach a node unions its
// two child boxes and continues.  Writes the root box to root_box (6 floats).
__device__ void climb(uint32_t j, uint32_t n, float* box, const uint32_t* __restrict__ parents, float4* nodes,
                      uint32_t* flags, float* root_box, DevStatus* st) {
    if (n == 1) {
        for (int a = 0; a < 6; ++a) root_box[a] = box[a];
        return;
    }
    uint32_t cur = kLeaf | j;
    uint32_t p = parents[(size_t)(n - 1) + j];
    for (uint32_t step = 0; step < n; ++step) {
        const uint32_t* n3 = reinterpret_cast<const uint32_t*>(nodes + 4 * (size_t)p + 3);
        int side = (n3[0] == cur) ? 0 : 1;
        store_slot(nodes, p, side, box);
        __threadfence();
        uint32_t old = atomicAdd(flags + p, 1u);
        if (old == 0) return;
        __threadfence();
        float other[6];
        load_slot_cg(nodes, p, 1 - side, other);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            box[a] = fminf(box[a], other[a]);
            box[3 + a] = fmaxf(box[3 + a], other[3 + a]);
        }
        if (p == 0) {
            for (int a = 0; a < 6; ++a) root_box[a] = box[a];
            return;
        }
        cur = p;
        p = parents[p];
    }
    record_error(st, RG_ERR_TIMEOUT);
}

__global__ void k_blas_leaves_refit(const float* __restrict__ vtx, const uint32_t* __restrict__ idx,
                                    const uint32_t* __restrict__ perm, const float* __restrict__ lohi, uint32_t n,
                                    const uint32_t* __restrict__ parents, float4* nodes, uint32_t* flags,
                                    float4* __restrict__ tris, BlasDev* blas_out, DevStatus* st) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t prim = perm[j];
    uint32_t vi[3] = {idx[3 * (size_t)prim], idx[3 * (size_t)prim + 1], idx[3 * (size_t)prim + 2]};
    // the triangle record: its vertices in the axis orders (x, y, z), (y, z, x)
    // and (z, x, y), prim in the first vertex's w of each
    float4* t = tris + 9 * (size_t)j;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float x = vtx[3 * (size_t)vi[c]], y = vtx[3 * (size_t)vi[c] + 1], z = vtx[3 * (size_t)vi[c] + 2];
        const float w = c == 0 ? __uint_as_float(prim) : 0.0f;
        t[c] = make_float4(x, y, z, w);
        t[3 + c] = make_float4(y, z, x, w);
        t[6 + c] = make_float4(z, x, y, w);
    }
    float box[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) box[a] = lohi[6 * (size_t)prim + a];
    climb(j, n, box, parents, nodes, flags, blas_out->lo, st);
}

// check_blas: a refit; the BLAS id of instance k must equal the one stored in
// tmp[k] by the build (read before tmp[k] is overwritten by the same thread).
// Bounding sphere: the largest upward-rounded squared distance of a vertex
// from the root box centre, reduced per warp, one atomicMax per warp.
__global__ void k_bound_sphere(const float* __restrict__ vtx, uint32_t nv, BlasDev* blas) {
    float c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) c[q] = __fmul_rn(__fadd_rn(blas->lo[q], blas->hi[q]), 0.5f);
    uint32_t best = 0;  // bits of a non-negative float: integer order = float order
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        float e[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float x = vtx[3 * (size_t)v + q];
            e[q] = x >= c[q] ? __fsub_ru(x, c[q]) : __fsub_ru(c[q], x);
        }
        const float d2 = __fadd_ru(__fadd_ru(__fmul_ru(e[0], e[0]), __fmul_ru(e[1], e[1])), __fmul_ru(e[2], e[2]));
        best = max(best, __float_as_uint(d2));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(0xFFFFFFFFu, best, off));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&blas->r2_bits, best);
}

// Instance k: float64 inverse, InstDev record into tmp[k], world box into
// wbox[k]; c receives the box centroid as ordered ints.
__device__ __forceinline__ void instance_prep_one(const rg_instance* __restrict__ in, uint32_t k,
                                                  const BlasDev* __restrict__ blas, uint32_t nblas, InstDev* tmp,
                                                  float* __restrict__ wbox, bool check_blas, DevStatus* st, int* c) {
    {
        const rg_instance& I = in[k];
        float m[12];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) m[4 * r + q] = I.m[r][q];
        uint32_t b = I.blas_id;
        if (b >= nblas || (check_blas && tmp[k].blas != b)) {
            record_error(st, RG_ERR_INVALID_ARG);
            b = 0;
        }
        const BlasDev B = blas[b];
        // float64 inverse of A = m[0..2 | 4..6 | 8..10]: adjugate / det
        double a0 = m[0], a1 = m[1], a2 = m[2], a3 = m[4], a4 = m[5], a5 = m[6], a6 = m[8], a7 = m[9], a8 = m[10];
        double c00 = a4 * a8 - a5 * a7, c01 = -(a3 * a8 - a5 * a6), c02 = a3 * a7 - a4 * a6;
        double det = a0 * c00 + a1 * c01 + a2 * c02;
        double inv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (det == 0.0 || !isfinite(det)) {
            record_error(st, RG_ERR_SINGULAR);
        } else {
            double id = 1.0 / det;
            inv[0] = c00 * id;
            inv[1] = -(a1 * a8 - a2 * a7) * id;
            inv[2] = (a1 * a5 - a2 * a4) * id;
            inv[3] = c01 * id;
            inv[4] = (a0 * a8 - a2 * a6) * id;
            inv[5] = -(a0 * a5 - a2 * a3) * id;
            inv[6] = c02 * id;
            inv[7] = -(a0 * a7 - a1 * a6) * id;
            inv[8] = (a0 * a4 - a1 * a3) * id;
        }
        InstDev D;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            double tr = -(inv[3 * r] * (double)m[3] + inv[3 * r + 1] * (double)m[7] + inv[3 * r + 2] * (double)m[11]);
            D.inv[r] = make_float4(__double2float_rn(inv[3 * r]), __double2float_rn(inv[3 * r + 1]),
                                   __double2float_rn(inv[3 * r + 2]), __double2float_rn(tr));
            D.m[r] = make_float4(m[4 * r], m[4 * r + 1], m[4 * r + 2], m[4 * r + 3]);
        }
        D.nodes = B.nodes;
        D.tris = B.tris;
        D.root = B.root;
        D.id = k;
        D.material = I.material_id;
        D.blas = b;
        tmp[k] = D;
        // Arvo box of the BLAS root box, outward rounded
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float mn = fminf(__fmul_rd(m[4 * r + q], B.lo[q]), __fmul_rd(m[4 * r + q], B.hi[q]));
                float mx = fmaxf(__fmul_ru(m[4 * r + q], B.lo[q]), __fmul_ru(m[4 * r + q], B.hi[q]));
                lo = q == 0 ? mn : __fadd_rd(lo, mn);
                hi = q == 0 ? mx : __fadd_ru(hi, mx);
            }
            lo = __fadd_rd(lo, m[4 * r + 3]);
            hi = __fadd_ru(hi, m[4 * r + 3]);
            // intersect with the box of the transformed bounding sphere:
            // A c + t -/+ r |row_r(A)|, outward rounded (a rotation leaves a
            // sphere's box unchanged, where it inflates the Arvo box)
            const float* row = m + 4 * r;
            float cx[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) cx[q] = __fmul_rn(__fadd_rn(B.lo[q], B.hi[q]), 0.5f);
            float cl = __fadd_rd(__fadd_rd(__fadd_rd(__fmul_rd(row[0], cx[0]), __fmul_rd(row[1], cx[1])),
                                           __fmul_rd(row[2], cx[2])), row[3]);
            float ch = __fadd_ru(__fadd_ru(__fadd_ru(__fmul_ru(row[0], cx[0]), __fmul_ru(row[1], cx[1])),
                                           __fmul_ru(row[2], cx[2])), row[3]);
            const float norm = __fsqrt_ru(__fadd_ru(__fadd_ru(__fmul_ru(row[0], row[0]), __fmul_ru(row[1], row[1])),
                                                    __fmul_ru(row[2], row[2])));
            const float R = __fmul_ru(__fsqrt_ru(__uint_as_float(B.r2_bits)), norm);
            lo = fmaxf(lo, __fsub_rd(cl, R));
            hi = fminf(hi, __fadd_ru(ch, R));
            wbox[6 * (size_t)k + r] = lo;
            wbox[6 * (size_t)k + 3 + r] = hi;
            c[r] = f2ord(centroid(lo, hi));
        }
    }
}

__global__ void k_instance_prep(const rg_instance* __restrict__ in, uint32_t n, const BlasDev* __restrict__ blas,
                                uint32_t nblas, InstDev* tmp, float* __restrict__ wbox, int* cb_ord, bool check_blas,
                                DevStatus* st) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = k < n;
    int c[3] = {0, 0, 0};
    if (valid) instance_prep_one(in, k, blas, nblas, tmp, wbox, check_blas, st, c);
    if (cb_ord) reduce_bounds(cb_ord, c[0], c[1], c[2], valid);
}

__global__ void k_tlas_leaves_refit(const InstDev* __restrict__ tmp, const float* __restrict__ wbox,
                                    const uint32_t* __restrict__ perm, uint32_t n, const uint32_t* __restrict__ parents,
                                    float4* nodes, uint32_t* flags, InstDev* __restrict__ inst_out, DevStatus* st,
                                    const uint32_t* __restrict__ boxes_done) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t k = perm[j];
    inst_out[j] = tmp[k];
    if (boxes_done && *boxes_done) return;
    float box[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) box[a] = wbox[6 * (size_t)k + a];
    float root_box[6];
    climb(j, n, box, parents, nodes, flags, root_box, st);
}

// The whole TLAS build (or refit) of up to kTlasSmallMax instances in one
// block, thread k = instance k: instance prep, centroid bounds, Morton codes,
// a stable sort, the Karras hierarchy and the bottom-up box refit.  Same
// per-element code and the same results as the multi-kernel path; a small
// TLAS is otherwise bound by the issue of its 17 launches.  The sort is an
// LSD sort by single bits (30 stable splits, each a block-wide prefix count
// of zeros), which starting from instance order gives the (key, index) order.
__global__ void __launch_bounds__(kTlasSmallMax) k_tlas_small(const rg_instance* __restrict__ in, uint32_t n,
                                                              const BlasDev* __restrict__ blas, uint32_t nblas,
                                                              InstDev* tmp, float* wbox, bool refit, float4* nodes,
                                                              uint32_t* perm, uint32_t* parents, uint32_t* flags,
                                                              uint32_t* ranges, InstDev* inst_out, DevStatus* st) {
    __shared__ int s_cb[6];
    __shared__ uint32_t s_key[kTlasSmallMax], s_val[kTlasSmallMax];
    __shared__ uint32_t s_warp[32], s_total;
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t n_warps = blockDim.x >> 5;
    const bool valid = t < n;
    if (t < 3) s_cb[t] = f2ord(__int_as_float(0x7F800000));
    else if (t < 6) s_cb[t] = f2ord(__int_as_float(0xFF800000));
    __syncthreads();
    int c[3] = {INT_MAX, INT_MAX, INT_MAX};
    if (valid) instance_prep_one(in, t, blas, nblas, tmp, wbox, refit, st, c);
    if (!refit) {
        int mn[3] = {c[0], c[1], c[2]}, mx[3] = {valid ? c[0] : INT_MIN, valid ? c[1] : INT_MIN, valid ? c[2] : INT_MIN};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                mn[a] = min(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], off));
                mx[a] = max(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], off));
            }
        if (lane == 0 && mn[0] != INT_MAX)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                atomicMin(s_cb + a, mn[a]);
                atomicMax(s_cb + 3 + a, mx[a]);
            }
        __syncthreads();
        const MortonGrid g = morton_grid(s_cb, 10);
        if (valid) {
            float b[6];
#pragma unroll
            for (int a = 0; a < 6; ++a) b[a] = wbox[6 * (size_t)t + a];
            s_key[t] = morton30(g, b);
            s_val[t] = t;
        }
        // stable LSD sort by single bits
        for (int bit = 0; bit < 30; ++bit) {
            __syncthreads();
            const uint32_t k = valid ? s_key[t] : 0u, v = valid ? s_val[t] : 0u;
            const bool zero = valid && !((k >> bit) & 1u);
            const uint32_t zb = __ballot_sync(0xFFFFFFFFu, zero);
            if (lane == 0) s_warp[warp] = __popc(zb);
            __syncthreads();
            if (warp == 0) {
                const uint32_t x = lane < n_warps ? s_warp[lane] : 0u;
                uint32_t inc = x;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, off);
                    if ((int)lane >= off) inc += y;
                }
                if (lane < n_warps) s_warp[lane] = inc - x;
                if (lane == 31) s_total = inc;
            }
            __syncthreads();
            // (every read of s_key in this pass came before the barrier above)
            const uint32_t zeros_before = s_warp[warp] + __popc(zb & ((1u << lane) - 1u));
            const uint32_t pos = zero ? zeros_before : s_total + (t - zeros_before);
            if (valid) {
                s_key[pos] = k;
                s_val[pos] = v;
            }
        }
        __syncthreads();
        if (valid) perm[t] = s_val[t];
        if (t + 1 < n) karras_node(s_key, n, t, reinterpret_cast<uint32_t*>(nodes) + 12, 16, parents, ranges);
    }
    if (t + 1 < n) flags[t] = 0;
    __syncthreads();
    __threadfence();
    if (valid) {
        const uint32_t k = perm[t];
        inst_out[t] = tmp[k];
        float box[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) box[a] = wbox[6 * (size_t)k + a];
        float root_box[6];
        climb(t, n, box, parents, nodes, flags, root_box, st);
    }
}

inline unsigned grid_for(size_t n, int block = kBlock) { return (unsigned)((n + block - 1) / block); }

}  // namespace

cudaError_t launch_init_bounds(int* cb_ord, cudaStream_t s) {
    k_init_bounds<<<1, 32, 0, s>>>(cb_ord);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tri_bounds(const float* vtx, uint32_t nv, const uint32_t* idx, uint32_t nt, float* lohi,
                              int* cb_ord, DevStatus* st, cudaStream_t s) {
    if (nt == 0) return cudaSuccess;
    k_tri_bounds<<<grid_for(nt), kBlock, 0, s>>>(vtx, nv, idx, nt, lohi, cb_ord, st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_centroid_bounds(const float* lohi, uint32_t n, int* cb_ord, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_centroid_bounds<<<grid_for(n), kBlock, 0, s>>>(lohi, n, cb_ord);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_morton(const float* lohi, uint32_t n, const int* cb_ord, int bits, void* codes, uint32_t* vals,
                          float* cb_out, cudaStream_t s) {
    unsigned g = grid_for(n > 0 ? n : 1);
    if (bits == 10)
        k_morton<10><<<g, kBlock, 0, s>>>(lohi, n, cb_ord, codes, vals, cb_out);
    else
        k_morton<21><<<g, kBlock, 0, s>>>(lohi, n, cb_ord, codes, vals, cb_out);
    count_launches(1);
    return cudaGetLastError();
}

static_assert(kSortTile == (int)kSortTilePairs, "sort tile size and scratch layout disagree");

template <class K>
static cudaError_t radix_sort_impl(const K* keys_in, const uint32_t* vals_in, uint32_t n, K* keys_out,
                                   uint32_t* vals_out, void* scratch, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int passes = (int)sizeof(K);
    uint32_t nb = (n + kSortTile - 1) / kSortTile;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* p = static_cast<char*>(scratch);
    K* kt = reinterpret_cast<K*>(p);
    p += al((size_t)n * sizeof(K));
    uint32_t* vt = reinterpret_cast<uint32_t*>(p);
    p += al((size_t)n * 4);
    uint32_t* hist = reinterpret_cast<uint32_t*>(p);
    // even pass count: in -> out -> tmp -> out ... ends in `out`
    const K* ksrc = keys_in;
    const uint32_t* vsrc = vals_in;
    for (int pass = 0; pass < passes; ++pass) {
        bool to_out = ((passes - pass) % 2) == 1;
        K* kdst = to_out ? keys_out : kt;
        uint32_t* vdst = to_out ? vals_out : vt;
        int shift = 8 * pass;
        k_rs_count<K><<<nb, kSortThreads, 0, s>>>(ksrc, n, shift, hist, nb);
        count_launches(1);
        k_rs_scan<<<1, 1024, 0, s>>>(hist, 256u * nb);
        count_launches(1);
        k_rs_scatter<K><<<nb, kSortThreads, 0, s>>>(ksrc, vsrc, n, shift, hist, nb, kdst, vdst);
        count_launches(1);
        ksrc = kdst;
        vsrc = vdst;
    }
    return cudaGetLastError();
}

cudaError_t radix_sort_pairs(const void* keys_in, const uint32_t* vals_in, uint32_t n, int key_bits, void* keys_out,
                             uint32_t* vals_out, void* scratch, cudaStream_t s) {
    if (key_bits == 64)
        return radix_sort_impl<uint64_t>(static_cast<const uint64_t*>(keys_in), vals_in, n,
                                         static_cast<uint64_t*>(keys_out), vals_out, scratch, s);
    return radix_sort_impl<uint32_t>(static_cast<const uint32_t*>(keys_in), vals_in, n,
                                     static_cast<uint32_t*>(keys_out), vals_out, scratch, s);
}

cudaError_t launch_karras(const void* keys, uint32_t n, int key_bits, uint32_t* child_base, int stride,
                          uint32_t* parents, cudaStream_t s, uint32_t* ranges) {
    if (n < 2) return cudaSuccess;
    if (key_bits == 64)
        k_karras<uint64_t><<<grid_for(n - 1), kBlock, 0, s>>>(static_cast<const uint64_t*>(keys), n, child_base, stride,
                                                              parents, ranges);
    else
        k_karras<uint32_t><<<grid_for(n - 1), kBlock, 0, s>>>(static_cast<const uint32_t*>(keys), n, child_base, stride,
                                                              parents, ranges);
    count_launches(1);
    return cudaGetLastError();
}

namespace {
__global__ void k_invert_perm(const uint32_t* __restrict__ perm, uint32_t n, uint32_t* __restrict__ inv) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) inv[perm[j]] = j;
}
}  // namespace

cudaError_t launch_karras_segments(const void* keys, int key_bits, const KarrasSeg* segs, uint32_t n_segs,
                                   uint32_t n_threads, uint32_t n_leaves, float4* nodes, uint32_t* parents,
                                   uint32_t* ranges, cudaStream_t s) {
    if (n_segs == 0 || n_threads == 0) return cudaSuccess;
    uint32_t* child_base = reinterpret_cast<uint32_t*>(nodes) + 12;
    if (key_bits == 64)
        k_karras_segments<uint64_t><<<grid_for(n_threads), kBlock, 0, s>>>(
            static_cast<const uint64_t*>(keys), segs, n_segs, n_threads, n_leaves, child_base, parents, ranges);
    else
        k_karras_segments<uint32_t><<<grid_for(n_threads), kBlock, 0, s>>>(
            static_cast<const uint32_t*>(keys), segs, n_segs, n_threads, n_leaves, child_base, parents, ranges);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_invert_perm(const uint32_t* perm, uint32_t n, uint32_t* inv, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_invert_perm<<<min(grid_for(n), 4096u), kBlock, 0, s>>>(perm, n, inv);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blas_leaves_refit(const float* vtx, const uint32_t* idx, const uint32_t* perm, const float* lohi,
                                     uint32_t n, const uint32_t* parents, float4* nodes, uint32_t* flags,
                                     float4* tris, BlasDev* blas_out, DevStatus* st, cudaStream_t s) {
    k_blas_leaves_refit<<<grid_for(n), kBlock, 0, s>>>(vtx, idx, perm, lohi, n, parents, nodes, flags, tris, blas_out,
                                                       st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bound_sphere(const float* vtx, uint32_t nv, BlasDev* blas, cudaStream_t s) {
    if (nv == 0) return cudaSuccess;
    const uint32_t blocks = (uint32_t)min((nv + 255u) / 256u, (uint32_t)device_sm_count() * 4u);
    k_bound_sphere<<<blocks, 256, 0, s>>>(vtx, nv, blas);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_instance_prep(const rg_instance* in, uint32_t n, const BlasDev* blas, uint32_t nblas,
                                 InstDev* tmp, float* wbox, int* cb_ord, bool check_blas, DevStatus* st,
                                 cudaStream_t s) {
    k_instance_prep<<<grid_for(n), kBlock, 0, s>>>(in, n, blas, nblas, tmp, wbox, cb_ord, check_blas, st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tlas_leaves_refit(const InstDev* tmp, const float* wbox, const uint32_t* perm, uint32_t n,
                                     const uint32_t* parents, float4* nodes, uint32_t* flags, InstDev* inst_out,
                                     DevStatus* st, cudaStream_t s, const uint32_t* boxes_done) {
    k_tlas_leaves_refit<<<grid_for(n), kBlock, 0, s>>>(tmp, wbox, perm, n, parents, nodes, flags, inst_out, st,
                                                       boxes_done);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tlas_small(const rg_instance* in, uint32_t n, const BlasDev* blas, uint32_t nblas, InstDev* tmp,
                              float* wbox, bool refit, float4* nodes, uint32_t* perm, uint32_t* parents,
                              uint32_t* flags, uint32_t* ranges, InstDev* inst_out, DevStatus* st, cudaStream_t s) {
    if (n == 0 || n > kTlasSmallMax) return cudaErrorInvalidValue;
    const uint32_t threads = (n + 31u) & ~31u;
    k_tlas_small<<<1, threads, 0, s>>>(in, n, blas, nblas, tmp, wbox, refit, nodes, perm, parents, flags, ranges,
                                       inst_out, st);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rg
