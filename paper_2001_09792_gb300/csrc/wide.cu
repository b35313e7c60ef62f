// Compressed 8-wide BVH (the precision row of the method's growth: node boxes
// stored as 8-bit integers against a float32 parent frame, rounded outward so
// that the float32 triangle test still decides every hit).
//
// Collapse: each wide node is rooted at a node of the binary LBVH.  Starting
// from that node's two children, the child with the largest surface area is
// replaced by its two children until there are 8 or only leaves remain.  A
// child whose subtree holds at most leaf_max (<= kWideLeafMax) items becomes a leaf slot
// (its items are contiguous in LBVH order); every other child becomes a new
// wide node.  Children are assigned to slots by the octant of their centre
// relative to the node's centre (greedy, best match first), which lets the
// traversal visit them roughly front to back with one xor.  The whole
// collapse is one launch of one block: levels of the wide tree are separated
// by __syncthreads, so no host synchronisation is needed.
//
// Quantization: p = min over children of lo; per axis the scale 2^e is the
// smallest power of two with 255 * 2^e >= (max hi - p) rounded up; then
// qlo = floor((lo - p) rounded down / 2^e), qhi = ceil((hi - p) rounded up / 2^e).
// Division by 2^e is exact, so p + qlo 2^e <= lo and p + qhi 2^e >= hi hold
// in exact arithmetic.
#include "rg_internal.cuh"

namespace rg {

namespace {

constexpr int kCollapseThreads = 1024;
constexpr int kMaxLevels = 256;

__device__ __forceinline__ float area6(const float* b) {
    float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ void read_slot(const float4* nodes, uint32_t node, int side, float* b) {
    const float* f = reinterpret_cast<const float*>(nodes + 4 * (size_t)node);
    const int o = side == 0 ? 0 : 6;
#pragma unroll
    for (int a = 0; a < 6; ++a) b[a] = f[o + a];
}

__device__ __forceinline__ uint2 children_of(const float4* nodes, uint32_t node) {
    const uint32_t* c = reinterpret_cast<const uint32_t*>(nodes + 4 * (size_t)node + 3);
    return make_uint2(c[0], c[1]);
}

// smallest e in [-126, 127] with 255 * 2^e >= ext
__device__ int exp_for(float ext) {
    if (!(ext > 0.0f)) return -126;
    int e;
    frexpf(ext / 255.0f, &e);
    if (e < -126) e = -126;
    if (e > 127) e = 127;
    while (e > -126 && ldexpf(255.0f, e - 1) >= ext) --e;
    while (e < 127 && ldexpf(255.0f, e) < ext) ++e;
    return e;
}

__device__ void quantize_write(float4* out, uint32_t node, const float (*box)[6], const int* slot_of, int n,
                               uint32_t imask, const uint32_t* meta, uint32_t child_base, uint32_t item_base) {
    float p[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < n; ++j)
        for (int a = 0; a < 3; ++a) {
            p[a] = fminf(p[a], box[j][a]);
            mx[a] = fmaxf(mx[a], box[j][3 + a]);
        }
    int e[3];
    float inv_scale[3];
    for (int a = 0; a < 3; ++a) {
        e[a] = exp_for(__fsub_ru(mx[a], p[a]));
        inv_scale[a] = ldexpf(1.0f, -e[a]);
    }
    uint32_t qlo[3][2] = {{0, 0}, {0, 0}, {0, 0}}, qhi[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int j = 0; j < n; ++j) {
        const int s = slot_of[j];
        for (int a = 0; a < 3; ++a) {
            float lo = floorf(__fmul_rn(__fsub_rd(box[j][a], p[a]), inv_scale[a]));
            float hi = ceilf(__fmul_rn(__fsub_ru(box[j][3 + a], p[a]), inv_scale[a]));
            uint32_t ql = (uint32_t)fminf(fmaxf(lo, 0.0f), 255.0f);
            uint32_t qh = (uint32_t)fminf(fmaxf(hi, 0.0f), 255.0f);
            qlo[a][s >> 2] |= ql << (8 * (s & 3));
            qhi[a][s >> 2] |= qh << (8 * (s & 3));
        }
    }
    uint32_t bits = (uint32_t)(e[0] & 0xFF) | ((uint32_t)(e[1] & 0xFF) << 8) | ((uint32_t)(e[2] & 0xFF) << 16) |
                    (imask << 24);
    uint32_t m0 = 0, m1 = 0;
    for (int s = 0; s < 8; ++s) {
        if (s < 4) m0 |= meta[s] << (8 * s);
        else m1 |= meta[s] << (8 * (s - 4));
    }
    float4* w = out + 5 * (size_t)node;
    w[0] = make_float4(p[0], p[1], p[2], __uint_as_float(bits));
    w[1] = make_float4(__uint_as_float(child_base), __uint_as_float(item_base), __uint_as_float(m0), __uint_as_float(m1));
    w[2] = make_float4(__uint_as_float(qlo[0][0]), __uint_as_float(qlo[0][1]), __uint_as_float(qlo[1][0]),
                       __uint_as_float(qlo[1][1]));
    w[3] = make_float4(__uint_as_float(qlo[2][0]), __uint_as_float(qlo[2][1]), __uint_as_float(qhi[0][0]),
                       __uint_as_float(qhi[0][1]));
    w[4] = make_float4(__uint_as_float(qhi[1][0]), __uint_as_float(qhi[1][1]), __uint_as_float(qhi[2][0]),
                       __uint_as_float(qhi[2][1]));
}

// greedy octant slot assignment: slot bit a set = child centre on the negative side of axis a
__device__ void assign_slots(const float (*box)[6], int n, int* slot_of) {
    float pc[3] = {0, 0, 0};
    {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int j = 0; j < n; ++j)
            for (int a = 0; a < 3; ++a) {
                lo[a] = fminf(lo[a], box[j][a]);
                hi[a] = fmaxf(hi[a], box[j][3 + a]);
            }
        for (int a = 0; a < 3; ++a) pc[a] = 0.5f * (lo[a] + hi[a]);
    }
    float v[8][3];
    for (int j = 0; j < n; ++j)
        for (int a = 0; a < 3; ++a) v[j][a] = 0.5f * (box[j][a] + box[j][3 + a]) - pc[a];
    uint32_t used_slot = 0, done = 0;
    for (int k = 0; k < n; ++k) {
        float best = -INFINITY;
        int bj = -1, bs = -1;
        for (int j = 0; j < n; ++j) {
            if (done & (1u << j)) continue;
            for (int s = 0; s < 8; ++s) {
                if (used_slot & (1u << s)) continue;
                float sc = ((s & 1) ? -v[j][0] : v[j][0]) + ((s & 2) ? -v[j][1] : v[j][1]) + ((s & 4) ? -v[j][2] : v[j][2]);
                if (sc > best || bj < 0) {
                    best = sc;
                    bj = j;
                    bs = s;
                }
            }
        }
        slot_of[bj] = bs;
        used_slot |= 1u << bs;
        done |= 1u << bj;
    }
}

struct CollapseArgs {
    const float4* nodes2;
    const uint32_t* ranges;
    uint32_t n;
    const float* leaf_box;   // box of the only leaf when n == 1
    const float4* tris2;
    float4* tris8;
    const InstDev* inst2;
    InstDev* inst8;
    const BlasDev* blas;
    WideOut out;
    DevStatus* st;
    uint32_t leaf_max;
};

__device__ void copy_item(const CollapseArgs& a, uint32_t from, uint32_t to) {
    if (a.tris2) {
        const float4* t = a.tris2 + kTriStride * (size_t)from;
        float4* d = a.tris8 + kTriStride * (size_t)to;
#pragma unroll
        for (uint32_t c = 0; c < kTriStride; ++c) d[c] = t[c];
    } else {
        InstDev I = a.inst2[from];
        const BlasDev& B = a.blas[I.blas];
        I.nodes = B.nodes8;
        I.tris = B.tris8;
        I.root = 0;
        a.inst8[to] = I;
    }
    a.out.item_src[to] = from;
}

// One wide node for binary node `src` (kNone: the single leaf of a one-item tree).
__device__ void collapse_task(const CollapseArgs& a, uint32_t src, uint32_t dst, uint32_t* s_nodes, uint32_t* s_items,
                              uint2* tasks_out, uint32_t* s_out) {
    uint32_t ref[8];
    float box[8][6];
    int n = 0;
    if (src == kNone) {
        ref[0] = kLeaf | 0u;
        for (int c = 0; c < 6; ++c) box[0][c] = a.leaf_box[c];
        n = 1;
    } else {
        uint2 ch = children_of(a.nodes2, src);
        ref[0] = ch.x;
        ref[1] = ch.y;
        read_slot(a.nodes2, src, 0, box[0]);
        read_slot(a.nodes2, src, 1, box[1]);
        n = 2;
        while (n < 8) {
            int bj = -1;
            float ba = -1.0f;
            for (int j = 0; j < n; ++j) {
                if (ref[j] & kLeaf) continue;
                float ar = area6(box[j]);
                if (ar > ba) {
                    ba = ar;
                    bj = j;
                }
            }
            if (bj < 0) break;
            uint32_t c = ref[bj];
            uint2 cc = children_of(a.nodes2, c);
            ref[bj] = cc.x;
            read_slot(a.nodes2, c, 0, box[bj]);
            ref[n] = cc.y;
            read_slot(a.nodes2, c, 1, box[n]);
            ++n;
        }
    }
    // classify: leaf slots (<= leaf_max items) and internal slots
    uint32_t first[8], cnt[8];
    bool internal[8];
    uint32_t n_int = 0, n_items = 0;
    for (int j = 0; j < n; ++j) {
        if (ref[j] & kLeaf) {
            first[j] = ref[j] & ~kLeaf;
            cnt[j] = 1;
            internal[j] = false;
        } else {
            uint32_t f = a.ranges[2 * (size_t)ref[j]], l = a.ranges[2 * (size_t)ref[j] + 1];
            first[j] = f;
            cnt[j] = l - f + 1;
            internal[j] = cnt[j] > a.leaf_max;
        }
        if (internal[j]) ++n_int;
        else n_items += cnt[j];
    }
    int slot_of[8];
    assign_slots(box, n, slot_of);
    uint32_t child_base = n_int ? atomicAdd(s_nodes, n_int) : 0;
    uint32_t item_base = atomicAdd(s_items, n_items);
    // slot order: internal rank and leaf offsets follow increasing slot index
    int at_slot[8];
    for (int s = 0; s < 8; ++s) at_slot[s] = -1;
    for (int j = 0; j < n; ++j) at_slot[slot_of[j]] = j;
    uint32_t imask = 0, meta[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t rank = 0, off = 0;
    for (int s = 0; s < 8; ++s) {
        int j = at_slot[s];
        a.out.src[8 * (size_t)dst + s] = j < 0 ? kNone : ref[j];
        if (j < 0) continue;
        if (internal[j]) {
            imask |= 1u << s;
            uint32_t t = atomicAdd(s_out, 1u);
            tasks_out[t] = make_uint2(ref[j], child_base + rank);
            ++rank;
        } else {
            meta[s] = (cnt[j] << 5) | off;
            for (uint32_t k = 0; k < cnt[j]; ++k) copy_item(a, first[j] + k, item_base + off + k);
            off += cnt[j];
        }
    }
    quantize_write(a.out.nodes, dst, box, slot_of, n, imask, meta, child_base, item_base);
}

__global__ void __launch_bounds__(kCollapseThreads) k_collapse(CollapseArgs a) {
    __shared__ uint32_t s_in, s_out, s_nodes, s_items;
    uint2* tin = a.out.tasks;
    uint2* tout = a.out.tasks + a.n;
    if (threadIdx.x == 0) {
        tin[0] = make_uint2(a.n > 1 ? 0u : kNone, 0u);
        s_in = 1;
        s_nodes = 1;
        s_items = 0;
    }
    __syncthreads();
    for (int level = 0; level < kMaxLevels; ++level) {
        const uint32_t n_in = s_in;
        if (n_in == 0) break;
        __syncthreads();
        if (threadIdx.x == 0) s_out = 0;
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < n_in; t += blockDim.x) {
            uint2 task = tin[t];
            collapse_task(a, task.x, task.y, &s_nodes, &s_items, tout, &s_out);
        }
        __syncthreads();
        uint2* tmp = tin;
        tin = tout;
        tout = tmp;
        if (threadIdx.x == 0) s_in = s_out;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (s_in != 0) record_error(a.st, RG_ERR_TIMEOUT);
        a.out.counts[0] = s_nodes;
        a.out.counts[1] = s_items;
    }
}

// box of a binary-tree reference after a refit
__device__ void ref_box(const float4* nodes2, const float* wbox, const uint32_t* perm, uint32_t ref, float* b) {
    if (ref & kLeaf) {
        const float* w = wbox + 6 * (size_t)perm[ref & ~kLeaf];
        for (int c = 0; c < 6; ++c) b[c] = w[c];
    } else {
        float l[6], r[6];
        read_slot(nodes2, ref, 0, l);
        read_slot(nodes2, ref, 1, r);
        for (int c = 0; c < 3; ++c) {
            b[c] = fminf(l[c], r[c]);
            b[3 + c] = fmaxf(l[3 + c], r[3 + c]);
        }
    }
}

__global__ void k_wide_refit(const float4* nodes2, const float* wbox, const uint32_t* perm, uint32_t n,
                             const InstDev* inst2, InstDev* inst8, const BlasDev* blas, WideOut out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n_nodes = out.counts[0], n_items = out.counts[1];
    if (i < n_items) {
        InstDev I = inst2[out.item_src[i]];
        const BlasDev& B = blas[I.blas];
        I.nodes = B.nodes8;
        I.tris = B.tris8;
        I.root = 0;
        inst8[i] = I;
    }
    if (i >= n_nodes) return;
    float4* w = out.nodes + 5 * (size_t)i;
    const float4 w1 = w[1];
    const uint32_t imask = __float_as_uint(w[0].w) >> 24;
    const uint32_t m0 = __float_as_uint(w1.z), m1 = __float_as_uint(w1.w);
    float box[8][6];
    int slot_of[8];
    uint32_t meta[8];
    int n_used = 0;
    for (int s = 0; s < 8; ++s) {
        meta[s] = (s < 4 ? (m0 >> (8 * s)) : (m1 >> (8 * (s - 4)))) & 0xFF;
        uint32_t ref = out.src[8 * (size_t)i + s];
        if (ref == kNone) continue;
        if (n == 1) {
            for (int c = 0; c < 6; ++c) box[n_used][c] = wbox[c];
        } else {
            ref_box(nodes2, wbox, perm, ref, box[n_used]);
        }
        slot_of[n_used] = s;
        ++n_used;
    }
    quantize_write(out.nodes, i, box, slot_of, n_used, imask, meta, __float_as_uint(w1.x), __float_as_uint(w1.y));
}

}  // namespace

cudaError_t launch_collapse(const float4* nodes2, const uint32_t* ranges, uint32_t n, const float* leaf_box,
                            const float4* tris2, float4* tris8, const InstDev* inst2, InstDev* inst8,
                            const BlasDev* blas, const WideOut& out, DevStatus* st, cudaStream_t s,
                            uint32_t leaf_max) {
    CollapseArgs a;
    a.leaf_max = leaf_max < 1 ? 1u : (leaf_max > (uint32_t)kWideLeafMax ? (uint32_t)kWideLeafMax : leaf_max);
    a.nodes2 = nodes2;
    a.ranges = ranges;
    a.n = n;
    a.leaf_box = leaf_box;
    a.tris2 = tris2;
    a.tris8 = tris8;
    a.inst2 = inst2;
    a.inst8 = inst8;
    a.blas = blas;
    a.out = out;
    a.st = st;
    k_collapse<<<1, kCollapseThreads, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_wide_refit(const float4* nodes2, const float* wbox, const uint32_t* perm, uint32_t n,
                              const InstDev* inst2, InstDev* inst8, const BlasDev* blas, const WideOut& out,
                              DevStatus* st, cudaStream_t s) {
    (void)st;
    k_wide_refit<<<(n + 127) / 128, 128, 0, s>>>(nodes2, wbox, perm, n, inst2, inst8, blas, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rg
