// Ray traversal of the two-level BVH: closest-hit, any-hit and miss (paper
// Sec. 1: per ray, the closest-hit or any-hit shader runs when the ray meets a
// triangle, the miss shader when it meets none).
//
// Persistent warps pull rays from a global counter (32 at a time, or as lanes
// fall idle: k_trace_warp / k_trace_lane; k_trace_pair serves a renderer's
// shadow rays of one depth level and closest-hit rays of the next from one
// counter, in one launch).  Each thread runs a stack
// traversal: TLAS nodes in world space; at an instance leaf the
// ray is moved to object space with the instance's float32 inverse (t is
// shared, the direction is not renormalised), a marker is pushed, and the
// BLAS is traversed; popping the marker restores the world ray.  Nodes are
// 64 B (two child boxes), read with four 16 B loads; triangles are 48 B, read
// with three 16 B loads.
//
// Triangle test: the watertight test of Woop, Benthin & Wald (JCGT 2013) in
// float32, with every product and difference of the edge functions rounded
// separately (no FMA), so that a shared edge evaluates to exactly opposite
// values in its two triangles and no ray leaks through it.  Box test: slabs
// with the far distance scaled by 1 + 2*gamma_3 (Ize, "Robust BVH Ray
// Traversal", JCGT 2013), and a relative slack of 2^-12 on the culling
// distance, so that a box is never culled while a triangle inside it can
// still win.  Child order: nearer entry first for closest hit, longer
// overlap with the ray's segment first for any hit.  Ties in t are broken by (instance, prim), which makes the
// result independent of the visit order (BVH == brute force).
#include "rg_internal.cuh"

namespace rg {

namespace {

constexpr int kStack = 64;
constexpr uint32_t kMarker = 0xFFFFFFFEu;
constexpr int kTraceBlock = 128;
// 1 + 2 * gamma_3, gamma_3 = 3u / (1 - 3u), u = 2^-24
constexpr float kIze = 1.0f + 2.0f * (3.0f * 5.9604644775390625e-08f) / (1.0f - 3.0f * 5.9604644775390625e-08f);
constexpr float kCullSlack = 1.0f + 1.0f / 4096.0f;

// 1/d correctly rounded (the same value as the IEEE division 1/d): a zero
// component gives +-inf.
__device__ __forceinline__ float safe_rcp(float d) { return __frcp_rn(d); }

struct SpaceRay {
    float ox, oy, oz;
    float ix, iy, iz;
};

// Per-axis slab interval.  For a zero direction component the distances are
// +-inf, or NaN (0 * inf) when the origin lies on the slab plane.  The PTX
// min.NaN / max.NaN forms return NaN if either operand is NaN, and the
// fminf/fmaxf that combine the axes drop NaN, so an axis whose origin lies in
// the (closed) slab with d == 0 leaves the interval unconstrained, and one
// outside it makes the interval empty.
__device__ __forceinline__ float nan_min(float a, float b) {
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float nan_max(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz, const SpaceRay& r,
                                     float tmin, float tlim, float& tnear, float& tfar) {
    float t0x = __fmul_rn(__fsub_rn(lx, r.ox), r.ix), t1x = __fmul_rn(__fsub_rn(hx, r.ox), r.ix);
    float t0y = __fmul_rn(__fsub_rn(ly, r.oy), r.iy), t1y = __fmul_rn(__fsub_rn(hy, r.oy), r.iy);
    float t0z = __fmul_rn(__fsub_rn(lz, r.oz), r.iz), t1z = __fmul_rn(__fsub_rn(hz, r.oz), r.iz);
    float tn = fmaxf(fmaxf(nan_min(t0x, t1x), nan_min(t0y, t1y)), fmaxf(nan_min(t0z, t1z), tmin));
    float tf = fminf(fminf(nan_max(t0x, t1x), nan_max(t0y, t1y)), nan_max(t0z, t1z));
    tf = fminf(__fmul_rn(tf, kIze), tlim);
    tnear = tn;
    tfar = tf;
    return tn <= tf;
}

// Which of two hit children a ray visits first.  Closest hit: the nearer
// entry.  Any hit: the child whose box covers the longer stretch of the ray's
// segment (more likely to hold an occluder; on the medium frame's shadow
// rays this halves the nodes visited against nearest-first).
template <bool ANY>
__device__ __forceinline__ bool visit_first0(float tn0, float tf0, float tn1, float tf1) {
    return ANY ? (tf0 - tn0) >= (tf1 - tn1) : tn0 <= tn1;
}


// Watertight-test state of the object-space ray.
struct Shear {
    float ox, oy, oz;  // origin in the axis order (kx, ky, kz)
    float Sx, Sy, Sz;
    uint32_t order;    // which order of the triangle records: 0 (x, y, z), 1 (y, z, x), 2 (z, x, y)
};

// Shear of the watertight test: kz is the dominant axis of the direction,
// (kx, ky, kz) the cyclic order ending in it; Sz = 1/d_kz and Sx, Sy = d_kx,
// d_ky times it, each correctly rounded.  Any fixed shear keeps the test
// watertight for the ray; all traversals use this one, so their hit records
// are bit-identical.  (Woop et al. swap kx and ky when d_kz < 0 to keep the
// winding for back-face culling; without culling the swap only negates U, V,
// W, det and T together, which leaves t and the barycentrics exactly as
// they are, so the order stays cyclic and matches a stored record.)
__device__ __forceinline__ Shear make_shear(float ox, float oy, float oz, float dx, float dy, float dz) {
    Shear s;
    float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dkz = kz == 0 ? dx : (kz == 1 ? dy : dz);
    float dkx = kx == 0 ? dx : (kx == 1 ? dy : dz);
    float dky = ky == 0 ? dx : (ky == 1 ? dy : dz);
    s.Sz = __frcp_rn(dkz);  // 1/d_kz, correctly rounded
    s.Sx = __fmul_rn(dkx, s.Sz);
    s.Sy = __fmul_rn(dky, s.Sz);
    s.order = (uint32_t)kx;  // (kx, ky, kz) = (0, 1, 2), (1, 2, 0) or (2, 0, 1)
    s.ox = kx == 0 ? ox : (kx == 1 ? oy : oz);
    s.oy = ky == 0 ? ox : (ky == 1 ? oy : oz);
    s.oz = kz == 0 ? ox : (kz == 1 ? oy : oz);
    return s;
}

// The vertices of triangle `leaf` in the ray's axis order (tris: the BLAS
// records offset by 3 * Shear::order at the instance entry).
__device__ __forceinline__ const float4* tri_rec(const float4* tris, uint32_t leaf) {
    return tris + kTriStride * (size_t)leaf;
}

struct TriResult {
    bool hit;
    float t, V, W, det;
};

// Woop-Benthin-Wald watertight test on vertices given in the ray's axis order
// (x = kx, y = ky, z = kz); returns the hit if t in [tmin, tmax_incl].
__device__ __forceinline__ TriResult tri_test(const Shear& s, float4 v0, float4 v1, float4 v2, float tmin,
                                              float tmax_incl) {
    TriResult r;
    r.hit = false;
    float az = __fsub_rn(v0.z, s.oz), bz = __fsub_rn(v1.z, s.oz), cz = __fsub_rn(v2.z, s.oz);
    float Ax = __fsub_rn(__fsub_rn(v0.x, s.ox), __fmul_rn(s.Sx, az));
    float Ay = __fsub_rn(__fsub_rn(v0.y, s.oy), __fmul_rn(s.Sy, az));
    float Bx = __fsub_rn(__fsub_rn(v1.x, s.ox), __fmul_rn(s.Sx, bz));
    float By = __fsub_rn(__fsub_rn(v1.y, s.oy), __fmul_rn(s.Sy, bz));
    float Cx = __fsub_rn(__fsub_rn(v2.x, s.ox), __fmul_rn(s.Sx, cz));
    float Cy = __fsub_rn(__fsub_rn(v2.y, s.oy), __fmul_rn(s.Sy, cz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return r;
    float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.0f) return r;
    float T = __fadd_rn(__fadd_rn(__fmul_rn(U, __fmul_rn(s.Sz, az)), __fmul_rn(V, __fmul_rn(s.Sz, bz))),
                        __fmul_rn(W, __fmul_rn(s.Sz, cz)));
    float t = __fdiv_rn(T, det);
    if (!(t >= tmin && t <= tmax_incl)) return r;
    r.hit = true;
    r.t = t;
    r.V = V;
    r.W = W;
    r.det = det;
    return r;
}

// Write one ray's result: an ABI hit record, a render hit, or (shadow rays)
// the unshadowed contribution added to the image.
template <int MODE>
__device__ __forceinline__ void emit(const TraceArgs& a, uint32_t i, uint32_t j, bool found, bool ok, float best_t, uint32_t best_id,
                                     uint32_t best_prim, uint32_t best_il, uint32_t best_tl, float best_V,
                                     float best_W, float best_det) {
    if (MODE == kModeClosestAbi || MODE == kModeAnyAbi) {
        rg_hit out;
        if (found) {
            out.instance = best_id;
            out.prim = best_prim;
            out.t = best_t;
            out.u = __fdiv_rn(best_V, best_det);
            out.v = __fdiv_rn(best_W, best_det);
        } else {
            out.instance = kMiss;
            out.prim = kMiss;
            out.t = __int_as_float(0x7F800000);
            out.u = 0.f;
            out.v = 0.f;
        }
        a.hits_abi[i] = out;
    } else if (MODE == kModeClosestRender || MODE == kModeClosestBatch) {
        HitDev hd;
        hd.inst_leaf = found ? best_il : kMiss;
        hd.tri_leaf = found ? best_tl : kMiss;
        hd.t = found ? best_t : __int_as_float(0x7F800000);
        hd.pad = 0;
        *reinterpret_cast<uint4*>(a.hits_render + i) = *reinterpret_cast<const uint4*>(&hd);
    } else {  // shadow: accumulate the unshadowed contribution
        if (!found && ok) {
            const Payload p = a.payload[j];
            float* px = (MODE == kModeShadowBatch ? a.slots[slot_of_px(p.pixel)].image : a.image) +
                        4 * (size_t)px_of(p.pixel);
            atomicAdd(px + 0, p.r);
            atomicAdd(px + 1, p.g);
            atomicAdd(px + 2, p.b);
        }
    }
}

// Shadow rays in per-light sub-queues: the block's prefix of the sub-queue
// counts goes to shared memory (pre[l] = rays before sub-queue l, pre[n_sub]
// = all); returns the number of rays.  Without sub-queues: *d_count or n.
// TOTAL: the first block adds the rays to the scene's shadow-ray statistic
// (once per launch, instead of an atomic per warp and light in shading, which
// serialised on the one counter).
template <bool TOTAL>
__device__ __forceinline__ uint32_t ray_count(const TraceArgs& a, uint32_t* pre) {
    if (!a.sub_counts) return a.d_count ? *a.d_count : a.n;
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (uint32_t l = 0; l < a.n_sub; ++l) {
            pre[l] = acc;
            acc += a.sub_counts[l];
        }
        pre[a.n_sub] = acc;
        if (TOTAL && blockIdx.x == 0) atomicAdd(&a.st->shadow_rays, (unsigned long long)acc);
    }
    __syncthreads();
    return pre[a.n_sub];
}

// Queue entry of ray i: its place in its light's sub-queue.
__device__ __forceinline__ uint32_t sub_entry(const TraceArgs& a, const uint32_t* pre, uint32_t i) {
    if (!a.sub_counts) return i;
    uint32_t l = 0;
    while (l + 1 < a.n_sub && pre[l + 1] <= i) ++l;
    return l * a.sub_stride + (i - pre[l]);
}

template <bool ANY, bool STATS>
__device__ __forceinline__ void flush_counts(const TraceArgs& a, unsigned long long c_nodes, unsigned long long c_tris,
                                             unsigned long long c_inst) {
    if constexpr (STATS) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            c_nodes += __shfl_xor_sync(0xFFFFFFFFu, c_nodes, off);
            c_tris += __shfl_xor_sync(0xFFFFFFFFu, c_tris, off);
            c_inst += __shfl_xor_sync(0xFFFFFFFFu, c_inst, off);
        }
        if ((threadIdx.x & 31) == 0) {
            unsigned long long* c = a.st->count[ANY ? 1 : 0];
            atomicAdd(c + 0, c_nodes);
            atomicAdd(c + 1, c_tris);
            atomicAdd(c + 2, c_inst);
        }
    }
}

// Counting-traversal tallies of one thread.
struct TraceCounts {
    unsigned long long nodes = 0, tris = 0, inst = 0;
};

// One ray, run to completion: one loop iteration per node visit, instance
// entry or triangle test; a stack pop joins the step that follows it.  i is
// the ray's dense index (queue entry via the sub-queues or the ring).
template <int MODE, bool BRUTE, bool STATS>
__device__ __forceinline__ void trace_ray(const TraceArgs& a, const uint32_t* pre, uint32_t head, uint32_t i,
                                          TraceCounts& cnt) {
    const uint32_t iter_cap = a.iter_cap;
    constexpr bool kAny = (MODE == kModeAnyAbi || MODE == kModeShadowRender || MODE == kModeShadowBatch);
    constexpr bool kBatch = (MODE == kModeClosestBatch || MODE == kModeShadowBatch);
    const uint32_t j = MODE == kModeClosestBatch ? ((head + i) & a.ring_mask) : sub_entry(a, pre, i);

    // the TLAS of this ray (per request slot in the batched modes)
    const float4* tlas_nodes = a.tlas_nodes;
    const InstDev* tlas_inst = a.inst;
    uint32_t tlas_root = a.tlas_root;
    if (kBatch) {
        const SlotDev* S = a.slots + slot_of_px(a.payload[j].pixel);
        tlas_nodes = S->tlas_nodes;
        tlas_inst = S->inst;
        tlas_root = S->tlas_root;
    }

    const float4 r0 = __ldg(a.rays + 2 * (size_t)j), r1 = __ldg(a.rays + 2 * (size_t)j + 1);
    const float tmin = r0.w, tmax = r1.w;
    SpaceRay wr;
    wr.ox = r0.x; wr.oy = r0.y; wr.oz = r0.z;
    wr.ix = safe_rcp(r1.x); wr.iy = safe_rcp(r1.y); wr.iz = safe_rcp(r1.z);
    SpaceRay cr = wr;  // ray of the current space
    Shear sh;

    float best_t = tmax;
    uint32_t best_id = kMiss, best_prim = kMiss;
    uint32_t best_il = kMiss, best_tl = kMiss;
    float best_V = 0.f, best_W = 0.f, best_det = 1.f;
    bool found = false;

    uint32_t stack[kStack];
    int sp = 0;
    uint32_t ref = tlas_root;
    bool in_blas = false;
    const float4* nodes = tlas_nodes;
    const float4* tris = nullptr;
    uint32_t cur_id = 0, cur_leaf = 0;
    bool ok = true;

    for (uint32_t iter = 0;; ++iter) {
        if (iter >= iter_cap) {
            record_error(a.st, RG_ERR_TIMEOUT);
            ok = false;
            break;
        }
        if (ref == kNone) {
            // pop, and go on with the popped entry in this iteration
            if (sp == 0) break;
            ref = stack[--sp];
            if (ref == kMarker) {
                in_blas = false;
                nodes = tlas_nodes;
                cr = wr;
                if (sp == 0) break;
                ref = stack[--sp];  // a TLAS entry: markers never follow each other
            }
        }
        if (!(ref & kLeaf)) {
            const float4* nd = nodes + 4 * (size_t)ref;
            const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
            const uint4 n3 = __ldg(reinterpret_cast<const uint4*>(nd + 3));
            if (STATS) ++cnt.nodes;
            const float tlim = kAny ? __fmul_rn(tmax, kCullSlack) : __fmul_rn(best_t, kCullSlack);
            float tn0, tn1, tf0, tf1;
            bool h0 = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, cr, tmin, tlim, tn0, tf0);
            bool h1 = slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, cr, tmin, tlim, tn1, tf1);
            if (BRUTE) h0 = h1 = true;
            if (h0 && h1) {
                const bool f0 = visit_first0<kAny>(tn0, tf0, tn1, tf1);
                uint32_t nearc = f0 ? n3.x : n3.y;
                uint32_t farc = f0 ? n3.y : n3.x;
                if (sp >= kStack) {
                    record_error(a.st, RG_ERR_STACK);
                    ok = false;
                    break;
                }
                stack[sp++] = farc;
                ref = nearc;
            } else if (h0) {
                ref = n3.x;
            } else if (h1) {
                ref = n3.y;
            } else {
                ref = kNone;
            }
            continue;
        }
        const uint32_t leaf = ref & ~kLeaf;
        if (!in_blas) {
            const InstDev* I = tlas_inst + leaf;
            const float4 m0 = __ldg(&I->inv[0]), m1 = __ldg(&I->inv[1]), m2 = __ldg(&I->inv[2]);
            const float4 meta0 = __ldg(reinterpret_cast<const float4*>(&I->nodes));        // nodes, tris
            const uint4 meta1 = __ldg(reinterpret_cast<const uint4*>(&I->root));           // root, id, mat, blas
            if (STATS) ++cnt.inst;
            const float dx = r1.x, dy = r1.y, dz = r1.z;
            float ox = fmaf(m0.x, wr.ox, fmaf(m0.y, wr.oy, fmaf(m0.z, wr.oz, m0.w)));
            float oy = fmaf(m1.x, wr.ox, fmaf(m1.y, wr.oy, fmaf(m1.z, wr.oz, m1.w)));
            float oz = fmaf(m2.x, wr.ox, fmaf(m2.y, wr.oy, fmaf(m2.z, wr.oz, m2.w)));
            float ddx = fmaf(m0.x, dx, fmaf(m0.y, dy, __fmul_rn(m0.z, dz)));
            float ddy = fmaf(m1.x, dx, fmaf(m1.y, dy, __fmul_rn(m1.z, dz)));
            float ddz = fmaf(m2.x, dx, fmaf(m2.y, dy, __fmul_rn(m2.z, dz)));
            cr.ox = ox; cr.oy = oy; cr.oz = oz;
            cr.ix = safe_rcp(ddx); cr.iy = safe_rcp(ddy); cr.iz = safe_rcp(ddz);
            sh = make_shear(ox, oy, oz, ddx, ddy, ddz);
            const unsigned long long pn = ((unsigned long long)__float_as_uint(meta0.y) << 32) | __float_as_uint(meta0.x);
            const unsigned long long pt = ((unsigned long long)__float_as_uint(meta0.w) << 32) | __float_as_uint(meta0.z);
            nodes = reinterpret_cast<const float4*>(pn);
            tris = reinterpret_cast<const float4*>(pt) + 3 * sh.order;  // the ray's axis order
            cur_id = meta1.y;
            cur_leaf = leaf;
            in_blas = true;
            if (sp >= kStack) {
                record_error(a.st, RG_ERR_STACK);
                ok = false;
                break;
            }
            stack[sp++] = kMarker;
            ref = meta1.x;
            continue;
        }
        // triangle leaf
        {
            const float4* tp = tri_rec(tris, leaf);
            const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
            if (STATS) ++cnt.tris;
            TriResult h = tri_test(sh, v0, v1, v2, tmin, kAny ? tmax : best_t);
            ref = kNone;
            if (h.hit) {
                const uint32_t prim = __float_as_uint(v0.w);
                if (kAny) {
                    best_t = h.t; best_id = cur_id; best_prim = prim;
                    best_V = h.V; best_W = h.W; best_det = h.det;
                    found = true;
                    break;
                }
                bool better = h.t < best_t || cur_id < best_id || (cur_id == best_id && prim < best_prim);
                if (better) {
                    best_t = h.t; best_id = cur_id; best_prim = prim;
                    best_il = cur_leaf; best_tl = leaf;
                    best_V = h.V; best_W = h.W; best_det = h.det;
                    found = true;
                }
            }
        }
    }
    if (!ok) found = false;
    emit<MODE>(a, i, j, found, ok, best_t, best_id, best_prim, best_il, best_tl, best_V, best_W, best_det);
}

// Binary traversal, whole-warp refill: a warp takes 32 rays from the work
// counter, each lane runs its ray to completion, and the warp takes the next
// 32 when all its lanes are done.  Best when the rays of a warp take similar
// work (camera and secondary rays).
template <int MODE, bool BRUTE, bool STATS, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_trace_warp(TraceArgs a) {
    constexpr bool kAny = (MODE == kModeAnyAbi || MODE == kModeShadowRender || MODE == kModeShadowBatch);
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t n = ray_count<MODE == kModeShadowRender>(a, pre);
    const int lane = threadIdx.x & 31;
    // batched closest-hit rays sit in a ring of 2^k entries from *ring_head
    const uint32_t head = MODE == kModeClosestBatch ? *a.ring_head : 0u;
    TraceCounts cnt;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(a.work_counter, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        const uint32_t i = base + lane;
        if (i < n) trace_ray<MODE, BRUTE, STATS>(a, pre, head, i, cnt);
    }
    flush_counts<kAny, STATS>(a, cnt.nodes, cnt.tris, cnt.inst);
}

// The shadow rays of one depth level and the closest-hit rays of the next in
// one persistent launch (both depend only on the shading of the level; in the
// render server, the shadow rays of the previous step and the closest-hit
// rays of this one): one work counter runs over the shadow rays (in whole
// warps of 32) and then over the closest-hit rays, so warps that run out of
// one kind take the other and the SMs stay busy until the last batch of both,
// instead of idling through the tail of two separate launches.
// Launched for 896 resident threads per SM (72 registers, 7 blocks of 128):
// with both ray kinds inlined the kernel would take more and fit 768, and
// held to 64 registers (1024 threads) it spills inside the traversal loop;
// on the medium frame 896 measured fastest (2587 Mrays/s against 2550 at
// 768 and 2381 at 1024).
template <int SMODE, int CMODE, bool STATS, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 896 / BLOCK) k_trace_pair(TraceArgs sa, TraceArgs ca) {
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t ns = ray_count<SMODE == kModeShadowRender>(sa, pre);
    const uint32_t nc = ca.d_count ? *ca.d_count : ca.n;
    const uint32_t ns_pad = (ns + 31u) & ~31u;
    // batched closest-hit rays sit in a ring of 2^k entries from *ring_head
    const uint32_t head = CMODE == kModeClosestBatch ? *ca.ring_head : 0u;
    const int lane = threadIdx.x & 31;
    TraceCounts cs, cc;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(sa.work_counter, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base < ns_pad) {
            const uint32_t i = base + lane;
            if (i < ns) trace_ray<SMODE, false, STATS>(sa, pre, 0u, i, cs);
        } else {
            const uint32_t b = base - ns_pad;
            if (b >= nc) break;
            const uint32_t i = b + lane;
            if (i < nc) trace_ray<CMODE, false, STATS>(ca, nullptr, head, i, cc);
        }
    }
    flush_counts<true, STATS>(sa, cs.nodes, cs.tris, cs.inst);
    flush_counts<false, STATS>(ca, cc.nodes, cc.tris, cc.inst);
}

// Binary traversal, per-lane refill.  Each lane holds one ray and advances it
// by one step per loop iteration (a node visit, an instance entry or a
// triangle test, then the stack pops that step leaves for the next one).  A
// warp refills its idle lanes from the work counter as soon as at least
// `refill` of them are idle, so lanes do not wait for the slowest ray of the
// warp; that pays when ray lengths vary widely (incoherent queries) and costs
// a warp vote per step otherwise.
template <int MODE, bool BRUTE, bool STATS, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_trace_lane(TraceArgs a) {
    const uint32_t iter_cap = a.iter_cap;
    constexpr bool kAny = (MODE == kModeAnyAbi || MODE == kModeShadowRender || MODE == kModeShadowBatch);
    constexpr bool kBatch = (MODE == kModeClosestBatch || MODE == kModeShadowBatch);
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t n = ray_count<MODE == kModeShadowRender>(a, pre);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t refill = a.refill;
    // batched closest-hit rays sit in a ring of 2^k entries from *ring_head
    const uint32_t head = MODE == kModeClosestBatch ? *a.ring_head : 0u;
    unsigned long long c_nodes = 0, c_tris = 0, c_inst = 0;

    bool active = false, exhausted = false;
    uint32_t i = 0, j = 0;  // ray index (dense) and queue entry
    const float4* tlas_nodes = a.tlas_nodes;
    const InstDev* tlas_inst = a.inst;
    float tmin = 0.f, tmax = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
    SpaceRay wr, cr;
    Shear sh;
    float best_t = 0.f, best_V = 0.f, best_W = 0.f, best_det = 1.f;
    uint32_t best_id = kMiss, best_prim = kMiss, best_il = kMiss, best_tl = kMiss;
    bool found = false, ok = true, in_blas = false;
    uint32_t stack[kStack];
    int sp = 0;
    uint32_t ref = kNone, iter = 0, cur_id = 0, cur_leaf = 0;
    const float4* nodes = nullptr;
    const float4* tris = nullptr;

    for (;;) {
        // refill the idle lanes (all lanes take part: the ballot is warp-wide)
        const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !active);
        if (!exhausted && idle != 0u && (__popc(idle) >= (int)refill || idle == 0xFFFFFFFFu)) {
            const uint32_t k = (uint32_t)__popc(idle);
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(a.work_counter, k);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base + k >= n) exhausted = true;
            if (!active) {
                const uint32_t idx = base + (uint32_t)__popc(idle & ((1u << lane) - 1u));
                if (idx < n) {
                    i = idx;
                    j = MODE == kModeClosestBatch ? ((head + i) & a.ring_mask) : sub_entry(a, pre, i);
                    uint32_t tlas_root = a.tlas_root;
                    if (kBatch) {  // the TLAS of this ray's request slot
                        const SlotDev* S = a.slots + slot_of_px(a.payload[j].pixel);
                        tlas_nodes = S->tlas_nodes;
                        tlas_inst = S->inst;
                        tlas_root = S->tlas_root;
                    }
                    const float4 r0 = __ldg(a.rays + 2 * (size_t)j), r1 = __ldg(a.rays + 2 * (size_t)j + 1);
                    tmin = r0.w;
                    tmax = r1.w;
                    dx = r1.x;
                    dy = r1.y;
                    dz = r1.z;
                    wr.ox = r0.x; wr.oy = r0.y; wr.oz = r0.z;
                    wr.ix = safe_rcp(dx); wr.iy = safe_rcp(dy); wr.iz = safe_rcp(dz);
                    cr = wr;
                    best_t = tmax;
                    best_id = best_prim = best_il = best_tl = kMiss;
                    best_V = best_W = 0.f;
                    best_det = 1.f;
                    found = false;
                    ok = true;
                    in_blas = false;
                    sp = 0;
                    ref = tlas_root;
                    nodes = tlas_nodes;
                    iter = 0;
                    active = true;
                }
            }
        }
        // every ray claimed above went to a lane, so a warp without one is done
        if (__ballot_sync(0xFFFFFFFFu, active) == 0u) break;
        if (!active) continue;

        bool finished = false;
        if (++iter > iter_cap) {
            record_error(a.st, RG_ERR_TIMEOUT);
            ok = false;
            finished = true;
        } else if (!(ref & kLeaf)) {
            const float4* nd = nodes + 4 * (size_t)ref;
            const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
            const uint4 n3 = __ldg(reinterpret_cast<const uint4*>(nd + 3));
            if (STATS) ++c_nodes;
            const float tlim = kAny ? __fmul_rn(tmax, kCullSlack) : __fmul_rn(best_t, kCullSlack);
            float tn0, tn1, tf0, tf1;
            bool h0 = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, cr, tmin, tlim, tn0, tf0);
            bool h1 = slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, cr, tmin, tlim, tn1, tf1);
            if (BRUTE) h0 = h1 = true;
            if (h0 && h1) {
                if (sp >= kStack) {
                    record_error(a.st, RG_ERR_STACK);
                    ok = false;
                    finished = true;
                } else {
                    const bool first0 = visit_first0<kAny>(tn0, tf0, tn1, tf1);
                    stack[sp++] = first0 ? n3.y : n3.x;
                    ref = first0 ? n3.x : n3.y;
                }
            } else {
                ref = h0 ? n3.x : (h1 ? n3.y : kNone);
            }
        } else if (!in_blas) {
            // instance: enter its BLAS with the object-space ray
            const uint32_t leaf = ref & ~kLeaf;
            const InstDev* I = tlas_inst + leaf;
            const float4 m0 = __ldg(&I->inv[0]), m1 = __ldg(&I->inv[1]), m2 = __ldg(&I->inv[2]);
            const float4 meta0 = __ldg(reinterpret_cast<const float4*>(&I->nodes));  // nodes, tris
            const uint4 meta1 = __ldg(reinterpret_cast<const uint4*>(&I->root));     // root, id, mat, blas
            if (STATS) ++c_inst;
            const float ox = fmaf(m0.x, wr.ox, fmaf(m0.y, wr.oy, fmaf(m0.z, wr.oz, m0.w)));
            const float oy = fmaf(m1.x, wr.ox, fmaf(m1.y, wr.oy, fmaf(m1.z, wr.oz, m1.w)));
            const float oz = fmaf(m2.x, wr.ox, fmaf(m2.y, wr.oy, fmaf(m2.z, wr.oz, m2.w)));
            const float ddx = fmaf(m0.x, dx, fmaf(m0.y, dy, __fmul_rn(m0.z, dz)));
            const float ddy = fmaf(m1.x, dx, fmaf(m1.y, dy, __fmul_rn(m1.z, dz)));
            const float ddz = fmaf(m2.x, dx, fmaf(m2.y, dy, __fmul_rn(m2.z, dz)));
            if (sp >= kStack) {
                record_error(a.st, RG_ERR_STACK);
                ok = false;
                finished = true;
            } else {
                cr.ox = ox; cr.oy = oy; cr.oz = oz;
                cr.ix = safe_rcp(ddx); cr.iy = safe_rcp(ddy); cr.iz = safe_rcp(ddz);
                sh = make_shear(ox, oy, oz, ddx, ddy, ddz);
                nodes = reinterpret_cast<const float4*>(
                    ((unsigned long long)__float_as_uint(meta0.y) << 32) | __float_as_uint(meta0.x));
                tris = reinterpret_cast<const float4*>(
                           ((unsigned long long)__float_as_uint(meta0.w) << 32) | __float_as_uint(meta0.z)) +
                       3 * sh.order;  // the ray's axis order
                cur_id = meta1.y;
                cur_leaf = leaf;
                in_blas = true;
                stack[sp++] = kMarker;
                ref = meta1.x;
            }
        } else {
            // triangle
            const uint32_t leaf = ref & ~kLeaf;
            const float4* tp = tri_rec(tris, leaf);
            const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
            if (STATS) ++c_tris;
            const TriResult h = tri_test(sh, v0, v1, v2, tmin, kAny ? tmax : best_t);
            ref = kNone;
            if (h.hit) {
                const uint32_t prim = __float_as_uint(v0.w);
                if (kAny || h.t < best_t || cur_id < best_id || (cur_id == best_id && prim < best_prim)) {
                    best_t = h.t; best_id = cur_id; best_prim = prim;
                    best_il = cur_leaf; best_tl = leaf;
                    best_V = h.V; best_W = h.W; best_det = h.det;
                    found = true;
                }
                if (kAny) finished = true;
            }
        }
        // pop what the step left (the BLAS marker brings back the world-space ray)
        if (!finished && ref == kNone) {
            if (sp > 0) {
                ref = stack[--sp];
                if (ref == kMarker) {
                    in_blas = false;
                    nodes = tlas_nodes;
                    cr = wr;
                    ref = sp > 0 ? stack[--sp] : kNone;
                }
            }
            finished = ref == kNone;
        }
        if (finished) {
            emit<MODE>(a, i, j, found && ok, ok, best_t, best_id, best_prim, best_il, best_tl, best_V, best_W, best_det);
            active = false;
        }
    }
    flush_counts<kAny, STATS>(a, c_nodes, c_tris, c_inst);
}

// ---------------------------------------------------------------- wide BVH
// Traversal of the compressed 8-wide BVH (layout in rg_internal.cuh).  The
// state is a node group (children of one node still to visit: base index,
// hit bits in visiting order, the node's internal-slot mask) and an item
// group (triangles or instances of the leaf slots hit at the last node: base
// index, one bit per item).  Items are handled before the next node is
// fetched; unfinished groups and the BLAS marker go on a short stack of
// 8-byte entries.  Child boxes are tested with one FMA per plane,
// t = q * (2^e / d) + (p - o) / d, which differs from the exact slab
// distance by at most kQuantErr * (255 |2^e / d| + |(p - o) / d|) (a few
// roundings of those magnitudes); widening every child interval of the node
// by that bound E keeps the test conservative, so the wide path finds the same
// hits as the binary one.
constexpr int kStack8 = 48;
constexpr uint32_t kKindNode = 0u, kKindItem = 1u << 30, kKindMarker = 2u << 30;
constexpr float kQuantErr = 8.0f * 5.9604644775390625e-08f;

__device__ __forceinline__ uint32_t oct_of(const SpaceRay& r) {
    return (__float_as_uint(r.ix) >> 31) | ((__float_as_uint(r.iy) >> 31) << 1) | ((__float_as_uint(r.iz) >> 31) << 2);
}

// Byte k of w as a float: one byte permute builds the bit pattern of 2^23 + q
// (exponent byte 0x4B above the byte), then an exact subtraction of 2^23.
__device__ __forceinline__ float byte_f(uint32_t w, int k) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, (uint32_t)k | 0x7440u)) - 8388608.0f;
}

template <int MODE, bool STATS>
__global__ void __launch_bounds__(kTraceBlock) k_trace8(TraceArgs a) {
    const uint32_t iter_cap = a.iter_cap;
    constexpr bool kAny = (MODE == kModeAnyAbi || MODE == kModeShadowRender);
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t n = ray_count<MODE == kModeShadowRender>(a, pre);
    const int lane = threadIdx.x & 31;
    unsigned long long c_nodes = 0, c_tris = 0, c_inst = 0;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(a.work_counter, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        const uint32_t i = base + lane;
        if (i >= n) continue;
        const uint32_t j = sub_entry(a, pre, i);

        const float4 r0 = __ldg(a.rays + 2 * (size_t)j), r1 = __ldg(a.rays + 2 * (size_t)j + 1);
        const float tmin = r0.w, tmax = r1.w;
        SpaceRay wr;
        wr.ox = r0.x; wr.oy = r0.y; wr.oz = r0.z;
        wr.ix = safe_rcp(r1.x); wr.iy = safe_rcp(r1.y); wr.iz = safe_rcp(r1.z);
        const uint32_t oct_w = oct_of(wr);
        SpaceRay cr = wr;
        uint32_t oct = oct_w;
        Shear sh;

        float best_t = tmax;
        uint32_t best_id = kMiss, best_prim = kMiss, best_il = kMiss, best_tl = kMiss;
        float best_V = 0.f, best_W = 0.f, best_det = 1.f;
        bool found = false, ok = true, in_blas = false;

        uint2 stack[kStack8];
        int sp = 0;
        const float4* nodes = a.tlas_nodes8;
        const float4* tris = nullptr;
        uint32_t cur_id = 0, cur_leaf = 0;
        // node group: the root as the only internal child (slot 0) of a virtual node
        uint32_t g_base = 0, g_hits = 1u << oct, g_imask = 1u;
        uint32_t i_base = 0, i_bits = 0;

        // Phases keep the lanes of a warp on the same kind of work: all lanes
        // fetch nodes until each has items pending (or is done with nodes),
        // then all process items; only then does a lane pop its stack.
        bool done = false;
        uint32_t iter = 0;
        while (!done) {
            while (g_hits && !i_bits) {
                if (++iter > iter_cap) {
                    record_error(a.st, RG_ERR_TIMEOUT);
                    ok = false;
                    done = true;
                    break;
                }
                    const uint32_t b = 31 - __clz(g_hits);
                    g_hits &= ~(1u << b);
                    const uint32_t s = b ^ oct;
                    const uint32_t node = g_base + __popc(g_imask & ((1u << s) - 1u));
                    if (g_hits) {
                        if (sp >= kStack8) {
                            record_error(a.st, RG_ERR_STACK);
                            ok = false;
                            done = true;
                            break;
                        }
                        stack[sp++] = make_uint2(g_base, g_hits | (g_imask << 8) | kKindNode);
                    }
                    const float4* nd = nodes + 5 * (size_t)node;
                    const float4 w0 = __ldg(nd);
                    const uint4 w1 = __ldg(reinterpret_cast<const uint4*>(nd + 1));
                    const uint4 w2 = __ldg(reinterpret_cast<const uint4*>(nd + 2));
                    const uint4 w3 = __ldg(reinterpret_cast<const uint4*>(nd + 3));
                    const uint4 w4 = __ldg(reinterpret_cast<const uint4*>(nd + 4));
                    if (STATS) ++c_nodes;
                    const uint32_t bits = __float_as_uint(w0.w);
                    const uint32_t imask = bits >> 24;
                    const float sx = __int_as_float((((int)(int8_t)(bits & 0xFF)) + 127) << 23);
                    const float sy = __int_as_float((((int)(int8_t)((bits >> 8) & 0xFF)) + 127) << 23);
                    const float sz = __int_as_float((((int)(int8_t)((bits >> 16) & 0xFF)) + 127) << 23);
                    const float Sx = sx * cr.ix, Sy = sy * cr.iy, Sz = sz * cr.iz;  // exact: powers of two
                    const float Bx = __fmul_rn(__fsub_rn(w0.x, cr.ox), cr.ix);
                    const float By = __fmul_rn(__fsub_rn(w0.y, cr.oy), cr.iy);
                    const float Bz = __fmul_rn(__fsub_rn(w0.z, cr.oz), cr.iz);
                    const float E = kQuantErr * fmaxf(fmaxf(fmaf(255.0f, fabsf(Sx), fabsf(Bx)), fmaf(255.0f, fabsf(Sy), fabsf(By))),
                                                      fmaf(255.0f, fabsf(Sz), fabsf(Bz)));
                    // near planes shifted down by E, far planes up by E
                    const float Bxn = Bx - E, Byn = By - E, Bzn = Bz - E;
                    const float Bxf = Bx + E, Byf = By + E, Bzf = Bz + E;
                    // near/far planes per axis from the direction signs
                    const bool nx = oct & 1, ny = oct & 2, nz = oct & 4;
                    const uint32_t nx0 = nx ? w3.z : w2.x, nx1 = nx ? w3.w : w2.y, fx0 = nx ? w2.x : w3.z, fx1 = nx ? w2.y : w3.w;
                    const uint32_t ny0 = ny ? w4.x : w2.z, ny1 = ny ? w4.y : w2.w, fy0 = ny ? w2.z : w4.x, fy1 = ny ? w2.w : w4.y;
                    const uint32_t nz0 = nz ? w4.z : w3.x, nz1 = nz ? w4.w : w3.y, fz0 = nz ? w3.x : w4.z, fz1 = nz ? w3.y : w4.w;
                    const float tlim = kAny ? __fmul_rn(tmax, kCullSlack) : __fmul_rn(best_t, kCullSlack);
                    const uint32_t meta_lo = w1.z, meta_hi = w1.w;
                    uint32_t hitmask = 0;
    #pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int k = c & 3;
                        const float tnx = fmaf(byte_f(c < 4 ? nx0 : nx1, k), Sx, Bxn);
                        const float tfx = fmaf(byte_f(c < 4 ? fx0 : fx1, k), Sx, Bxf);
                        const float tny = fmaf(byte_f(c < 4 ? ny0 : ny1, k), Sy, Byn);
                        const float tfy = fmaf(byte_f(c < 4 ? fy0 : fy1, k), Sy, Byf);
                        const float tnz = fmaf(byte_f(c < 4 ? nz0 : nz1, k), Sz, Bzn);
                        const float tfz = fmaf(byte_f(c < 4 ? fz0 : fz1, k), Sz, Bzf);
                        const float tn = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, tmin));
                        const float tf = fminf(fminf(tfx, tfy), fminf(tfz, tlim));
                        if (tn <= tf) hitmask |= 1u << c;
                    }
                    // keep occupied slots only: internal ones and leaves (meta != 0)
                    const uint32_t occ_lo = __vcmpne4(meta_lo, 0u) & 0x08040201u;
                    const uint32_t occ_hi = __vcmpne4(meta_hi, 0u) & 0x80402010u;
                    uint32_t occ = occ_lo | occ_hi;
                    occ = (occ | (occ >> 8) | (occ >> 16) | (occ >> 24)) & 0xFFu;
                    hitmask &= occ | imask;
                    // internal hits, bit positions permuted to visiting order (slot ^ oct)
                    uint32_t hits = hitmask & imask;
                    if (oct & 1u) hits = ((hits & 0x55u) << 1) | ((hits >> 1) & 0x55u);
                    if (oct & 2u) hits = ((hits & 0x33u) << 2) | ((hits >> 2) & 0x33u);
                    if (oct & 4u) hits = ((hits & 0x0Fu) << 4) | ((hits >> 4) & 0x0Fu);
                    uint32_t items = 0;
                    for (uint32_t lm = hitmask & ~imask; lm; lm &= lm - 1) {
                        const int c = __ffs(lm) - 1;
                        const uint32_t meta = ((c < 4 ? meta_lo : meta_hi) >> (8 * (c & 3))) & 0xFFu;
                        items |= ((1u << (meta >> 5)) - 1u) << (meta & 31u);
                    }
                    g_base = w1.x;
                    g_hits = hits;
                    g_imask = imask;
                    i_base = w1.y;
                    i_bits = items;
            }
            if (done) break;
            while (i_bits) {
                if (++iter > iter_cap) {
                    record_error(a.st, RG_ERR_TIMEOUT);
                    ok = false;
                    done = true;
                    break;
                }
                    const uint32_t k = __ffs(i_bits) - 1;
                    i_bits &= i_bits - 1;
                    const uint32_t item = i_base + k;
                    if (!in_blas) {
                        // instance: save the TLAS groups, enter its BLAS
                        if (sp + 3 > kStack8) {
                            record_error(a.st, RG_ERR_STACK);
                            ok = false;
                            done = true;
                            break;
                        }
                        if (g_hits) stack[sp++] = make_uint2(g_base, g_hits | (g_imask << 8) | kKindNode);
                        if (i_bits) stack[sp++] = make_uint2(i_base, i_bits | kKindItem);
                        stack[sp++] = make_uint2(0u, kKindMarker);
                        const InstDev* I = a.inst8 + item;
                        const float4 m0 = __ldg(&I->inv[0]), m1 = __ldg(&I->inv[1]), m2 = __ldg(&I->inv[2]);
                        const float4 meta0 = __ldg(reinterpret_cast<const float4*>(&I->nodes));
                        const uint4 meta1 = __ldg(reinterpret_cast<const uint4*>(&I->root));
                        if (STATS) ++c_inst;
                        const float dx = r1.x, dy = r1.y, dz = r1.z;
                        float ox = fmaf(m0.x, wr.ox, fmaf(m0.y, wr.oy, fmaf(m0.z, wr.oz, m0.w)));
                        float oy = fmaf(m1.x, wr.ox, fmaf(m1.y, wr.oy, fmaf(m1.z, wr.oz, m1.w)));
                        float oz = fmaf(m2.x, wr.ox, fmaf(m2.y, wr.oy, fmaf(m2.z, wr.oz, m2.w)));
                        float ddx = fmaf(m0.x, dx, fmaf(m0.y, dy, __fmul_rn(m0.z, dz)));
                        float ddy = fmaf(m1.x, dx, fmaf(m1.y, dy, __fmul_rn(m1.z, dz)));
                        float ddz = fmaf(m2.x, dx, fmaf(m2.y, dy, __fmul_rn(m2.z, dz)));
                        cr.ox = ox; cr.oy = oy; cr.oz = oz;
                        cr.ix = safe_rcp(ddx); cr.iy = safe_rcp(ddy); cr.iz = safe_rcp(ddz);
                        oct = oct_of(cr);
                        sh = make_shear(ox, oy, oz, ddx, ddy, ddz);
                        const unsigned long long pn =
                            ((unsigned long long)__float_as_uint(meta0.y) << 32) | __float_as_uint(meta0.x);
                        const unsigned long long pt =
                            ((unsigned long long)__float_as_uint(meta0.w) << 32) | __float_as_uint(meta0.z);
                        nodes = reinterpret_cast<const float4*>(pn);
                        tris = reinterpret_cast<const float4*>(pt) + 3 * sh.order;  // the ray's axis order
                        cur_id = meta1.y;
                        cur_leaf = item;
                        in_blas = true;
                        g_base = 0;
                        g_hits = 1u << oct;
                        g_imask = 1u;
                        i_bits = 0;
                        continue;
                    }
                    const float4* tp = tri_rec(tris, item);
                    const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
                    if (STATS) ++c_tris;
                    TriResult h = tri_test(sh, v0, v1, v2, tmin, kAny ? tmax : best_t);
                    if (h.hit) {
                        const uint32_t prim = __float_as_uint(v0.w);
                        if (kAny) {
                            best_t = h.t; best_id = cur_id; best_prim = prim;
                            best_V = h.V; best_W = h.W; best_det = h.det;
                            found = true;
                            done = true;
                            break;
                        }
                        if (h.t < best_t || cur_id < best_id || (cur_id == best_id && prim < best_prim)) {
                            best_t = h.t; best_id = cur_id; best_prim = prim;
                            best_il = cur_leaf; best_tl = item;
                            best_V = h.V; best_W = h.W; best_det = h.det;
                            found = true;
                        }
                    }
            }
            if (done) break;
            if (g_hits) continue;
            if (sp == 0) break;
            const uint2 e = stack[--sp];
            const uint32_t kind = e.y & (3u << 30);
            if (kind == kKindMarker) {
                in_blas = false;
                nodes = a.tlas_nodes8;
                cr = wr;
                oct = oct_w;
            } else if (kind == kKindItem) {
                i_base = e.x;
                i_bits = e.y & 0xFFFFFFu;
            } else {
                g_base = e.x;
                g_hits = e.y & 0xFFu;
                g_imask = (e.y >> 8) & 0xFFu;
            }
        }
        if (!ok) found = false;
        emit<MODE>(a, i, j, found, ok, best_t, best_id, best_prim, best_il, best_tl, best_V, best_W, best_det);
    }
    flush_counts<kAny, STATS>(a, c_nodes, c_tris, c_inst);
}

template <int MODE, bool STATS>
cudaError_t launch_mode8(const TraceArgs& a, cudaStream_t s) {
    static int blocks = 0;
    if (blocks == 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace8<MODE, STATS>, kTraceBlock, 0);
        if (e != cudaSuccess) return e;
        blocks = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    }
    k_trace8<MODE, STATS><<<blocks, kTraceBlock, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int MODE, bool BRUTE, bool STATS, int BLOCK, bool LANE>
cudaError_t launch_block(const TraceArgs& a, int blocks_per_sm, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = LANE ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_lane<MODE, BRUTE, STATS, BLOCK>,
                                                                             BLOCK, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_warp<MODE, BRUTE, STATS, BLOCK>,
                                                                             BLOCK, 0);
        if (e != cudaSuccess) return e;
        if (per_sm <= 0) per_sm = 1;
    }
    const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
    if (LANE)
        k_trace_lane<MODE, BRUTE, STATS, BLOCK><<<device_sm_count() * b, BLOCK, 0, s>>>(a);
    else
        k_trace_warp<MODE, BRUTE, STATS, BLOCK><<<device_sm_count() * b, BLOCK, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int SMODE, int CMODE, bool STATS, int BLOCK>
cudaError_t launch_pair_t(const TraceArgs& sa, const TraceArgs& ca, int blocks_per_sm, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_pair<SMODE, CMODE, STATS, BLOCK>,
                                                                      BLOCK, 0);
        if (e != cudaSuccess) return e;
        if (per_sm <= 0) per_sm = 1;
    }
    const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
    k_trace_pair<SMODE, CMODE, STATS, BLOCK><<<device_sm_count() * b, BLOCK, 0, s>>>(sa, ca);
    count_launches(1);
    return cudaGetLastError();
}

// Refill threshold when the shape leaves it open (0): per-lane refill (8 idle
// lanes) for the closest-hit queries of rg_trace_rays, whose rays are often
// incoherent; whole-warp refill elsewhere (faster on camera, secondary and
// shadow rays and on incoherent any-hit queries, as measured on GB300).
template <int MODE>
constexpr int default_refill() {
    return MODE == kModeClosestAbi ? 8 : 32;
}

// Shapes other than 128 threads are compiled for the render and batched modes
// (the ones the autotuner sets); the rest run with 128.  refill < 32 selects
// the per-lane-refill kernel, 32 the whole-warp one.
template <int MODE, bool BRUTE, bool STATS>
cudaError_t launch_mode(const TraceArgs& a0, cudaStream_t s, const TraceShape& shape = TraceShape()) {
    TraceArgs a = a0;
    const int refill = (shape.refill >= 1 && shape.refill <= 32) ? shape.refill : default_refill<MODE>();
    a.refill = (uint32_t)refill;
    constexpr bool kTunable = !BRUTE && !STATS && MODE >= kModeClosestRender;
    if (refill < 32) {
        if constexpr (kTunable) {
            if (shape.block == 64) return launch_block<MODE, BRUTE, STATS, 64, true>(a, shape.blocks_per_sm, s);
            if (shape.block == 256) return launch_block<MODE, BRUTE, STATS, 256, true>(a, shape.blocks_per_sm, s);
        }
        return launch_block<MODE, BRUTE, STATS, 128, true>(a, shape.blocks_per_sm, s);
    }
    if constexpr (kTunable) {
        if (shape.block == 64) return launch_block<MODE, BRUTE, STATS, 64, false>(a, shape.blocks_per_sm, s);
        if (shape.block == 256) return launch_block<MODE, BRUTE, STATS, 256, false>(a, shape.blocks_per_sm, s);
    }
    return launch_block<MODE, BRUTE, STATS, 128, false>(a, shape.blocks_per_sm, s);
}

}  // namespace

cudaError_t launch_trace(int mode, bool brute, bool stats, const TraceArgs& a0, cudaStream_t s,
                         const TraceShape& shape) {
    TraceArgs a = a0;
    if (a.tlas_nodes8 && !brute) {
        switch (mode) {
            case kModeClosestAbi:
                return stats ? launch_mode8<kModeClosestAbi, true>(a, s) : launch_mode8<kModeClosestAbi, false>(a, s);
            case kModeAnyAbi:
                return stats ? launch_mode8<kModeAnyAbi, true>(a, s) : launch_mode8<kModeAnyAbi, false>(a, s);
            case kModeClosestRender:
                return stats ? launch_mode8<kModeClosestRender, true>(a, s)
                             : launch_mode8<kModeClosestRender, false>(a, s);
            case kModeShadowRender:
                return stats ? launch_mode8<kModeShadowRender, true>(a, s)
                             : launch_mode8<kModeShadowRender, false>(a, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (mode) {
        case kModeClosestAbi:
            if (brute) return launch_mode<kModeClosestAbi, true, false>(a, s);
            return stats ? launch_mode<kModeClosestAbi, false, true>(a, s) : launch_mode<kModeClosestAbi, false, false>(a, s);
        case kModeAnyAbi:
            if (brute) return launch_mode<kModeAnyAbi, true, false>(a, s);
            return stats ? launch_mode<kModeAnyAbi, false, true>(a, s) : launch_mode<kModeAnyAbi, false, false>(a, s);
        case kModeClosestRender:
            return stats ? launch_mode<kModeClosestRender, false, true>(a, s)
                         : launch_mode<kModeClosestRender, false, false>(a, s, shape);
        case kModeShadowRender:
            return stats ? launch_mode<kModeShadowRender, false, true>(a, s)
                         : launch_mode<kModeShadowRender, false, false>(a, s, shape);
        case kModeClosestBatch:
            return launch_mode<kModeClosestBatch, false, false>(a, s, shape);
        case kModeShadowBatch:
            return launch_mode<kModeShadowBatch, false, false>(a, s, shape);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_trace_pair(bool batch, bool stats, const TraceArgs& sa, const TraceArgs& ca, cudaStream_t s,
                              const TraceShape& shape) {
    if (sa.tlas_nodes8 || ca.tlas_nodes8) return cudaErrorInvalidValue;  // binary BVH only
    if (batch) {
        if (stats) return cudaErrorInvalidValue;
        if (shape.block == 64)
            return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 64>(sa, ca, shape.blocks_per_sm, s);
        if (shape.block == 256)
            return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 256>(sa, ca, shape.blocks_per_sm, s);
        return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 128>(sa, ca, shape.blocks_per_sm, s);
    }
    return stats ? launch_pair_t<kModeShadowRender, kModeClosestRender, true, kTraceBlock>(sa, ca, 0, s)
                 : launch_pair_t<kModeShadowRender, kModeClosestRender, false, kTraceBlock>(sa, ca, 0, s);
}

}  // namespace rg
