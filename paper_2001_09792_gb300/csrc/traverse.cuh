// Per-ray traversal of the two-level BVH: closest-hit, any-hit and miss (paper
// Sec. 1: per ray, the closest-hit or any-hit shader runs when the ray meets a
// triangle, the miss shader when it meets none).
//
// Each thread runs a stack traversal: TLAS nodes in world space; at an
// instance leaf the ray is moved to object space with the instance's float32
// inverse (t is shared, the direction is not renormalised), a marker is
// pushed, and the BLAS is traversed; popping the marker restores the world
// ray.  Nodes are 64 B (two child boxes), read with four 16 B loads; a
// triangle is read as three 16 B vertices from its record, in the ray's axis
// order.
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
//
// This code is shared by the traversal kernels (trace.cu) and the renderer
// (render.cu); every operation whose rounding matters is an explicit
// intrinsic, so both files compute the same hits whatever their contraction
// flags.
#pragma once

#include "rg_internal.cuh"

namespace rg {

namespace {

constexpr int kStack = (int)kTraceStack;
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

// The renderer's closest-hit launches add their ray count to the scene's
// statistic (first thread of the first block), so a render needs no count on
// the host.
template <int MODE>
__device__ __forceinline__ void count_closest(const TraceArgs& a, uint32_t n) {
    if (MODE == kModeClosestRender && blockIdx.x == 0 && threadIdx.x == 0 && n)
        atomicAdd(&a.st->closest_rays, (unsigned long long)n);
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

// What one traversal found (found: a hit within the ray's interval; ok:
// no stack overflow or iteration cap; il / tl: the hit's instance leaf and
// triangle leaf, closest hit only).
struct RayHit {
    bool found, ok;
    float t, V, W, det;
    uint32_t id, prim, il, tl;
};

// One ray, run to completion: one loop iteration per node visit, instance
// entry or triangle test; a stack pop joins the step that follows it.  The ray
// is r0 = (origin, tmin), r1 = (direction, tmax) in world space; ANY: the
// first hit ends it.
template <bool ANY, bool BRUTE, bool STATS>
__device__ __forceinline__ RayHit trace_core(const TraceArgs& a, const float4* tlas_nodes, const InstDev* tlas_inst,
                                             uint32_t tlas_root, float4 r0, float4 r1, TraceCounts& cnt) {
    const uint32_t iter_cap = a.iter_cap;
    constexpr bool kAny = ANY;
    const float tmin = r0.w, tmax = r1.w;
    SpaceRay wr;
    wr.ox = r0.x; wr.oy = r0.y; wr.oz = r0.z;
    wr.ix = safe_rcp(r1.x); wr.iy = safe_rcp(r1.y); wr.iz = safe_rcp(r1.z);
    SpaceRay cr = wr;  // ray of the current space
    Shear sh;

    float best_t = tmax;
    // culling distance of the box tests: the ray's end (any hit) or the best
    // hit so far (closest hit), with the relative slack
    float tlim = __fmul_rn(tmax, kCullSlack);
    uint32_t best_id = kMiss, best_prim = kMiss;
    uint32_t best_il = kMiss, best_tl = kMiss;
    float best_V = 0.f, best_W = 0.f, best_det = 1.f;
    bool found = false;

    uint32_t stack[kStack];
    int sp = 0;
    // the test limit on the stack applies to the counting instantiations only,
    // so the timed kernels compare with the constant
    const int smax = (STATS && a.stack_max >= 1 && a.stack_max < (uint32_t)kStack) ? (int)a.stack_max : kStack;
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
            float tn0, tn1, tf0, tf1;
            bool h0 = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, cr, tmin, tlim, tn0, tf0);
            bool h1 = slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, cr, tmin, tlim, tn1, tf1);
            if (BRUTE) h0 = h1 = true;
            if (h0 && h1) {
                const bool f0 = visit_first0<kAny>(tn0, tf0, tn1, tf1);
                uint32_t nearc = f0 ? n3.x : n3.y;
                uint32_t farc = f0 ? n3.y : n3.x;
                if (sp >= smax) {
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
            if (sp >= smax) {
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
                    tlim = __fmul_rn(best_t, kCullSlack);
                    best_V = h.V; best_W = h.W; best_det = h.det;
                    found = true;
                }
            }
        }
    }
    RayHit h;
    h.found = found && ok;
    h.ok = ok;
    h.t = best_t;
    h.V = best_V;
    h.W = best_W;
    h.det = best_det;
    h.id = best_id;
    h.prim = best_prim;
    h.il = best_il;
    h.tl = best_tl;
    return h;
}

// Segments per shadow ray in a launch of n rays: a.split when the queue is
// small enough to leave lanes idle (its longest rays then set the launch
// time, and segments of one ray run side by side), else 1.
template <int MODE>
__device__ __forceinline__ uint32_t shadow_split(const TraceArgs& a, uint32_t n) {
    return (MODE == kModeShadowRender && a.seg_count && n <= a.split_max && a.split > 1) ? a.split : 1u;
}

// Work item w of a shadow launch split into k segments per ray: segment
// w % k of ray w / k, over [b_s, b_s+1] with b_0 = tmin, b_k = tmax and the
// inner bounds computed by one expression, so neighbouring segments share
// their bound exactly and the closed intervals cover [tmin, tmax]; the ray is
// unoccluded iff all its segments are.
template <bool BRUTE, bool STATS>
__device__ __forceinline__ void trace_segment(const TraceArgs& a, const uint32_t* pre, uint32_t w, uint32_t k,
                                              TraceCounts& cnt) {
    const uint32_t i = w / k, seg = w - i * k;
    const uint32_t j = sub_entry(a, pre, i);
    float4 r0 = __ldg(a.rays + 2 * (size_t)j), r1 = __ldg(a.rays + 2 * (size_t)j + 1);
    const float t0 = r0.w, t1 = r1.w, len = __fsub_rn(t1, t0), inv_k = __frcp_rn((float)k);
    auto bound = [&](uint32_t q) { return q == 0 ? t0 : (q == k ? t1 : __fmaf_rn(len, __fmul_rn((float)q, inv_k), t0)); };
    r0.w = bound(seg);
    r1.w = bound(seg + 1);
    const RayHit h = trace_core<true, BRUTE, STATS>(a, a.tlas_nodes, a.inst, a.tlas_root, r0, r1, cnt);
    // low 16 bits: segments finished, high 16 bits: segments occluded (or
    // failed); the ray's last segment adds the contribution if none was, and
    // clears the count for the next launch
    const bool lit = !h.found && h.ok;
    const uint32_t old = atomicAdd(a.seg_count + i, lit ? 1u : 0x10001u);
    if ((old & 0xFFFFu) != k - 1) return;
    a.seg_count[i] = 0u;
    if (lit && (old >> 16) == 0u) {
        const Payload p = a.payload[j];
        float* px = a.image + 4 * (size_t)px_of(p.pixel);
        atomicAdd(px + 0, p.r);
        atomicAdd(px + 1, p.g);
        atomicAdd(px + 2, p.b);
    }
}

// Ray i of a queue (its entry via the sub-queues or the ring), traced and
// written out.
template <int MODE, bool BRUTE, bool STATS>
__device__ __forceinline__ void trace_ray(const TraceArgs& a, const uint32_t* pre, uint32_t head, uint32_t i,
                                          TraceCounts& cnt) {
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
    const RayHit h = trace_core<kAny, BRUTE, STATS>(a, tlas_nodes, tlas_inst, tlas_root, r0, r1, cnt);
    emit<MODE>(a, i, j, h.found, h.ok, h.t, h.id, h.prim, h.il, h.tl, h.V, h.W, h.det);
}

}  // namespace

}  // namespace rg
