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

// Short traversal stack: the first SD entries of each thread's stack live in
// the block's dynamic shared memory, the deeper ones in the thread's local
// array (cached in L1).  Column layout: entry k of thread t is
// rg_sstack[k * BLOCK + t], so the lanes of a warp touch 32 different banks
// whatever depths they are at.  SD = 0 is the plain local-memory stack.
extern __shared__ uint32_t rg_sstack[];

template <int BLOCK, int SD>
struct ShortStack {
    uint32_t lo[kTraceStack];
    __device__ __forceinline__ void put(int i, uint32_t v) {
        if (SD > 0 && i < SD)
            rg_sstack[i * BLOCK + threadIdx.x] = v;
        else
            lo[i] = v;
    }
    __device__ __forceinline__ uint32_t get(int i) const {
        return (SD > 0 && i < SD) ? rg_sstack[i * BLOCK + threadIdx.x] : lo[i];
    }
};
constexpr int kTraceBlock = 128;
// 1 + 2 * gamma_3, gamma_3 = 3u / (1 - 3u), u = 2^-24
constexpr float kIze = 1.0f + 2.0f * (3.0f * 5.9604644775390625e-08f) / (1.0f - 3.0f * 5.9604644775390625e-08f);
constexpr float kCullSlack = 1.0f + 1.0f / 4096.0f;
// Closest-hit queries of the ABI keep, beside the best candidate, the next one
// in the order (t, instance, prim); when its float32 distance lies within this
// relative band of the best one, the two are decided again on their exact
// distances (k_refine_hits).  The band is a quarter of the culling slack, so a
// box holding such a candidate is never culled and every traversal (binary,
// wide, brute force) sees the same pair.
constexpr float kTieBand = 1.0f + 1.0f / 16384.0f;

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
// Closest-hit ABI queries write a provisional record that k_refine_hits
// completes: for a hit {instance, prim, float32 t, runner-up instance or kMiss,
// runner-up prim}; a miss is written in its final form.  Any-hit ABI queries (only occluded / not is defined) write
// their final record: the hit's ids, float32 t and barycentrics V/det, W/det
// of the watertight test.
template <int MODE>
__device__ __forceinline__ void emit(const TraceArgs& a, uint32_t i, uint32_t j, bool found, bool ok, float best_t, uint32_t best_id,
                                     uint32_t best_prim, uint32_t best_il, uint32_t best_tl, uint32_t run_il = kMiss,
                                     uint32_t run_tl = kMiss, float any_V = 0.f, float any_W = 0.f, float any_det = 1.f) {
    if (MODE == kModeClosestAbi || MODE == kModeAnyAbi) {
        rg_hit out;
        if (found && MODE == kModeAnyAbi) {
            out.instance = best_id;
            out.prim = best_prim;
            out.t = best_t;
            out.u = __fdiv_rn(any_V, any_det);
            out.v = __fdiv_rn(any_W, any_det);
        } else if (found) {
            out.instance = best_id;
            out.prim = best_prim;
            out.t = best_t;
            out.u = __uint_as_float(run_il);
            out.v = __uint_as_float(run_tl);
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
    float t;
    uint32_t id, prim, il, tl;
    uint32_t id2, prim2;  // ABI closest hit: the runner-up within kTieBand of t (id2 = kMiss: none)
    float V, W, det;    // any hit: the watertight test's V, W and det of the hit
};

// Order of closest-hit candidates: distance, then instance, then primitive.
__device__ __forceinline__ bool hit_before(float t, uint32_t id, uint32_t prim, float t0, uint32_t id0, uint32_t prim0) {
    return t < t0 || (t == t0 && (id < id0 || (id == id0 && prim < prim0)));
}

// The two first candidates of a closest-hit query in hit_before order.
struct Best2 {
    float t, t2;
    uint32_t id, prim, il, tl;  // il, tl: TLAS leaf and BLAS leaf of the best (the renderer's hit record)
    uint32_t id2, prim2;
    __device__ __forceinline__ void reset(float tmax) {
        t = tmax;
        t2 = __int_as_float(0x7F800000);
        id = prim = il = tl = kMiss;
        id2 = prim2 = kMiss;
    }
    // ABI closest hit (no leaf indices kept); returns true when c became the best
    __device__ __forceinline__ bool offer(float ct, uint32_t cid, uint32_t cprim) {
        if (hit_before(ct, cid, cprim, t, id, prim)) {
            if (id != kMiss) {
                t2 = t; id2 = id; prim2 = prim;
            }
            t = ct; id = cid; prim = cprim;
            return true;
        }
        if (hit_before(ct, cid, cprim, t2, id2, prim2)) {
            t2 = ct; id2 = cid; prim2 = cprim;
        }
        return false;
    }
    // the runner-up's instance, if it lies within the tie band of the best (else kMiss)
    __device__ __forceinline__ uint32_t tie_id() const { return (id2 != kMiss && t2 <= __fmul_rn(t, kTieBand)) ? id2 : kMiss; }
};

// One ray, run to completion: one loop iteration per node visit, instance
// entry or triangle test; a stack pop joins the step that follows it.  The ray
// is r0 = (origin, tmin), r1 = (direction, tmax) in world space; ANY: the
// first hit ends it.
// TIES (closest-hit queries of the ABI): also keep the runner-up (Best2), and
// test triangles up to the tie band beyond the best distance.  BLOCK: the
// launch's threads per block (the short stack's column stride).
template <bool ANY, bool BRUTE, bool STATS, int BLOCK, int SD, bool TIES = false>
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

    Best2 best;
    best.reset(tmax);
    float any_V = 0.f, any_W = 0.f, any_det = 1.f;
    // culling distance of the box tests: the ray's end (any hit) or the best
    // hit so far (closest hit), with the relative slack
    float tlim = __fmul_rn(tmax, kCullSlack);
    bool found = false;

    ShortStack<BLOCK, SD> stack;
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
            ref = stack.get(--sp);
            if (ref == kMarker) {
                in_blas = false;
                nodes = tlas_nodes;
                cr = wr;
                if (sp == 0) break;
                ref = stack.get(--sp);  // a TLAS entry: markers never follow each other
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
                stack.put(sp++, farc);
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
            stack.put(sp++, kMarker);
            ref = meta1.x;
            continue;
        }
        // triangle leaf
        {
            const float4* tp = tri_rec(tris, leaf);
            const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
            if (STATS) ++cnt.tris;
            const float tlo = kAny ? tmax : (TIES && found ? fminf(__fmul_rn(best.t, kTieBand), tmax) : best.t);
            TriResult h = tri_test(sh, v0, v1, v2, tmin, tlo);
            ref = kNone;
            if (h.hit) {
                const uint32_t prim = __float_as_uint(v0.w);
                if (kAny) {
                    best.t = h.t; best.id = cur_id; best.prim = prim;
                    best.il = cur_leaf; best.tl = leaf;
                    any_V = h.V; any_W = h.W; any_det = h.det;
                    found = true;
                    break;
                }
                if (TIES) {
                    if (best.offer(h.t, cur_id, prim)) {
                        tlim = __fmul_rn(best.t, kCullSlack);
                        found = true;
                    }
                } else if (h.t < best.t || cur_id < best.id || (cur_id == best.id && prim < best.prim)) {
                    best.t = h.t; best.id = cur_id; best.prim = prim;
                    best.il = cur_leaf; best.tl = leaf;
                    tlim = __fmul_rn(best.t, kCullSlack);
                    found = true;
                }
            }
        }
    }
    RayHit h;
    h.found = found && ok;
    h.ok = ok;
    h.t = best.t;
    h.id = best.id;
    h.prim = best.prim;
    h.il = best.il;
    h.tl = best.tl;
    h.id2 = TIES ? best.tie_id() : kMiss;
    h.prim2 = best.prim2;
    h.V = any_V;
    h.W = any_W;
    h.det = any_det;
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
template <bool BRUTE, bool STATS, int BLOCK, int SD>
__device__ __forceinline__ void trace_segment(const TraceArgs& a, const uint32_t* pre, uint32_t w, uint32_t k,
                                              TraceCounts& cnt) {
    const uint32_t i = w / k, seg = w - i * k;
    const uint32_t j = sub_entry(a, pre, i);
    float4 r0 = __ldg(a.rays + 2 * (size_t)j), r1 = __ldg(a.rays + 2 * (size_t)j + 1);
    const float t0 = r0.w, t1 = r1.w, len = __fsub_rn(t1, t0), inv_k = __frcp_rn((float)k);
    auto bound = [&](uint32_t q) { return q == 0 ? t0 : (q == k ? t1 : __fmaf_rn(len, __fmul_rn((float)q, inv_k), t0)); };
    r0.w = bound(seg);
    r1.w = bound(seg + 1);
    const RayHit h = trace_core<true, BRUTE, STATS, BLOCK, SD>(a, a.tlas_nodes, a.inst, a.tlas_root, r0, r1, cnt);
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
template <int MODE, bool BRUTE, bool STATS, int BLOCK, int SD>
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
    const RayHit h =
        trace_core<kAny, BRUTE, STATS, BLOCK, SD, MODE == kModeClosestAbi>(a, tlas_nodes, tlas_inst, tlas_root, r0, r1, cnt);
    emit<MODE>(a, i, j, h.found, h.ok, h.t, h.id, h.prim, h.il, h.tl, h.id2, h.prim2, h.V, h.W, h.det);
}


// ---------------------------------------------------------------- exact hit attributes
// The ABI's hit records carry t, u, v of the chosen triangle to far better
// than float32 resolution of the scene: a float32 evaluation loses about
// 2^-24 of the ray's travel distance and of the coordinates' magnitude, which
// is far beyond 1e-5 of u for a small triangle seen from afar, or of t for a
// hit close to an origin far from the world origin.  k_refine_hits recomputes
// them in float-float arithmetic (a value is the unevaluated sum hi + lo of two
// floats) from the exact float32 inputs: the world ray (o, d), the instance's
// object-to-world rows [A | T] and the triangle's object-space vertices.
//
//   c_i = A v_i + T - (o + t0 d)       vertex i seen from the float32 hit
//                                      point, exact to ~2^-44 of the terms
//   X0 = c1 x c2, X1 = c2 x c0, X2 = c0 x c1
//   E_i = d . X_i                      signed volume spanned by d and the edge
//                                      opposite vertex i (the edge functions of
//                                      the watertight test, free of the shear)
//   u = E_1 / (E_0 + E_1 + E_2),  v = E_2 / (E_0 + E_1 + E_2)
//   t = t0 + det(c0, c1, c2) / (E_0 + E_1 + E_2)
//
// E_i does not change when the origin slides along d, and det(c0, c1, c2) is
// (t - t0) times the same sum, so no step depends on t0 being accurate; t0
// only keeps the magnitudes of c_i near the triangle's size.  Error-free
// transformations: Knuth's TwoSum and the FMA product (Dekker; Ogita, Rump &
// Oishi 2005, "Accurate sum and dot product"), with every operation an
// explicit intrinsic so no contraction changes the roundings.
struct FF {
    float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ FF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// row . v + B (row, v exact floats, B float-float)
__device__ __forceinline__ FF affine_ff(float4 row, float4 v, FF B) {
    const FF p0 = two_prod(row.x, v.x), p1 = two_prod(row.y, v.y), p2 = two_prod(row.z, v.z);
    const FF s0 = two_sum(B.h, p0.h);
    const FF s1 = two_sum(s0.h, p1.h);
    const FF s2 = two_sum(s1.h, p2.h);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(B.l, p0.l), __fadd_rn(p1.l, p2.l)),
                               __fadd_rn(__fadd_rn(s0.l, s1.l), s2.l));
    return two_sum(s2.h, lo);
}

// a1 b2 - a2 b1 in float-float
__device__ __forceinline__ FF cross_ff(FF a1, FF b2, FF a2, FF b1) {
    const FF p = two_prod(a1.h, b2.h), q = two_prod(a2.h, b1.h);
    const FF s = two_sum(p.h, -q.h);
    const float cross_lo = __fsub_rn(__fmaf_rn(a1.h, b2.l, __fmul_rn(a1.l, b2.h)),
                                     __fmaf_rn(a2.h, b1.l, __fmul_rn(a2.l, b1.h)));
    return two_sum(s.h, __fadd_rn(__fadd_rn(__fsub_rn(p.l, q.l), s.l), cross_lo));
}

// x . y for float-float vectors (x0 may have a zero lo part), rounded once at the end
__device__ __forceinline__ float dot_ff(FF x0, FF x1, FF x2, FF y0, FF y1, FF y2) {
    const FF p0 = two_prod(x0.h, y0.h), p1 = two_prod(x1.h, y1.h), p2 = two_prod(x2.h, y2.h);
    const FF s0 = two_sum(p0.h, p1.h);
    const FF s1 = two_sum(s0.h, p2.h);
    const float cross_lo = __fadd_rn(__fadd_rn(__fmaf_rn(x0.h, y0.l, __fmul_rn(x0.l, y0.h)),
                                               __fmaf_rn(x1.h, y1.l, __fmul_rn(x1.l, y1.h))),
                                     __fmaf_rn(x2.h, y2.l, __fmul_rn(x2.l, y2.h)));
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(p0.l, p1.l), __fadd_rn(p2.l, s0.l)), __fadd_rn(s1.l, cross_lo));
    return __fadd_rn(s1.h, lo);
}

struct Refined {
    float t, u, v;
};

// t, u, v of the ray (o, d) against one triangle of one instance, from the
// approximate distance t0 (see above).  m: the instance's object-to-world rows
// {A_k0, A_k1, A_k2, T_k}; v0..v2: object-space vertices (x, y, z).  If the
// ray is parallel to the triangle's plane (no finite solution), t0 is kept
// and u = v = 0.
__device__ __forceinline__ Refined refine_hit(float4 r0, float4 r1, float t0, float4 m0, float4 m1, float4 m2,
                                              float4 v0, float4 v1, float4 v2) {
    // B_k = T_k - o_k - t0 d_k
    auto base = [&](float T, float o, float d) {
        const FF a = two_sum(T, -o);
        const FF p = two_prod(t0, d);
        const FF b = two_sum(a.h, -p.h);
        return two_sum(b.h, __fadd_rn(__fsub_rn(a.l, p.l), b.l));
    };
    const FF Bx = base(m0.w, r0.x, r1.x), By = base(m1.w, r0.y, r1.y), Bz = base(m2.w, r0.z, r1.z);
    const FF c0x = affine_ff(m0, v0, Bx), c0y = affine_ff(m1, v0, By), c0z = affine_ff(m2, v0, Bz);
    const FF c1x = affine_ff(m0, v1, Bx), c1y = affine_ff(m1, v1, By), c1z = affine_ff(m2, v1, Bz);
    const FF c2x = affine_ff(m0, v2, Bx), c2y = affine_ff(m1, v2, By), c2z = affine_ff(m2, v2, Bz);
    const FF zero = {0.f, 0.f};
    const FF dx = {r1.x, 0.f}, dy = {r1.y, 0.f}, dz = {r1.z, 0.f};
    // X0 = c1 x c2
    const FF X0x = cross_ff(c1y, c2z, c1z, c2y), X0y = cross_ff(c1z, c2x, c1x, c2z), X0z = cross_ff(c1x, c2y, c1y, c2x);
    const float E0 = dot_ff(dx, dy, dz, X0x, X0y, X0z);
    const float D = dot_ff(c0x, c0y, c0z, X0x, X0y, X0z);
    // X1 = c2 x c0
    const FF X1x = cross_ff(c2y, c0z, c2z, c0y), X1y = cross_ff(c2z, c0x, c2x, c0z), X1z = cross_ff(c2x, c0y, c2y, c0x);
    const float E1 = dot_ff(dx, dy, dz, X1x, X1y, X1z);
    // X2 = c0 x c1
    const FF X2x = cross_ff(c0y, c1z, c0z, c1y), X2y = cross_ff(c0z, c1x, c0x, c1z), X2z = cross_ff(c0x, c1y, c0y, c1x);
    const float E2 = dot_ff(dx, dy, dz, X2x, X2y, X2z);
    (void)zero;
    const float det = __fadd_rn(__fadd_rn(E0, E1), E2);
    Refined r;
    const float dt = __fdiv_rn(D, det);
    if (!(fabsf(det) > 0.f) || !(fabsf(dt) < INFINITY)) {
        r.t = t0;
        r.u = r.v = 0.f;
        return r;
    }
    r.t = __fadd_rn(t0, dt);
    r.u = __fdiv_rn(E1, det);
    r.v = __fdiv_rn(E2, det);
    return r;
}

}  // namespace

}  // namespace rg
