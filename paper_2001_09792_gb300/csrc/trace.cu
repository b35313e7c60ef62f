// Ray traversal kernels of the two-level BVH (the per-ray code is in
// traverse.cuh): persistent warps pull rays from a global counter, 32 at a
// time (k_trace_warp), as lanes fall idle (k_trace_lane), or from two queues
// in one launch (k_trace_pair); k_trace8 walks the compressed 8-wide BVH.
#include <atomic>

#include "traverse.cuh"

namespace rg {

namespace {

// Binary traversal, whole-warp refill: a warp takes 32 rays from the work
// counter, each lane runs its ray to completion, and the warp takes the next
// 32 when all its lanes are done.  Best when the rays of a warp take similar
// work (camera and secondary rays).
template <int MODE, bool BRUTE, bool STATS, int BLOCK, int SD>
__global__ void __launch_bounds__(BLOCK) k_trace_warp(TraceArgs a) {
    constexpr bool kAny = (MODE == kModeAnyAbi || MODE == kModeShadowRender || MODE == kModeShadowBatch);
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t n = ray_count<MODE == kModeShadowRender>(a, pre);
    count_closest<MODE>(a, n);
    const int lane = threadIdx.x & 31;
    // batched closest-hit rays sit in a ring of 2^k entries from *ring_head
    const uint32_t head = MODE == kModeClosestBatch ? *a.ring_head : 0u;
    const uint32_t k = shadow_split<MODE>(a, n);
    const uint32_t items = n * k;
    TraceCounts cnt;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(a.work_counter, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= items) break;
        const uint32_t i = base + lane;
        if (i < items) {
            if (MODE == kModeShadowRender && k > 1)
                trace_segment<BRUTE, STATS, BLOCK, SD>(a, pre, i, k, cnt);
            else
                trace_ray<MODE, BRUTE, STATS, BLOCK, SD>(a, pre, head, i, cnt);
        }
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
// Launched for 1024 resident threads per SM (64 registers, 8 blocks of 128)
// at the cost of a few spilled values: with several frames in flight this
// measured 2.8 % faster than 896 threads (72 registers, no spills), one frame
// at a time the same, and 768 threads slower than both.
template <int SMODE, int CMODE, bool STATS, int BLOCK, int SD>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_trace_pair(TraceArgs sa, TraceArgs ca) {
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t ns_rays = ray_count<SMODE == kModeShadowRender>(sa, pre);
    const uint32_t k = shadow_split<SMODE>(sa, ns_rays);
    const uint32_t ns = ns_rays * k;  // shadow work items (segments)
    const uint32_t nc = ca.d_count ? *ca.d_count : ca.n;
    count_closest<CMODE>(ca, nc);
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
            if (i < ns) {
                if (SMODE == kModeShadowRender && k > 1)
                    trace_segment<false, STATS, BLOCK, SD>(sa, pre, i, k, cs);
                else
                    trace_ray<SMODE, false, STATS, BLOCK, SD>(sa, pre, 0u, i, cs);
            }
        } else {
            const uint32_t b = base - ns_pad;
            if (b >= nc) break;
            const uint32_t i = b + lane;
            if (i < nc) trace_ray<CMODE, false, STATS, BLOCK, SD>(ca, nullptr, head, i, cc);
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
// Leaf batching: every lane of the warp runs the node code in each
// iteration, but a triangle test or an instance entry runs its code for the
// lanes that need it, which on incoherent rays were one or two lanes in
// 71 % (triangles) and 54 % (instances) of the iterations.  A lane whose step
// is a triangle test (instance entry) therefore waits, its ray unchanged,
// until at least kLeafBatch lanes hold one or fewer than kLeafNodesMin lanes
// are left with a node to visit.  Each ray takes the same steps in the same
// order as without waiting, so the results do not change; on the large
// incoherent query the closest-hit launch took 10.5 against 11.2 ms.
// Timed instantiations are held to 64 registers (8 blocks of 128 per SM; the
// batched closest-hit mode to 72, 7 blocks), which they meet without spills.
// Node runs: a lane on an internal node takes up to kNodeRun node visits in
// one iteration (to the nearer child hit, or to an internal node popped from
// its stack) before the warp's votes of the next iteration.  The votes and
// the refill check run once per iteration for the whole warp, so the runs
// spread them over more visits; a longer run keeps the lanes that reached a
// leaf waiting.  On the large closest-hit query: 9.23 ms against 9.89 ms
// with single visits; runs of 3, 5, 6, 8, 16 took 9.24, 9.36, 9.46, 9.84 and
// 11.36 ms, and runs of 2 or 4 without the pops 9.90 and 9.31 ms.  The visits
// and their order per ray are unchanged.
constexpr int kLeafBatch = 4, kLeafNodesMin = 8, kNodeRun = 4;
template <int MODE, bool BRUTE, bool STATS, int BLOCK, int SD>
__global__ void __launch_bounds__(BLOCK, (BRUTE || STATS) ? 1 : (MODE == kModeClosestBatch ? 896 : 1024) / BLOCK)
    k_trace_lane(TraceArgs a) {
    const uint32_t iter_cap = a.iter_cap;
    constexpr bool kAny = (MODE == kModeAnyAbi || MODE == kModeShadowRender || MODE == kModeShadowBatch);
    constexpr bool kBatch = (MODE == kModeClosestBatch || MODE == kModeShadowBatch);
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t n = ray_count<MODE == kModeShadowRender>(a, pre);
    count_closest<MODE>(a, n);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t refill = a.refill;
    // batched closest-hit rays sit in a ring of 2^k entries from *ring_head
    const uint32_t head = MODE == kModeClosestBatch ? *a.ring_head : 0u;
    unsigned long long c_nodes = 0, c_tris = 0, c_inst = 0;

    bool active = false, exhausted = false;
    uint32_t i = 0, j = 0;  // ray index (dense) and queue entry
    const float4* tlas_nodes = a.tlas_nodes;
    const InstDev* tlas_inst = a.inst;
    float tmin = 0.f, tmax = 0.f;
    SpaceRay wr, cr;
    Shear sh;
    constexpr bool kTies = MODE == kModeClosestAbi;
    Best2 best;
    best.reset(0.f);
    float any_V = 0.f, any_W = 0.f, any_det = 1.f;
    bool found = false, ok = true, in_blas = false;
    ShortStack<BLOCK, SD> stack;
    int sp = 0;
    // the test limit on the stack applies to the counting instantiations only,
    // so the timed kernels compare with the constant
    const int smax = (STATS && a.stack_max >= 1 && a.stack_max < (uint32_t)kStack) ? (int)a.stack_max : kStack;
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
                    wr.ox = r0.x; wr.oy = r0.y; wr.oz = r0.z;
                    wr.ix = safe_rcp(r1.x); wr.iy = safe_rcp(r1.y); wr.iz = safe_rcp(r1.z);
                    cr = wr;
                    best.reset(tmax);
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
        const uint32_t act = __ballot_sync(0xFFFFFFFFu, active);
        if (act == 0u) break;
        // leaf batching: triangle tests and instance entries wait until
        // enough lanes of the warp hold one, or too few lanes are left on nodes
        const uint32_t bt = __ballot_sync(0xFFFFFFFFu, active && (ref & kLeaf) && in_blas);
        const uint32_t bi = __ballot_sync(0xFFFFFFFFu, active && (ref & kLeaf) && !in_blas);
        const bool few_nodes = __popc(act & ~bt & ~bi) < kLeafNodesMin;
        const bool wait = (ref & kLeaf) && !few_nodes && __popc(in_blas ? bt : bi) < kLeafBatch;
        if (!active) continue;

        bool finished = false;
        if (wait) {
            // the step is taken in a later iteration
        } else if (++iter > iter_cap) {
            record_error(a.st, RG_ERR_TIMEOUT);
            ok = false;
            finished = true;
        } else if (!(ref & kLeaf)) {
            for (int v = 0;;) {
                const float4* nd = nodes + 4 * (size_t)ref;
                const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2);
                const uint4 n3 = __ldg(reinterpret_cast<const uint4*>(nd + 3));
                if (STATS) ++c_nodes;
                const float tlim = kAny ? __fmul_rn(tmax, kCullSlack) : __fmul_rn(best.t, kCullSlack);
                float tn0, tn1, tf0, tf1;
                bool h0 = slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, cr, tmin, tlim, tn0, tf0);
                bool h1 = slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, cr, tmin, tlim, tn1, tf1);
                if (BRUTE) h0 = h1 = true;
                if (h0 && h1) {
                    if (sp >= smax) {
                        record_error(a.st, RG_ERR_STACK);
                        ok = false;
                        finished = true;
                        break;
                    } else {
                        const bool first0 = visit_first0<kAny>(tn0, tf0, tn1, tf1);
                        stack.put(sp++, first0 ? n3.y : n3.x);
                        ref = first0 ? n3.x : n3.y;
                    }
                } else {
                    ref = h0 ? n3.x : (h1 ? n3.y : kNone);
                }
                if (ref == kNone && sp > 0) {  // go on with a popped internal node
                    const uint32_t top = stack.get(sp - 1);
                    if (top != kMarker && !(top & kLeaf)) {
                        ref = top;
                        --sp;
                    }
                }
                if (++v >= kNodeRun || ref == kNone || (ref & kLeaf)) break;
                if (++iter > iter_cap) {
                    record_error(a.st, RG_ERR_TIMEOUT);
                    ok = false;
                    finished = true;
                    break;
                }
            }
        } else if (!in_blas) {
            // instance: enter its BLAS with the object-space ray
            const uint32_t leaf = ref & ~kLeaf;
            const InstDev* I = tlas_inst + leaf;
            const float4 m0 = __ldg(&I->inv[0]), m1 = __ldg(&I->inv[1]), m2 = __ldg(&I->inv[2]);
            const float4 meta0 = __ldg(reinterpret_cast<const float4*>(&I->nodes));  // nodes, tris
            const uint4 meta1 = __ldg(reinterpret_cast<const uint4*>(&I->root));     // root, id, mat, blas
            if (STATS) ++c_inst;
            // the world direction, read again (kept in registers it would
            // cost three for the whole ray)
            const float4 r1w = __ldg(a.rays + 2 * (size_t)j + 1);
            const float dx = r1w.x, dy = r1w.y, dz = r1w.z;
            const float ox = fmaf(m0.x, wr.ox, fmaf(m0.y, wr.oy, fmaf(m0.z, wr.oz, m0.w)));
            const float oy = fmaf(m1.x, wr.ox, fmaf(m1.y, wr.oy, fmaf(m1.z, wr.oz, m1.w)));
            const float oz = fmaf(m2.x, wr.ox, fmaf(m2.y, wr.oy, fmaf(m2.z, wr.oz, m2.w)));
            const float ddx = fmaf(m0.x, dx, fmaf(m0.y, dy, __fmul_rn(m0.z, dz)));
            const float ddy = fmaf(m1.x, dx, fmaf(m1.y, dy, __fmul_rn(m1.z, dz)));
            const float ddz = fmaf(m2.x, dx, fmaf(m2.y, dy, __fmul_rn(m2.z, dz)));
            if (sp >= smax) {
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
                stack.put(sp++, kMarker);
                ref = meta1.x;
            }
        } else {
            // triangle
            const uint32_t leaf = ref & ~kLeaf;
            const float4* tp = tri_rec(tris, leaf);
            const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
            if (STATS) ++c_tris;
            const float tlo = kAny ? tmax : (kTies && found ? fminf(__fmul_rn(best.t, kTieBand), tmax) : best.t);
            const TriResult h = tri_test(sh, v0, v1, v2, tmin, tlo);
            ref = kNone;
            if (h.hit) {
                const uint32_t prim = __float_as_uint(v0.w);
                if (kTies) {
                    if (best.offer(h.t, cur_id, prim)) found = true;
                } else if (kAny || h.t < best.t || cur_id < best.id || (cur_id == best.id && prim < best.prim)) {
                    best.t = h.t; best.id = cur_id; best.prim = prim;
                    best.il = cur_leaf; best.tl = leaf;
                    any_V = h.V; any_W = h.W; any_det = h.det;
                    found = true;
                }
                if (kAny) finished = true;
            }
        }
        // pop what the step left (the BLAS marker brings back the world-space ray)
        if (!finished && ref == kNone) {
            if (sp > 0) {
                ref = stack.get(--sp);
                if (ref == kMarker) {
                    in_blas = false;
                    nodes = tlas_nodes;
                    cr = wr;
                    ref = sp > 0 ? stack.get(--sp) : kNone;
                }
            }
            finished = ref == kNone;
        }
        if (finished) {
            emit<MODE>(a, i, j, found && ok, ok, best.t, best.id, best.prim, best.il, best.tl,
                       kTies ? best.tie_id() : kMiss, best.prim2, any_V, any_W, any_det);
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
// 8-byte entries.  Child boxes are tested with one FMA per plane on the
// byte's float v = 1 + q 2^-15 (built by a byte permute, exact):
// t = v * 2^15 S + (B - 2^15 S) with S = 2^e / d and B = (p - o) / d, which
// is q S + B up to a few roundings of magnitude 255 |S| + |B| and two of
// magnitude 2^15 |S| (at most 2^-9 |S| each).  Widening each axis' child
// intervals by E = kQuantErr (255 |S| + |B|) + 2^-7 |S| keeps the test
// conservative, so the wide path finds the same hits as the binary one.  A
// plane offset that overflows (or a zero direction component) becomes NaN,
// which leaves that axis open.
constexpr int kStack8 = 48;
constexpr uint32_t kKindNode = 0u, kKindItem = 1u << 30, kKindMarker = 2u << 30;
constexpr float kQuantErr = 8.0f * 5.9604644775390625e-08f;
constexpr float kPlaneErr = 0.0078125f;  // 2^-7
constexpr float kBias = 32768.0f;        // 2^15

__device__ __forceinline__ uint32_t oct_of(const SpaceRay& r) {
    return (__float_as_uint(r.ix) >> 31) | ((__float_as_uint(r.iy) >> 31) << 1) | ((__float_as_uint(r.iz) >> 31) << 2);
}

// Byte k of w as the float 1 + q 2^-15: one byte permute puts q in the
// second byte of the mantissa of 1.0 (bit pattern 0x3F80qq00).
__device__ __forceinline__ float byte_v(uint32_t w, int k) {
    return __uint_as_float(__byte_perm(w, 0x3F800000u, ((uint32_t)k << 4) | 0x7604u));
}

// Plane offset B - 2^15 S in one rounding; NaN where it overflows.
__device__ __forceinline__ float plane_offset(float S, float B) {
    const float c = fmaf(-kBias, S, B);
    return fabsf(c) < INFINITY ? c : __int_as_float(0x7FFFFFFF);
}

// Per-axis widening of the child intervals (see above).
__device__ __forceinline__ float plane_err(float S, float B) {
    return fmaf(kQuantErr, fmaf(255.0f, fabsf(S), fabsf(B)), kPlaneErr * fabsf(S));
}

template <int MODE, bool STATS>
__global__ void __launch_bounds__(kTraceBlock) k_trace8(TraceArgs a) {
    const uint32_t iter_cap = a.iter_cap;
    constexpr bool kAny = (MODE == kModeAnyAbi || MODE == kModeShadowRender);
    __shared__ uint32_t pre[kMaxLights + 1];
    const uint32_t n = ray_count<MODE == kModeShadowRender>(a, pre);
    count_closest<MODE>(a, n);
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

        constexpr bool kTies = MODE == kModeClosestAbi;
        Best2 best;
        best.reset(tmax);
        float any_V = 0.f, any_W = 0.f, any_det = 1.f;
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
                    const float Ux = Sx * kBias, Uy = Sy * kBias, Uz = Sz * kBias;  // exact (or inf)
                    const float Cx = plane_offset(Sx, Bx), Cy = plane_offset(Sy, By), Cz = plane_offset(Sz, Bz);
                    const float Ex = plane_err(Sx, Bx), Ey = plane_err(Sy, By), Ez = plane_err(Sz, Bz);
                    // near planes shifted down by E, far planes up by E
                    const float Bxn = Cx - Ex, Byn = Cy - Ey, Bzn = Cz - Ez;
                    const float Bxf = Cx + Ex, Byf = Cy + Ey, Bzf = Cz + Ez;
                    // near/far planes per axis from the direction signs
                    const bool nx = oct & 1, ny = oct & 2, nz = oct & 4;
                    const uint32_t nx0 = nx ? w3.z : w2.x, nx1 = nx ? w3.w : w2.y, fx0 = nx ? w2.x : w3.z, fx1 = nx ? w2.y : w3.w;
                    const uint32_t ny0 = ny ? w4.x : w2.z, ny1 = ny ? w4.y : w2.w, fy0 = ny ? w2.z : w4.x, fy1 = ny ? w2.w : w4.y;
                    const uint32_t nz0 = nz ? w4.z : w3.x, nz1 = nz ? w4.w : w3.y, fz0 = nz ? w3.x : w4.z, fz1 = nz ? w3.y : w4.w;
                    const float tlim = kAny ? __fmul_rn(tmax, kCullSlack) : __fmul_rn(best.t, kCullSlack);
                    const uint32_t meta_lo = w1.z, meta_hi = w1.w;
                    uint32_t hitmask = 0;
    #pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int k = c & 3;
                        const float tnx = fmaf(byte_v(c < 4 ? nx0 : nx1, k), Ux, Bxn);
                        const float tfx = fmaf(byte_v(c < 4 ? fx0 : fx1, k), Ux, Bxf);
                        const float tny = fmaf(byte_v(c < 4 ? ny0 : ny1, k), Uy, Byn);
                        const float tfy = fmaf(byte_v(c < 4 ? fy0 : fy1, k), Uy, Byf);
                        const float tnz = fmaf(byte_v(c < 4 ? nz0 : nz1, k), Uz, Bzn);
                        const float tfz = fmaf(byte_v(c < 4 ? fz0 : fz1, k), Uz, Bzf);
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
                    const float tlo =
                        kAny ? tmax : (kTies && found ? fminf(__fmul_rn(best.t, kTieBand), tmax) : best.t);
                    TriResult h = tri_test(sh, v0, v1, v2, tmin, tlo);
                    if (h.hit) {
                        const uint32_t prim = __float_as_uint(v0.w);
                        if (kAny) {
                            best.t = h.t; best.id = cur_id; best.prim = prim;
                            best.il = cur_leaf; best.tl = item;
                            any_V = h.V; any_W = h.W; any_det = h.det;
                            found = true;
                            done = true;
                            break;
                        }
                        if (kTies) {
                            if (best.offer(h.t, cur_id, prim)) found = true;
                        } else if (h.t < best.t || cur_id < best.id || (cur_id == best.id && prim < best.prim)) {
                            best.t = h.t; best.id = cur_id; best.prim = prim;
                            best.il = cur_leaf; best.tl = item;
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
        emit<MODE>(a, i, j, found, ok, best.t, best.id, best.prim, best.il, best.tl, kTies ? best.tie_id() : kMiss,
                   best.prim2, any_V, any_W, any_det);
    }
    flush_counts<kAny, STATS>(a, c_nodes, c_tris, c_inst);
}

template <int MODE, bool STATS>
cudaError_t launch_mode8(const TraceArgs& a, cudaStream_t s) {
    static std::atomic<int> cached{0};  // per process; concurrent first callers store the same value
    int blocks = cached.load(std::memory_order_relaxed);
    if (blocks == 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace8<MODE, STATS>, kTraceBlock, 0);
        if (e != cudaSuccess) return e;
        blocks = device_sm_count() * (per_sm > 0 ? per_sm : 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    k_trace8<MODE, STATS><<<blocks, kTraceBlock, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

// Resident blocks per SM of `kernel` with `smem` bytes of dynamic shared
// memory (the short stack), looked up once per process and instantiation
// (concurrent first callers store the same value).
template <class K>
cudaError_t resident_blocks(K kernel, int block, size_t smem, std::atomic<int>& cache, int* out) {
    int per_sm = cache.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
        if (e != cudaSuccess) return e;
        if (per_sm <= 0) per_sm = 1;
        cache.store(per_sm, std::memory_order_relaxed);
    }
    *out = per_sm;
    return cudaSuccess;
}

template <int MODE, bool BRUTE, bool STATS, int BLOCK, bool LANE, int SD>
cudaError_t launch_block(const TraceArgs& a, int blocks_per_sm, cudaStream_t s) {
    static std::atomic<int> cached{0};
    constexpr size_t smem = (size_t)SD * BLOCK * sizeof(uint32_t);
    int per_sm = 0;
    cudaError_t e = LANE ? resident_blocks(k_trace_lane<MODE, BRUTE, STATS, BLOCK, SD>, BLOCK, smem, cached, &per_sm)
                         : resident_blocks(k_trace_warp<MODE, BRUTE, STATS, BLOCK, SD>, BLOCK, smem, cached, &per_sm);
    if (e != cudaSuccess) return e;
    const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
    if (LANE)
        k_trace_lane<MODE, BRUTE, STATS, BLOCK, SD><<<device_sm_count() * b, BLOCK, smem, s>>>(a);
    else
        k_trace_warp<MODE, BRUTE, STATS, BLOCK, SD><<<device_sm_count() * b, BLOCK, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int SMODE, int CMODE, bool STATS, int BLOCK, int SD>
cudaError_t launch_pair_t(const TraceArgs& sa, const TraceArgs& ca, int blocks_per_sm, cudaStream_t s) {
    static std::atomic<int> cached{0};
    constexpr size_t smem = (size_t)SD * BLOCK * sizeof(uint32_t);
    int per_sm = 0;
    cudaError_t e = resident_blocks(k_trace_pair<SMODE, CMODE, STATS, BLOCK, SD>, BLOCK, smem, cached, &per_sm);
    if (e != cudaSuccess) return e;
    const int b = (blocks_per_sm > 0 && blocks_per_sm < per_sm) ? blocks_per_sm : per_sm;
    k_trace_pair<SMODE, CMODE, STATS, BLOCK, SD><<<device_sm_count() * b, BLOCK, smem, s>>>(sa, ca);
    count_launches(1);
    return cudaGetLastError();
}

// Refill threshold when the shape leaves it open (0): per-lane refill for the
// queries of rg_trace_rays, whose rays are often incoherent (8 idle lanes for
// closest hits; 16 for any hits: 3.51 ms on the large any-hit query, 3.53 ms
// with 8, against 3.66 ms for whole-warp refill once node runs cut the
// per-lane kernel's votes); whole-warp refill elsewhere (faster on the
// renderer's camera, secondary and shadow rays, as measured on GB300).
template <int MODE>
constexpr int default_refill() {
    return MODE == kModeClosestAbi ? 8 : (MODE == kModeAnyAbi ? 16 : 32);
}

// Launch of one binary-traversal mode.  Shapes other than 128 threads are
// compiled for the render and batched modes (the ones the autotuner sets);
// the rest run with 128.  refill < 32 selects the per-lane-refill kernel, 32
// the whole-warp one.  The batched modes at 128 threads are also compiled with
// a short stack of 8 or 16 entries in shared memory (shape.stack), which the
// autotuner chooses among; everything else keeps the whole stack in local
// memory (measured fastest for the render and query kernels).
template <int MODE, bool BRUTE, bool STATS, bool LANE>
cudaError_t launch_block_128(const TraceArgs& a, const TraceShape& shape, cudaStream_t s) {
    constexpr bool kBatch = MODE == kModeClosestBatch || MODE == kModeShadowBatch;
    if constexpr (kBatch && !BRUTE && !STATS) {
        if (shape.stack == 8) return launch_block<MODE, BRUTE, STATS, 128, LANE, 8>(a, shape.blocks_per_sm, s);
        if (shape.stack == 16) return launch_block<MODE, BRUTE, STATS, 128, LANE, 16>(a, shape.blocks_per_sm, s);
    }
    return launch_block<MODE, BRUTE, STATS, 128, LANE, 0>(a, shape.blocks_per_sm, s);
}

template <int MODE, bool BRUTE, bool STATS>
cudaError_t launch_mode(const TraceArgs& a0, cudaStream_t s, const TraceShape& shape = TraceShape()) {
    TraceArgs a = a0;
    const int refill = (shape.refill >= 1 && shape.refill <= 32) ? shape.refill : default_refill<MODE>();
    a.refill = (uint32_t)refill;
    constexpr bool kTunable = !BRUTE && !STATS && MODE >= kModeClosestRender;
    if (refill < 32) {
        if constexpr (kTunable) {
            if (shape.block == 64) return launch_block<MODE, BRUTE, STATS, 64, true, 0>(a, shape.blocks_per_sm, s);
            if (shape.block == 256) return launch_block<MODE, BRUTE, STATS, 256, true, 0>(a, shape.blocks_per_sm, s);
        }
        return launch_block_128<MODE, BRUTE, STATS, true>(a, shape, s);
    }
    if constexpr (kTunable) {
        if (shape.block == 64) return launch_block<MODE, BRUTE, STATS, 64, false, 0>(a, shape.blocks_per_sm, s);
        if (shape.block == 256) return launch_block<MODE, BRUTE, STATS, 256, false, 0>(a, shape.blocks_per_sm, s);
    }
    return launch_block_128<MODE, BRUTE, STATS, false>(a, shape, s);
}

// Completes one provisional ABI hit record of a traversal launch (emit;
// record i is a hit): t, u, v of the chosen triangle recomputed exactly
// (refine_hit), and, when the traversal found a runner-up within the tie band,
// the two candidates decided again on their exact distances rounded to
// float32, then instance, then primitive (the tie rule).  t is kept within the
// ray's [tmin, tmax], which the float32 test enforced.  Both traversals (binary
// and wide) name candidates by (instance, prim); the binary TLAS's instance
// records and the BLAS triangle records locate them.
__device__ __forceinline__ void refine_one(const float4* __restrict__ rays, rg_hit* __restrict__ hits, uint32_t i,
                                           const InstDev* __restrict__ inst, const uint32_t* __restrict__ leaf_of_inst,
                                           const BlasDev* __restrict__ blas) {
    uint32_t* rec = reinterpret_cast<uint32_t*>(hits + i);
    uint32_t id = rec[0], prim = rec[1];
    const uint32_t id2 = rec[3], prim2 = rec[4];
    const float t0 = __uint_as_float(rec[2]);
    const float4 r0 = __ldg(rays + 2 * (size_t)i), r1 = __ldg(rays + 2 * (size_t)i + 1);
    auto candidate = [&](uint32_t cid, uint32_t cprim) {
        const InstDev* I = inst + __ldg(leaf_of_inst + cid);
        const float4 m0 = __ldg(&I->m[0]), m1 = __ldg(&I->m[1]), m2 = __ldg(&I->m[2]);
        const float4 meta0 = __ldg(reinterpret_cast<const float4*>(&I->nodes));  // nodes, tris
        const uint32_t b = __ldg(&I->blas);
        const float4* tris = reinterpret_cast<const float4*>(
            ((unsigned long long)__float_as_uint(meta0.w) << 32) | __float_as_uint(meta0.z));
        const uint32_t* lp = reinterpret_cast<const uint32_t*>(__ldg(reinterpret_cast<const unsigned long long*>(
            &blas[b].leaf_of_prim)));
        const float4* tp = tris + kTriStride * (size_t)__ldg(lp + cprim);  // axis order (x, y, z)
        const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
        Refined q = refine_hit(r0, r1, t0, m0, m1, m2, v0, v1, v2);
        q.t = fminf(fmaxf(q.t, r0.w), r1.w);
        return q;
    };
    Refined q = candidate(id, prim);
    if (id2 != kMiss) {
        const Refined q2 = candidate(id2, prim2);
        if (hit_before(q2.t, id2, prim2, q.t, id, prim)) {
            q = q2;
            id = id2;
            prim = prim2;
        }
    }
    rec[0] = id;
    rec[1] = prim;
    rec[2] = __float_as_uint(q.t);
    rec[3] = __float_as_uint(q.u);
    rec[4] = __float_as_uint(q.v);
}

// The exact attributes of every closest hit.  Misses are already final.  A
// warp walks tiles of 32 records and queues the hits' indices in shared
// memory (ballots), then refines them 32 at a time, so the long float-float
// path runs with full warps whatever the hit rate.
constexpr int kRefineBlock = 256;
__global__ void __launch_bounds__(kRefineBlock, 4) k_refine_hits(const float4* __restrict__ rays,
                                                              rg_hit* __restrict__ hits, uint32_t n,
                                                              const InstDev* __restrict__ inst,
                                                              const uint32_t* __restrict__ leaf_of_inst,
                                                              const BlasDev* __restrict__ blas) {
    __shared__ uint32_t queue[kRefineBlock / 32][64];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t* q = queue[warp];
    uint32_t qn = 0;  // queued hits (the same in every lane)
    const size_t stride = (size_t)gridDim.x * kRefineBlock;
    for (size_t tile = ((size_t)blockIdx.x * kRefineBlock + warp * 32u); tile < n; tile += stride) {
        const size_t i = tile + lane;
        const bool hit = i < n && reinterpret_cast<const uint32_t*>(hits + i)[0] != kMiss;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, hit);
        if (hit) q[qn + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
        qn += __popc(bal);
        __syncwarp();
        if (qn >= 32) {
            refine_one(rays, hits, q[lane], inst, leaf_of_inst, blas);
            __syncwarp();
            if (lane + 32u < qn) q[lane] = q[lane + 32u];
            qn -= 32;
            __syncwarp();
        }
    }
    if (lane < qn) refine_one(rays, hits, q[lane], inst, leaf_of_inst, blas);
}

}  // namespace

cudaError_t launch_refine_hits(const float4* rays, rg_hit* hits, uint32_t n, const InstDev* inst,
                               const uint32_t* leaf_of_inst, const BlasDev* blas, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = min((n + kRefineBlock - 1u) / kRefineBlock, (uint32_t)device_sm_count() * 8u);
    k_refine_hits<<<blocks, kRefineBlock, 0, s>>>(rays, hits, n, inst, leaf_of_inst, blas);
    count_launches(1);
    return cudaGetLastError();
}

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
            return stats ? launch_mode<kModeClosestAbi, false, true>(a, s, shape)
                         : launch_mode<kModeClosestAbi, false, false>(a, s, shape);
        case kModeAnyAbi:
            if (brute) return launch_mode<kModeAnyAbi, true, false>(a, s);
            return stats ? launch_mode<kModeAnyAbi, false, true>(a, s, shape)
                         : launch_mode<kModeAnyAbi, false, false>(a, s, shape);
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
            return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 64, 0>(sa, ca, shape.blocks_per_sm, s);
        if (shape.block == 256)
            return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 256, 0>(sa, ca, shape.blocks_per_sm, s);
        if (shape.stack == 8)
            return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 128, 8>(sa, ca, shape.blocks_per_sm, s);
        if (shape.stack == 16)
            return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 128, 16>(sa, ca, shape.blocks_per_sm, s);
        return launch_pair_t<kModeShadowBatch, kModeClosestBatch, false, 128, 0>(sa, ca, shape.blocks_per_sm, s);
    }
    return stats ? launch_pair_t<kModeShadowRender, kModeClosestRender, true, kTraceBlock, 0>(sa, ca, 0, s)
                 : launch_pair_t<kModeShadowRender, kModeClosestRender, false, kTraceBlock, 0>(sa, ca, 0, s);
}

}  // namespace rg
