// Wavefront Whitted renderer (paper Sec. 2.1: multiple objects, shadow
// casting, reflection and refraction; Sec. 1: the ray-generation shader casts
// the initial rays, hit shaders spawn further rays up to a fixed depth, and a
// payload travels with each ray).
//
// Instead of recursion, every depth level is one queue of rays with a 16 B
// payload (pixel, RGB weight).  Per level: closest-hit traversal of the queue,
// then k_shade turns each hit into (a) radiance added to the image (misses:
// background; diffuse: ambient), (b) one shadow ray per light facing the
// surface, carrying its unshadowed Lambert contribution, and (c) reflection /
// refraction rays for the next level.  Shadow rays run through any-hit
// traversal, which adds the contribution of every unoccluded one.  Queue slots
// are claimed with one atomic per warp (warp prefix sums over the per-thread
// counts).
//
// Shading model (a reading of Sec. 2.1, which names the effects only):
//   n  = normalize(Minv^T ((v1-v0) x (v2-v0))), flipped to face the ray (nf);
//   p  = o + t d;  offset eps = 1e-4 * max(1, max_i |p_i|);
//   diffuse: a*ambient + sum_l a*I_l*max(0, nf.l) * visible(p + eps nf -> light);
//   mirror : tint * L(reflect(d, nf)) from p + eps nf;
//   glass  : Schlick R, R*L(reflect) + (1-R)*L(refract) (refracted ray from
//            p - eps nf), or L(reflect) on total internal reflection;
//   miss   : background; alpha = 1 where the primary ray hit.
#include "rg_internal.cuh"

namespace rg {

namespace {

// Shading blocks of 128 threads: the block-wide queue claims wait at two
// barriers, and smaller blocks wait for fewer warps; with several frames in
// flight 128 measured 1.9 % faster than 256 (one frame at a time 1.5 %
// slower), 512 slower in both.
constexpr int kShadeBlock = 128;

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) { return rsqrtf(dot3(a, a)) * a; }

// Pinhole camera ray through the centre of pixel (x, y), row 0 at the top.
__device__ __forceinline__ void camera_ray(const CameraDev& cam, uint32_t w, uint32_t h, uint32_t x, uint32_t y,
                                           float4& o, float4& dir) {
    float3 eye = f3(cam.eye[0], cam.eye[1], cam.eye[2]);
    float3 F = normalize3(f3(cam.target[0], cam.target[1], cam.target[2]) - eye);
    float3 R = normalize3(cross3(F, f3(cam.up[0], cam.up[1], cam.up[2])));
    float3 U = cross3(R, F);
    float th = tanf(0.5f * cam.vfov_deg * 0.017453292519943295f);
    float aspect = (float)w / (float)h;
    float px = (2.0f * ((float)x + 0.5f) / (float)w - 1.0f) * aspect * th;
    float py = (1.0f - 2.0f * ((float)y + 0.5f) / (float)h) * th;
    float3 d = normalize3(px * R + py * U + F);
    o = make_float4(eye.x, eye.y, eye.z, 0.0f);
    dir = make_float4(d.x, d.y, d.z, __int_as_float(0x7F800000));
}

// Pixel of primary ray i: rays run over 8x4 tiles (a warp's 32 rays cover
// one tile, which keeps their paths together longer than a 32x1 strip).
// The image is cut into bands of 4 rows (the last band may be thinner),
// each band into blocks of 8 columns (the last may be narrower), pixels row
// by row inside a block; a bijection of [0, w h) onto the pixels.
__device__ __forceinline__ void tile_pixel(uint32_t i, uint32_t w, uint32_t h, uint32_t& x, uint32_t& y) {
    const uint32_t band = i / (4u * w);
    const uint32_t rows = min(4u, h - 4u * band);
    const uint32_t local = i - band * 4u * w;
    const uint32_t blk = local / (8u * rows);
    const uint32_t bw = min(8u, w - 8u * blk);
    const uint32_t rem = local - blk * 8u * rows;
    y = 4u * band + rem / bw;
    x = 8u * blk + rem % bw;
}

__global__ void k_raygen(CameraDev cam, uint32_t w, uint32_t h, float4* __restrict__ rays,
                         Payload* __restrict__ payload) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w * h) return;
    uint32_t x, y;
    tile_pixel(i, w, h, x, y);
    float4 o, d;
    camera_ray(cam, w, h, x, y, o, d);
    rays[2 * (size_t)i] = o;
    rays[2 * (size_t)i + 1] = d;
    Payload p;
    p.pixel = y * w + x;
    p.r = p.g = p.b = 1.0f;
    payload[i] = p;
}

// Queue slots of one shading round, claimed per block: for each queue (one
// per light, then the next level's path rays) every warp adds its count
// (ballots: a ray wants 0 or 1 shadow rays per light and 0, 1 or 2 path rays)
// to a shared-memory total, and the block makes one atomicAdd per queue on
// its tail.  The tails are single addresses that every block of a level
// appends to; claims per warp measured 6 % of the frame slower, and a round
// per queue costs two barriers each.
struct ClaimSmem {
    uint32_t cnt[kMaxLights + 1];
    uint32_t base[kMaxLights + 1];
    uint32_t woff[kShadeBlock / 32][kMaxLights + 1];
};

__device__ __forceinline__ void claim_init(ClaimSmem* cs) {
    for (uint32_t q = threadIdx.x; q <= kMaxLights; q += blockDim.x) cs->cnt[q] = 0u;
}


struct Surf {
    float3 p, nf, d;
    float eps;
    bool entering;
};

// What one ray's shading needs besides the ray: the tables of its scene or
// request slot, its image, its depth and its pixel.
struct RayCtx {
    const InstDev* inst;
    const rg_material* mats;
    const rg_light* lights;
    float* image;
    uint32_t n_mats, n_lights, depth, max_depth, pixel, slot;
    float bg[3];
    float ambient;
};

template <bool BATCH>
__device__ __forceinline__ RayCtx ray_ctx(const ShadeArgs& a, const SlotDev* slots, uint32_t pw) {
    RayCtx c;
    if (BATCH) {
        const SlotDev* S = slots + slot_of_px(pw);
        c.inst = S->inst;
        c.mats = S->mats;
        c.lights = S->lights;
        c.image = S->image;
        c.n_mats = S->n_mats;
        c.n_lights = S->n_lights;
        c.max_depth = S->max_depth;
        c.bg[0] = S->bg[0];
        c.bg[1] = S->bg[1];
        c.bg[2] = S->bg[2];
        c.ambient = S->ambient;
        c.depth = depth_of(pw);
        c.pixel = px_of(pw);
        c.slot = slot_of_px(pw);
    } else {
        c.inst = a.inst;
        c.mats = a.mats;
        c.lights = a.lights;
        c.image = a.image;
        c.n_mats = a.n_mats;
        c.n_lights = a.n_lights;
        c.max_depth = a.max_depth;
        c.bg[0] = a.bg[0];
        c.bg[1] = a.bg[1];
        c.bg[2] = a.bg[2];
        c.ambient = a.ambient;
        c.depth = a.depth;
        c.pixel = pw;
        c.slot = 0;
    }
    return c;
}

// What shading one ray decides (the closest-hit or miss shader's part that
// does not depend on where its spawned rays go).
struct ShadeEval {
    RayCtx c;
    Surf s;
    float3 thr, alb;
    float ior;
    uint32_t type, n_next;
    bool lit;  // a diffuse hit: ambient term and shadow rays
    bool hit;
};

__device__ __forceinline__ ShadeEval shade_none() {
    ShadeEval e;
    e.c = RayCtx{};
    e.thr = e.alb = f3(0.f, 0.f, 0.f);
    e.ior = 1.0f;
    e.type = 0;
    e.n_next = 0;
    e.lit = false;
    e.hit = false;
    return e;
}

// The ray (r0 = origin, tmin; r1 = direction, tmax), its payload and its hit:
// the miss colour or the ambient term into the image, alpha for camera hits,
// the surface, its material and how many path rays it spawns.
template <bool BATCH>
__device__ __forceinline__ ShadeEval shade_eval(const ShadeArgs& a, float4 r0, float4 r1, const Payload& pl,
                                                const HitDev& hd) {
    ShadeEval e = shade_none();
    e.c = ray_ctx<BATCH>(a, a.slots, pl.pixel);
    const RayCtx& c = e.c;
    Surf& s = e.s;
    const float3 thr = f3(pl.r, pl.g, pl.b);
    e.thr = thr;
    float* px = c.image + 4 * (size_t)c.pixel;
    if (hd.inst_leaf == kMiss) {
        atomicAdd(px + 0, thr.x * c.bg[0]);
        atomicAdd(px + 1, thr.y * c.bg[1]);
        atomicAdd(px + 2, thr.z * c.bg[2]);
        return e;
    }
    e.hit = true;
    if (c.depth == 1) px[3] = 1.0f;
    const InstDev* I = c.inst + hd.inst_leaf;
    const float4 i0 = I->inv[0], i1 = I->inv[1], i2 = I->inv[2];
    const float4* tp = I->tris + kTriStride * (size_t)hd.tri_leaf;  // the (x, y, z) order
    const float4 v0 = tp[0], v1 = tp[1], v2 = tp[2];
    float3 e1 = f3(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z);
    float3 e2 = f3(v2.x - v0.x, v2.y - v0.y, v2.z - v0.z);
    float3 no = cross3(e1, e2);
    float3 nw = f3(i0.x * no.x + i1.x * no.y + i2.x * no.z, i0.y * no.x + i1.y * no.y + i2.y * no.z,
                   i0.z * no.x + i1.z * no.y + i2.z * no.z);
    nw = normalize3(nw);
    s.d = f3(r1.x, r1.y, r1.z);
    s.p = f3(fmaf(hd.t, r1.x, r0.x), fmaf(hd.t, r1.y, r0.y), fmaf(hd.t, r1.z, r0.z));
    s.entering = dot3(s.d, nw) < 0.0f;
    s.nf = s.entering ? nw : -1.0f * nw;
    s.eps = 1e-4f * fmaxf(1.0f, fmaxf(fabsf(s.p.x), fmaxf(fabsf(s.p.y), fabsf(s.p.z))));
    uint32_t mi = I->material;
    if (mi >= c.n_mats) {
        record_error(a.st, RG_ERR_INVALID_ARG);
        mi = 0;
    }
    const rg_material M = c.mats[mi];
    e.type = M.type;
    e.alb = f3(M.albedo[0], M.albedo[1], M.albedo[2]);
    e.ior = M.ior;
    const float3 alb = e.alb;
    if (e.type == RG_MAT_DIFFUSE) {
        atomicAdd(px + 0, thr.x * alb.x * c.ambient);
        atomicAdd(px + 1, thr.y * alb.y * c.ambient);
        atomicAdd(px + 2, thr.z * alb.z * c.ambient);
        e.lit = true;
    } else if (c.depth < c.max_depth) {
        e.n_next = 1;
        if (e.type == RG_MAT_GLASS) {
            float eta = s.entering ? 1.0f / e.ior : e.ior;
            float ci = -dot3(s.d, s.nf);
            float k = 1.0f - eta * eta * (1.0f - ci * ci);
            if (k >= 0.0f) e.n_next = 2;
        }
    }
    return e;
}

// Origin of the shadow rays of a lit surface point.
__device__ __forceinline__ float3 shadow_origin(const ShadeEval& e) {
    return e.lit ? e.s.p + e.s.eps * e.s.nf : f3(0.f, 0.f, 0.f);
}

// Whether the lit surface point faces light l (lv: from the shadow origin os
// toward the light).
__device__ __forceinline__ bool faces_light(const ShadeEval& e, float3 os, uint32_t l, rg_light* L, float3* lv) {
    if (!e.lit || l >= e.c.n_lights) return false;
    *L = e.c.lights[l];
    *lv = f3(L->pos[0], L->pos[1], L->pos[2]) - os;
    return dot3(e.s.nf, *lv) > 0.0f;
}

// The shadow ray toward a faced light: r0 = (os, 0), r1 = (direction, distance
// - eps), and the Lambert contribution it adds if nothing occludes it
// (ta = throughput * albedo).
__device__ __forceinline__ void shadow_ray(float3 os, float3 nf, float eps, float3 ta, const rg_light& L, float3 lv,
                                           float4* r0, float4* r1, float3* contrib) {
    const float dist = sqrtf(dot3(lv, lv));
    const float3 ld = (1.0f / dist) * lv;
    const float cl = dot3(nf, ld);
    *r0 = make_float4(os.x, os.y, os.z, 0.0f);
    *r1 = make_float4(ld.x, ld.y, ld.z, dist - eps);
    *contrib = f3(ta.x * L.intensity[0] * cl, ta.y * L.intensity[1] * cl, ta.z * L.intensity[2] * cl);
}

// The reflected (and, for glass, refracted) rays of a hit, at queue positions
// nbase (and nbase + 1), ring-mapped from next_base in the batched mode.
template <bool BATCH>
__device__ __forceinline__ void write_path_rays(const ShadeArgs& a, const ShadeEval& e, uint32_t next_base,
                                                uint32_t nbase) {
    const Surf& s = e.s;
    const float3 thr = e.thr, alb = e.alb;
    const float ior = e.ior;
    const uint32_t next_pw = BATCH ? pack_pixel(e.c.pixel, e.c.depth + 1, e.c.slot) : e.c.pixel;
    float dn = dot3(s.d, s.nf);
    float3 r = normalize3(s.d - (2.0f * dn) * s.nf);
    float3 ro = s.p + s.eps * s.nf;
    float3 w_r = thr;
    if (e.type == RG_MAT_MIRROR) {
        w_r = f3(thr.x * alb.x, thr.y * alb.y, thr.z * alb.z);
    } else if (e.n_next == 2) {
        float eta = s.entering ? 1.0f / ior : ior;
        float ci = -dn;
        float k = 1.0f - eta * eta * (1.0f - ci * ci);
        float sk = sqrtf(k);
        float3 T = normalize3(eta * s.d + (eta * ci - sk) * s.nf);
        float R0 = (1.0f - ior) / (1.0f + ior);
        R0 = R0 * R0;
        float cc = s.entering ? ci : sk;
        float m = 1.0f - cc;
        float R = R0 + (1.0f - R0) * (m * m * m * m * m);
        w_r = R * thr;
        float3 to = s.p - s.eps * s.nf;
        uint32_t slot = BATCH ? ((next_base + nbase + 1) & a.ring_mask) : nbase + 1;
        a.next_rays[2 * (size_t)slot] = make_float4(to.x, to.y, to.z, 0.0f);
        a.next_rays[2 * (size_t)slot + 1] = make_float4(T.x, T.y, T.z, __int_as_float(0x7F800000));
        Payload tp;
        tp.pixel = next_pw;
        tp.r = (1.0f - R) * thr.x;
        tp.g = (1.0f - R) * thr.y;
        tp.b = (1.0f - R) * thr.z;
        a.next_payload[slot] = tp;
    }
    const uint32_t rslot = BATCH ? ((next_base + nbase) & a.ring_mask) : nbase;
    a.next_rays[2 * (size_t)rslot] = make_float4(ro.x, ro.y, ro.z, 0.0f);
    a.next_rays[2 * (size_t)rslot + 1] = make_float4(r.x, r.y, r.z, __int_as_float(0x7F800000));
    Payload rp;
    rp.pixel = next_pw;
    rp.r = w_r.x;
    rp.g = w_r.y;
    rp.b = w_r.z;
    a.next_payload[rslot] = rp;
}

// Shade ray i into the queues (valid == false: take part in the block's queue
// claims only).  live_delta (batched only): per-slot sums of (path rays
// spawned - 1) of this block, in shared memory.
template <bool BATCH>
__device__ __forceinline__ void shade_one(const ShadeArgs& a, uint32_t head, uint32_t next_base, uint32_t i,
                                          bool valid, int* live_delta, ClaimSmem* cs) {
    ShadeEval e = shade_none();
    if (valid) {
        const uint32_t j = BATCH ? ((head + i) & a.ring_mask) : i;
        const float4 r0 = a.rays[2 * (size_t)j], r1 = a.rays[2 * (size_t)j + 1];
        e = shade_eval<BATCH>(a, r0, r1, a.payload[j], a.hits[i]);
    }
    // shadow rays: one sub-queue per light, so that a warp of shadow rays
    // holds neighbouring surface points seen toward the same light; every
    // thread of the block takes part in the claims
    const uint32_t shadow_pw = BATCH ? pack_pixel(e.c.pixel, e.c.depth, e.c.slot) : e.c.pixel;
    const float3 os = shadow_origin(e);
    const float3 ta = f3(e.thr.x * e.alb.x, e.thr.y * e.alb.y, e.thr.z * e.alb.z);
    const uint32_t n_loop = BATCH ? a.max_lights : a.n_lights;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    rg_light L;
    float3 lv = f3(0.f, 0.f, 0.f);
    for (uint32_t l = 0; l < n_loop; ++l) {
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, faces_light(e, os, l, &L, &lv));
        if (lane == 0 && b) cs->woff[warp][l] = atomicAdd(&cs->cnt[l], (uint32_t)__popc(b));
    }
    const uint32_t n_next = e.n_next;
    const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, n_next >= 1), b2 = __ballot_sync(0xFFFFFFFFu, n_next >= 2);
    if (lane == 0 && b1) cs->woff[warp][n_loop] = atomicAdd(&cs->cnt[n_loop], (uint32_t)(__popc(b1) + __popc(b2)));
    __syncthreads();
    for (uint32_t q = threadIdx.x; q <= n_loop; q += blockDim.x) {
        const uint32_t t = cs->cnt[q];
        cs->base[q] = t ? atomicAdd(q < n_loop ? a.shadow_count + q : a.next_count, t) : 0u;
        cs->cnt[q] = 0u;
    }
    __syncthreads();
    for (uint32_t l = 0; l < n_loop; ++l) {
        const bool want = faces_light(e, os, l, &L, &lv);
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, want);
        if (!want) continue;
        const uint32_t k = cs->base[l] + cs->woff[warp][l] + (uint32_t)__popc(b & lt);
        const size_t slot = (size_t)l * a.shadow_stride + k;
        float4 r0, r1;
        float3 col;
        shadow_ray(os, e.s.nf, e.s.eps, ta, L, lv, &r0, &r1, &col);
        a.shadow_rays[2 * slot] = r0;
        a.shadow_rays[2 * slot + 1] = r1;
        Payload sp;
        sp.pixel = shadow_pw;
        sp.r = col.x;
        sp.g = col.y;
        sp.b = col.z;
        a.shadow_payload[slot] = sp;
    }
    // path rays
    const uint32_t nbase =
        cs->base[n_loop] + cs->woff[warp][n_loop] + (uint32_t)(__popc(b1 & lt) + __popc(b2 & lt));
    // live path rays of the slot: this ray leaves, its spawns join
    if (BATCH && valid && n_next != 1) atomicAdd(live_delta + e.c.slot, (int)n_next - 1);
    if (valid && e.hit && n_next) write_path_rays<BATCH>(a, e, next_base, nbase);
}

// One depth level's rays: n_host of them, or *a.d_count when the count is
// only on the device; whole blocks step together through the queue so that
// every thread takes part in the block claims.
__global__ void __launch_bounds__(kShadeBlock) k_shade(ShadeArgs a, uint32_t n_host) {
    __shared__ ClaimSmem cs;
    claim_init(&cs);
    __syncthreads();
    const uint32_t n = a.d_count ? *a.d_count : n_host;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        shade_one<false>(a, 0u, 0u, i, i < n, nullptr, &cs);
    }
}

// Mixed queue: the count is read on the device; whole blocks step together so
// that every thread takes part in the block claims.
__global__ void __launch_bounds__(kShadeBlock) k_shade_batch(ShadeArgs a) {
    __shared__ int live_delta[kMaxSlots];
    __shared__ ClaimSmem cs;
    static_assert(kShadeBlock >= kMaxSlots, "one thread per slot flushes the block's sums");
    if (threadIdx.x < kMaxSlots) live_delta[threadIdx.x] = 0;
    claim_init(&cs);
    __syncthreads();
    const uint32_t n = *a.d_count;
    const uint32_t head = *a.ring_head, next_base = *a.next_base;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        shade_one<true>(a, head, next_base, i, i < n, live_delta, &cs);
    }
    __syncthreads();
    if (threadIdx.x < kMaxSlots && live_delta[threadIdx.x] != 0)
        atomicAdd(a.slot_live + threadIdx.x, live_delta[threadIdx.x]);
}

// Primary rays of the requests admitted in this step; ray r belongs to the
// request whose [offset, offset + w h) range holds it (offsets ascending).
__global__ void k_raygen_batch(const RaygenReq* __restrict__ reqs, const uint32_t* __restrict__ n_reqs_p,
                               const uint32_t* __restrict__ n_rays_p, const uint32_t* __restrict__ gen_base_p,
                               uint32_t ring_mask, float4* __restrict__ rays, Payload* __restrict__ payload) {
    __shared__ RaygenReq sr[kMaxSlots];
    const uint32_t n_reqs = min(*n_reqs_p, kMaxSlots);
    const uint32_t n_rays = *n_rays_p, gen_base = *gen_base_p;
    for (uint32_t k = threadIdx.x; k < n_reqs; k += blockDim.x) sr[k] = reqs[k];
    __syncthreads();
    if (n_reqs == 0) return;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rays; r += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = n_reqs - 1;  // last request with offset <= r
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (sr[mid].offset <= r) lo = mid; else hi = mid - 1;
        }
        const RaygenReq& q = sr[lo];
        const uint32_t i = r - q.offset;
        const uint32_t w = q.w, h = q.h;
        if (i >= w * h) continue;  // not a ray of any request (host offsets are dense)
        uint32_t x, y;
        tile_pixel(i, w, h, x, y);
        float4 o, d;
        camera_ray(q.cam, w, h, x, y, o, d);
        const uint32_t e = (gen_base + r) & ring_mask;
        rays[2 * (size_t)e] = o;
        rays[2 * (size_t)e + 1] = d;
        const uint32_t pix = y * w + x;
        Payload p;
        p.pixel = pack_pixel(pix, 1u, q.slot);
        p.r = p.g = p.b = 1.0f;
        payload[e] = p;
        reinterpret_cast<float4*>(q.image)[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ---------------------------------------------------------------- FXAA
// Fast approximate anti-aliasing (Lottes 2009) of an RGBA32F image, one
// thread per pixel, clamp-to-edge addressing, pixel centres at integer
// coordinates.  Every step is a float32 threshold decision; this file is
// compiled without FMA contraction so each operation rounds on its own.
//  1. luma = sqrt(max(0.299 R + 0.587 G + 0.114 B, 0));
//  2. pixels whose 5-point luma range is below max(0.0312, 0.125 max) are copied;
//  3. the edge is horizontal if the vertical second differences of the 3x3
//     block (weights 1, 2, 1) are at least the horizontal ones;
//  4. it lies toward the neighbour across it with the larger luma step; the
//     edge luma is the mean of that neighbour and the pixel;
//  5. half a pixel across, the search steps along the edge both ways (1, 1,
//     1, 1, 1, 1.5, 2, 2, 2, 2, 4, 8 pixels) until the bilinear luma leaves
//     the edge luma by a quarter of the larger step;
//  6. offset across the edge: 0.5 - (distance to the nearer end) / (edge
//     length) for a pixel whose luma change is opposite to the one at that
//     end, else 0; at least the sub-pixel offset 0.75 s^2, s the smoothstep
//     of the contrast of the 3x3 mean (neighbours weighted 2, corners 1);
//  7. output = bilinear colour at that offset; alpha kept.
// luma of one RGBA pixel (step 1)
__device__ __forceinline__ float fxaa_luma(float4 c) {
    const float v = 0.299f * c.x + 0.587f * c.y + 0.114f * c.z;
    return sqrtf(v > 0.0f ? v : 0.0f);
}

// The luma image, once per pixel: the main kernel reads 4 B lumas instead of
// recomputing them from 16 B pixels (an edge pixel looks up about a hundred).
__global__ void __launch_bounds__(256) k_fxaa_luma(const float4* __restrict__ in, uint32_t n, float* __restrict__ lum) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        lum[i] = fxaa_luma(__ldg(in + i));
}

struct FxaaImg {
    const float4* p;
    const float* lum;  // fxaa_luma of every pixel
    int w, h;
    __device__ __forceinline__ float4 at(int x, int y) const {
        x = min(max(x, 0), w - 1);
        y = min(max(y, 0), h - 1);
        return __ldg(p + (size_t)y * (size_t)w + (size_t)x);
    }
    __device__ __forceinline__ float luma(int x, int y) const {
        x = min(max(x, 0), w - 1);
        y = min(max(y, 0), h - 1);
        return __ldg(lum + (size_t)y * (size_t)w + (size_t)x);
    }
    __device__ __forceinline__ float luma_at(float px, float py) const {
        const float fx0 = floorf(px), fy0 = floorf(py);
        const float fx = px - fx0, fy = py - fy0;
        const int x0 = (int)fx0, y0 = (int)fy0;
        const float a = luma(x0, y0), b = luma(x0 + 1, y0), d = luma(x0, y0 + 1), e = luma(x0 + 1, y0 + 1);
        const float top = a + fx * (b - a), bot = d + fx * (e - d);
        return top + fy * (bot - top);
    }
    __device__ __forceinline__ float3 color_at(float px, float py) const {
        const float fx0 = floorf(px), fy0 = floorf(py);
        const float fx = px - fx0, fy = py - fy0;
        const int x0 = (int)fx0, y0 = (int)fy0;
        const float4 a = at(x0, y0), b = at(x0 + 1, y0), d = at(x0, y0 + 1), e = at(x0 + 1, y0 + 1);
        float3 r;
        float top = a.x + fx * (b.x - a.x), bot = d.x + fx * (e.x - d.x);
        r.x = top + fy * (bot - top);
        top = a.y + fx * (b.y - a.y);
        bot = d.y + fx * (e.y - d.y);
        r.y = top + fy * (bot - top);
        top = a.z + fx * (b.z - a.z);
        bot = d.z + fx * (e.z - d.z);
        r.z = top + fy * (bot - top);
        return r;
    }
};

__device__ __forceinline__ float second_diff(float a, float m, float b) { return fabsf((a + b) - 2.0f * m); }

__global__ void __launch_bounds__(256) k_fxaa(FxaaImg I, float4* __restrict__ out) {
    const int x = blockIdx.x * 16 + (threadIdx.x & 15), y = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (x >= I.w || y >= I.h) return;
    const float4 c = I.at(x, y);
    float4 o = c;
    const float lM = I.luma(x, y), lN = I.luma(x, y - 1), lS = I.luma(x, y + 1);
    const float lW = I.luma(x - 1, y), lE = I.luma(x + 1, y);
    const float lo = fminf(lM, fminf(fminf(lN, lS), fminf(lW, lE)));
    const float hi = fmaxf(lM, fmaxf(fmaxf(lN, lS), fmaxf(lW, lE)));
    const float range = hi - lo;
    if (!(range < fmaxf(0.0312f, hi * 0.125f))) {
        const float lNW = I.luma(x - 1, y - 1), lNE = I.luma(x + 1, y - 1);
        const float lSW = I.luma(x - 1, y + 1), lSE = I.luma(x + 1, y + 1);
        const float eH = (second_diff(lNW, lW, lSW) + 2.0f * second_diff(lN, lM, lS)) + second_diff(lNE, lE, lSE);
        const float eV = (second_diff(lNW, lN, lNE) + 2.0f * second_diff(lW, lM, lE)) + second_diff(lSW, lS, lSE);
        const bool horiz = eH >= eV;
        const float l1 = horiz ? lN : lW, l2 = horiz ? lS : lE;
        const float g1 = l1 - lM, g2 = l2 - lM;
        const bool neg = fabsf(g1) >= fabsf(g2);
        const float gs = 0.25f * fmaxf(fabsf(g1), fabsf(g2));
        const float edge = neg ? 0.5f * (l1 + lM) : 0.5f * (l2 + lM);
        const float sgn = neg ? -1.0f : 1.0f;
        const float fx = (float)x, fy = (float)y;
        const float sx = horiz ? fx : fx + 0.5f * sgn, sy = horiz ? fy + 0.5f * sgn : fy;
        constexpr float kStep[12] = {1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.5f, 2.0f, 2.0f, 2.0f, 2.0f, 4.0f, 8.0f};
        float dist[2], endl[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const float dir = side == 0 ? -1.0f : 1.0f;
            float d = 0.0f, e = 0.0f;
            for (int k = 0; k < 12; ++k) {
                d = d + kStep[k];
                const float px = horiz ? sx + dir * d : sx;
                const float py = horiz ? sy : sy + dir * d;
                e = I.luma_at(px, py) - edge;
                if (fabsf(e) >= gs) break;
            }
            dist[side] = d;
            endl[side] = e;
        }
        const float len = dist[0] + dist[1];
        const bool near0 = dist[0] < dist[1];
        const float dmin = near0 ? dist[0] : dist[1];
        const float e_near = near0 ? endl[0] : endl[1];
        const float off = ((lM < edge) != (e_near < 0.0f)) ? 0.5f - __fdiv_rn(dmin, len) : 0.0f;
        const float sum4 = (lN + lS) + (lW + lE);
        const float sumc = (lNW + lNE) + (lSW + lSE);
        const float avg = __fdiv_rn(2.0f * sum4 + sumc, 12.0f);
        float sp = __fdiv_rn(fabsf(avg - lM), range);
        if (sp > 1.0f) sp = 1.0f;
        sp = ((3.0f - 2.0f * sp) * sp) * sp;
        const float f = fmaxf(off, (sp * sp) * 0.75f);
        const float3 r = I.color_at(horiz ? fx : fx + f * sgn, horiz ? fy + f * sgn : fy);
        o.x = r.x;
        o.y = r.y;
        o.z = r.z;
    }
    out[(size_t)y * (size_t)I.w + (size_t)x] = o;
}

}  // namespace

cudaError_t launch_raygen(const CameraDev& cam, uint32_t w, uint32_t h, float4* rays, Payload* payload,
                          cudaStream_t s) {
    size_t n = (size_t)w * h;
    k_raygen<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cam, w, h, rays, payload);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_shade(const ShadeArgs& a, uint32_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    // n: the rays (a.d_count null) or a bound on them; blocks loop over the queue
    const uint32_t blocks = min((n + kShadeBlock - 1) / kShadeBlock, (uint32_t)device_sm_count() * 8u);
    k_shade<<<blocks, kShadeBlock, 0, s>>>(a, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_raygen_batch(const RaygenReq* reqs, const uint32_t* n_reqs, uint32_t max_rays,
                                const uint32_t* n_rays, const uint32_t* gen_base, uint32_t ring_mask, float4* rays,
                                Payload* payload, cudaStream_t s) {
    const uint32_t blocks = (uint32_t)min((max_rays + 255u) / 256u, (uint32_t)device_sm_count() * 8u);
    k_raygen_batch<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(reqs, n_reqs, n_rays, gen_base, ring_mask, rays, payload);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_shade_batch(const ShadeArgs& a, cudaStream_t s) {
    k_shade_batch<<<device_sm_count() * 8, kShadeBlock, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fxaa(const float4* in, uint32_t w, uint32_t h, float* lum, float4* out, cudaStream_t s) {
    if (w == 0 || h == 0) return cudaSuccess;
    const uint32_t n = w * h;
    k_fxaa_luma<<<min((n + 255u) / 256u, (uint32_t)device_sm_count() * 16u), 256, 0, s>>>(in, n, lum);
    FxaaImg I{in, lum, (int)w, (int)h};
    k_fxaa<<<dim3((w + 15) / 16, (h + 15) / 16), 256, 0, s>>>(I, out);
    count_launches(2);
    return cudaGetLastError();
}


}  // namespace rg
