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

constexpr int kShadeBlock = 256;

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) { return rsqrtf(dot3(a, a)) * a; }

__global__ void k_raygen(CameraDev cam, uint32_t w, uint32_t h, float4* __restrict__ rays,
                         Payload* __restrict__ payload) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w * h) return;
    uint32_t x = i % w, y = i / w;
    float3 eye = f3(cam.eye[0], cam.eye[1], cam.eye[2]);
    float3 F = normalize3(f3(cam.target[0], cam.target[1], cam.target[2]) - eye);
    float3 R = normalize3(cross3(F, f3(cam.up[0], cam.up[1], cam.up[2])));
    float3 U = cross3(R, F);
    float th = tanf(0.5f * cam.vfov_deg * 0.017453292519943295f);
    float aspect = (float)w / (float)h;
    float px = (2.0f * ((float)x + 0.5f) / (float)w - 1.0f) * aspect * th;
    float py = (1.0f - 2.0f * ((float)y + 0.5f) / (float)h) * th;
    float3 d = normalize3(px * R + py * U + F);
    rays[2 * (size_t)i] = make_float4(eye.x, eye.y, eye.z, 0.0f);
    rays[2 * (size_t)i + 1] = make_float4(d.x, d.y, d.z, __int_as_float(0x7F800000));
    Payload p;
    p.pixel = i;
    p.r = p.g = p.b = 1.0f;
    payload[i] = p;
}

// exclusive warp prefix of `c`; the warp total goes to one atomicAdd on *tail
// (and, if `counter` is given, to a 64-bit statistics counter)
__device__ __forceinline__ uint32_t warp_claim(uint32_t c, uint32_t* tail, unsigned long long* counter = nullptr) {
    const int lane = threadIdx.x & 31;
    uint32_t x = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
    uint32_t base = 0;
    if (lane == 31 && total) {
        base = atomicAdd(tail, total);
        if (counter) atomicAdd(counter, (unsigned long long)total);
    }
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + x - c;
}

struct Surf {
    float3 p, nf, d;
    float eps;
    bool entering;
};

__global__ void __launch_bounds__(kShadeBlock) k_shade(ShadeArgs a, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    uint32_t n_shadow = 0, n_next = 0;
    Surf s;
    uint32_t type = 0;
    float3 alb = f3(0, 0, 0), thr = f3(0, 0, 0);
    float ior = 1.0f;
    uint32_t pixel = 0;
    bool hit = false;
    if (valid) {
        const float4 r0 = a.rays[2 * (size_t)i], r1 = a.rays[2 * (size_t)i + 1];
        const Payload pl = a.payload[i];
        const HitDev hd = a.hits[i];
        pixel = pl.pixel;
        thr = f3(pl.r, pl.g, pl.b);
        float* px = a.image + 4 * (size_t)pixel;
        if (hd.inst_leaf == kMiss) {
            atomicAdd(px + 0, thr.x * a.bg[0]);
            atomicAdd(px + 1, thr.y * a.bg[1]);
            atomicAdd(px + 2, thr.z * a.bg[2]);
        } else {
            hit = true;
            if (a.depth == 1) px[3] = 1.0f;
            const InstDev* I = a.inst + hd.inst_leaf;
            const float4 i0 = I->inv[0], i1 = I->inv[1], i2 = I->inv[2];
            const float4* tp = I->tris + 3 * (size_t)hd.tri_leaf;
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
            if (mi >= a.n_mats) {
                record_error(a.st, RG_ERR_INVALID_ARG);
                mi = 0;
            }
            const rg_material M = a.mats[mi];
            type = M.type;
            alb = f3(M.albedo[0], M.albedo[1], M.albedo[2]);
            ior = M.ior;
            if (type == RG_MAT_DIFFUSE) {
                atomicAdd(px + 0, thr.x * alb.x * a.ambient);
                atomicAdd(px + 1, thr.y * alb.y * a.ambient);
                atomicAdd(px + 2, thr.z * alb.z * a.ambient);
                float3 os = s.p + s.eps * s.nf;
                for (uint32_t l = 0; l < a.n_lights; ++l) {
                    const rg_light L = a.lights[l];
                    float3 lv = f3(L.pos[0], L.pos[1], L.pos[2]) - os;
                    if (dot3(s.nf, lv) > 0.0f) ++n_shadow;
                }
            } else if (a.depth < a.max_depth) {
                n_next = 1;
                if (type == RG_MAT_GLASS) {
                    float eta = s.entering ? 1.0f / ior : ior;
                    float ci = -dot3(s.d, s.nf);
                    float k = 1.0f - eta * eta * (1.0f - ci * ci);
                    if (k >= 0.0f) n_next = 2;
                }
            }
        }
    }
    // claim queue slots (all lanes take part)
    uint32_t sbase = warp_claim(n_shadow, a.shadow_count, &a.st->shadow_rays);
    uint32_t nbase = warp_claim(n_next, a.next_count);
    if (!valid || !hit) return;
    if (n_shadow) {
        float3 os = s.p + s.eps * s.nf;
        uint32_t k = 0;
        for (uint32_t l = 0; l < a.n_lights; ++l) {
            const rg_light L = a.lights[l];
            float3 lv = f3(L.pos[0], L.pos[1], L.pos[2]) - os;
            if (!(dot3(s.nf, lv) > 0.0f)) continue;
            float dist = sqrtf(dot3(lv, lv));
            float3 ld = (1.0f / dist) * lv;
            float c = dot3(s.nf, ld);
            uint32_t slot = sbase + k++;
            a.shadow_rays[2 * (size_t)slot] = make_float4(os.x, os.y, os.z, 0.0f);
            a.shadow_rays[2 * (size_t)slot + 1] = make_float4(ld.x, ld.y, ld.z, dist - s.eps);
            Payload sp;
            sp.pixel = pixel;
            sp.r = thr.x * alb.x * L.intensity[0] * c;
            sp.g = thr.y * alb.y * L.intensity[1] * c;
            sp.b = thr.z * alb.z * L.intensity[2] * c;
            a.shadow_payload[slot] = sp;
        }
    }
    if (n_next) {
        float dn = dot3(s.d, s.nf);
        float3 r = normalize3(s.d - (2.0f * dn) * s.nf);
        float3 ro = s.p + s.eps * s.nf;
        float3 w_r = thr;
        if (type == RG_MAT_MIRROR) {
            w_r = f3(thr.x * alb.x, thr.y * alb.y, thr.z * alb.z);
        } else if (n_next == 2) {
            float eta = s.entering ? 1.0f / ior : ior;
            float ci = -dn;
            float k = 1.0f - eta * eta * (1.0f - ci * ci);
            float sk = sqrtf(k);
            float3 T = normalize3(eta * s.d + (eta * ci - sk) * s.nf);
            float R0 = (1.0f - ior) / (1.0f + ior);
            R0 = R0 * R0;
            float c = s.entering ? ci : sk;
            float m = 1.0f - c;
            float R = R0 + (1.0f - R0) * (m * m * m * m * m);
            w_r = R * thr;
            float3 to = s.p - s.eps * s.nf;
            uint32_t slot = nbase + 1;
            a.next_rays[2 * (size_t)slot] = make_float4(to.x, to.y, to.z, 0.0f);
            a.next_rays[2 * (size_t)slot + 1] = make_float4(T.x, T.y, T.z, __int_as_float(0x7F800000));
            Payload tp;
            tp.pixel = pixel;
            tp.r = (1.0f - R) * thr.x;
            tp.g = (1.0f - R) * thr.y;
            tp.b = (1.0f - R) * thr.z;
            a.next_payload[slot] = tp;
        }
        a.next_rays[2 * (size_t)nbase] = make_float4(ro.x, ro.y, ro.z, 0.0f);
        a.next_rays[2 * (size_t)nbase + 1] = make_float4(r.x, r.y, r.z, __int_as_float(0x7F800000));
        Payload rp;
        rp.pixel = pixel;
        rp.r = w_r.x;
        rp.g = w_r.y;
        rp.b = w_r.z;
        a.next_payload[nbase] = rp;
    }
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
    k_shade<<<(n + kShadeBlock - 1) / kShadeBlock, kShadeBlock, 0, s>>>(a, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace rg
