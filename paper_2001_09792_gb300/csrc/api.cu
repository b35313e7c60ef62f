// The extern "C" boundary of librg: argument checks, ownership of the
// acceleration structures and ray queues, and the launch sequences of the
// build, trace and render calls.  See include/rg.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "rg_internal.cuh"

using namespace rg;

namespace {

thread_local std::string g_last_error;

rg_status fail(rg_status code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

rg_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky launch error
    return fail(e == cudaErrorMemoryAllocation ? RG_ERR_OOM : RG_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define RG_CK(call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

// Host-side fault injection for tests: RG_FAULT=alloc:N fails the N-th
// device allocation (1-based) made by the library with RG_ERR_OOM.
long g_alloc_count = 0;
long fault_alloc_index() {
    static long idx = -2;
    if (idx == -2) {
        idx = -1;
        const char* f = std::getenv("RG_FAULT");
        if (f && std::strncmp(f, "alloc:", 6) == 0) idx = std::atol(f + 6);
    }
    return idx;
}

// Test limits for the failure paths (no GPU fault is involved): a smaller
// traversal stack (RG_TEST_STACK=n) or iteration cap (RG_TEST_ITER_CAP=n) for
// every traversal the library launches; 0 when unset.
uint32_t test_limit(const char* name) {
    const char* v = std::getenv(name);
    if (!v) return 0;
    const long x = std::atol(v);
    return x > 0 && x < (1l << 30) ? (uint32_t)x : 0u;
}

rg_status dev_alloc(void** p, size_t bytes, const char* what) {
    *p = nullptr;
    long k = ++g_alloc_count;
    if (fault_alloc_index() == k) return fail(RG_ERR_OOM, std::string("injected allocation failure: ") + what);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, what);
    }
    return RG_OK;
}

struct TempAlloc {
    // stream-ordered temporaries, freed on the stream when the call ends
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit TempAlloc(cudaStream_t st) : s(st) {}
    ~TempAlloc() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    rg_status get(void** p, size_t bytes, const char* what) {
        *p = nullptr;
        long k = ++g_alloc_count;
        if (fault_alloc_index() == k) return fail(RG_ERR_OOM, std::string("injected allocation failure: ") + what);
        cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
        if (e != cudaSuccess) {
            *p = nullptr;
            return cuda_fail(e, what);
        }
        ptrs.push_back(*p);
        return RG_OK;
    }
};

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;  // elements
    rg_status ensure(size_t n, const char* what) {
        if (n <= cap && p) return RG_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = n < 16 ? 16 : n;
        rg_status st = dev_alloc(reinterpret_cast<void**>(&p), want * sizeof(T), what);
        if (st == RG_OK) cap = want;
        return st;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

struct BlasHost {
    float4* nodes = nullptr;
    float4* tris = nullptr;
    uint32_t nt = 0;
    uint32_t root = 0;
    uint32_t* leaf_of_prim = nullptr;  // BLAS leaf of each triangle index
    // compressed 8-wide form (null if not built)
    float4* nodes8 = nullptr;
    float4* tris8 = nullptr;
    uint32_t* src8 = nullptr;
    uint32_t* item_src8 = nullptr;
    uint32_t* counts8 = nullptr;
};

void free_blas(BlasHost& b) {
    cudaFree(b.nodes);
    cudaFree(b.tris);
    if (b.leaf_of_prim) cudaFree(b.leaf_of_prim);
    if (b.nodes8) cudaFree(b.nodes8);
    if (b.tris8) cudaFree(b.tris8);
    if (b.src8) cudaFree(b.src8);
    if (b.item_src8) cudaFree(b.item_src8);
    if (b.counts8) cudaFree(b.counts8);
    b = BlasHost();
}

// The last depth level's shadow rays, when at most kShadowSplitMax, are traced
// as kShadowSplit segments each (the launch is then short of rays, and its
// longest rays set its time).
constexpr uint32_t kShadowSplit = 8, kShadowSplitMax = 32768;
// Queue bytes a render may take for its worst case to run without waiting
// for the host (1080p at depth 4 with 4 lights takes 4.6 GB).
constexpr uint64_t kAsyncQueueBudget = 16ull << 30;

// The BLAS of one or more scenes; freed with the last scene that holds it
// (its destructor runs on that scene's device).
struct BlasSet {
    std::vector<BlasHost> blas;
    DevBuf<BlasDev> d_blas;
    uint32_t max_nt = 0;
    ~BlasSet() {
        for (BlasHost& b : blas) free_blas(b);
        d_blas.release();
    }
};

struct EventPair {
    cudaEvent_t a, b;
    int kind;  // 0 closest, 1 any, 2 shadow + closest pair
};

}  // namespace

// rg_trace_rays calls that may be in flight at once (each takes a work
// counter of its own, in turn)
constexpr uint32_t kTraceSlots = 64;

struct rg_scene {
    int device = 0;
    rg_scene_desc desc{};
    DevStatus* st = nullptr;
    // BLAS (shared with the scenes made by rg_scene_create_shared)
    std::shared_ptr<BlasSet> B = std::make_shared<BlasSet>();
    // TLAS
    bool tlas_built = false;
    uint32_t n_inst = 0;
    uint32_t tlas_root = 0;
    DevBuf<float4> tlas_nodes;
    DevBuf<InstDev> inst, inst_tmp;
    DevBuf<float> wbox;
    DevBuf<uint32_t> perm, parents, flags;
    DevBuf<uint32_t> leaf_of_inst;  // TLAS leaf of each instance index (made on first need after a build)
    bool leaf_of_inst_valid = false;
    // compressed 8-wide TLAS
    bool wide = false;
    DevBuf<float4> tlas8;
    DevBuf<InstDev> inst8;
    DevBuf<uint32_t> src8, item_src8, counts8;
    DevBuf<uint2> tasks8;
    // shading
    DevBuf<rg_material> mats;
    uint32_t n_mats = 0;
    DevBuf<rg_light> lights;
    uint32_t n_lights = 0;
    // queues
    DevBuf<float4> q_rays[2], s_rays;
    DevBuf<Payload> q_pay[2], s_pay;
    DevBuf<HitDev> hits;
    DevBuf<uint32_t> seg_count;    // per shadow ray of a split launch: segments finished / occluded (kept zero)
    DevBuf<uint32_t> counters;     // [0] closest work, [1] next count, [2] shadow work, [3] unused,
                                   // [4 + l] shadow rays toward light l
    DevBuf<uint32_t> trace_ctr;    // rg_trace_rays work counters: kTraceSlots slots, 128 B apart
    uint32_t trace_slot = 0;       // the next call's slot
    uint32_t* h_counts = nullptr;  // pinned, 16 entries
    cudaEvent_t count_ev = nullptr;  // the next level's ray count has reached h_counts
    // statistics and timing
    uint64_t closest_rays = 0, shadow_rays_host = 0;
    std::vector<EventPair> events, free_events;
    double trace_ms = 0, any_ms = 0, pair_ms = 0, refine_ms = 0;
    uint64_t trace_launches = 0, any_launches = 0, pair_launches = 0, refine_launches = 0;
    unsigned long long launch_base = 0;
};

namespace {

rg_status check_scene(rg_scene* s) {
    if (!s) return fail(RG_ERR_INVALID_ARG, "scene is NULL");
    return RG_OK;
}

rg_status set_device(rg_scene* s) {
    int cur = -1;
    RG_CK(cudaGetDevice(&cur));
    if (cur != s->device) RG_CK(cudaSetDevice(s->device));
    return RG_OK;
}

rg_status event_begin(rg_scene* s, int kind, cudaStream_t st, EventPair** out) {
    *out = nullptr;
    if (!(s->desc.flags & RG_SCENE_TIMING)) return RG_OK;
    EventPair ep;
    if (!s->free_events.empty()) {
        ep = s->free_events.back();
        s->free_events.pop_back();
    } else {
        RG_CK(cudaEventCreate(&ep.a));
        RG_CK(cudaEventCreate(&ep.b));
    }
    ep.kind = kind;
    RG_CK(cudaEventRecord(ep.a, st));
    s->events.push_back(ep);
    *out = &s->events.back();
    return RG_OK;
}

rg_status event_end(rg_scene* s, cudaStream_t st) {
    if (!(s->desc.flags & RG_SCENE_TIMING) || s->events.empty()) return RG_OK;
    RG_CK(cudaEventRecord(s->events.back().b, st));
    return RG_OK;
}

rg_status collect_events(rg_scene* s) {
    for (EventPair& ep : s->events) {
        RG_CK(cudaEventSynchronize(ep.b));
        float ms = 0;
        RG_CK(cudaEventElapsedTime(&ms, ep.a, ep.b));
        if (ep.kind == 0) {
            s->trace_ms += ms;
            s->trace_launches++;
        } else if (ep.kind == 1) {
            s->any_ms += ms;
            s->any_launches++;
        } else if (ep.kind == 3) {
            s->refine_ms += ms;
            s->refine_launches++;
        } else {
            s->pair_ms += ms;
            s->pair_launches++;
        }
        s->free_events.push_back(ep);
    }
    s->events.clear();
    return RG_OK;
}

uint32_t iter_cap_for(const rg_scene* s, bool brute) {
    // brute force: every node and triangle of every instance once, with pops;
    // a BVH traversal visits a tiny fraction of that, and 2^22 steps per ray
    // bound it far above any valid traversal of the supported scene sizes
    uint64_t per_inst = 4ull * (uint64_t)s->B->max_nt + 16;
    uint64_t cap = 4ull * (uint64_t)s->n_inst + (uint64_t)s->n_inst * per_inst + 64;
    if (!brute && cap > (1ull << 22)) cap = 1ull << 22;
    static const uint32_t test_cap = test_limit("RG_TEST_ITER_CAP");
    if (test_cap) cap = test_cap;
    return cap > 0xFFFFFFF0ull ? 0xFFFFFFF0u : (uint32_t)cap;
}

TraceArgs base_trace_args(rg_scene* s, bool wide) {
    TraceArgs a{};
    a.tlas_nodes = s->tlas_nodes.p;
    a.tlas_root = s->tlas_root;
    a.inst = s->inst.p;
    a.n_inst = s->n_inst;
    a.st = s->st;
    a.iter_cap = iter_cap_for(s, false);
    static const uint32_t test_stack = test_limit("RG_TEST_STACK");
    a.stack_max = test_stack;
    if (wide && s->wide) {
        a.tlas_nodes8 = s->tlas8.p;
        a.inst8 = s->inst8.p;
    }
    return a;
}

// Shared LBVH steps: lohi + centroid bounds already computed into cb_ord.
// Sorts the Morton codes of `lohi` and emits the topology into `nodes`.
rg_status lbvh_topology(TempAlloc& tmp, const float* lohi, uint32_t n, const int* cb_ord, int bits, float4* nodes,
                        uint32_t* perm, uint32_t* parents, cudaStream_t s, uint32_t* ranges = nullptr) {
    const int key_bits = bits == 21 ? 64 : 32;
    const size_t kb = key_bits / 8;
    void *codes, *sorted, *vals, *scratch;
    rg_status r;
    if ((r = tmp.get(&codes, n * kb, "morton codes"))) return r;
    if ((r = tmp.get(&sorted, n * kb, "sorted codes"))) return r;
    if ((r = tmp.get(&vals, n * 4ull, "sort values"))) return r;
    if ((r = tmp.get(&scratch, radix_sort_scratch_bytes(n, key_bits), "sort scratch"))) return r;
    RG_CK(launch_morton(lohi, n, cb_ord, bits, codes, static_cast<uint32_t*>(vals), nullptr, s));
    RG_CK(radix_sort_pairs(codes, static_cast<uint32_t*>(vals), n, key_bits, sorted, perm, scratch, s));
    RG_CK(launch_karras(sorted, n, key_bits, reinterpret_cast<uint32_t*>(nodes) + 12, 16, parents, s, ranges));
    return RG_OK;
}

// The call's stream-ordered temporaries, for builders outside this file.
rg_status temp_get(void* ctx, void** p, size_t bytes, const char* what) {
    return static_cast<TempAlloc*>(ctx)->get(p, bytes, what);
}

}  // namespace

extern "C" {

const char* rg_last_error(void) { return g_last_error.c_str(); }

rg_status rg_scene_create(rg_scene** out, const rg_scene_desc* desc) {
    if (!out) return fail(RG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    rg_scene* s = new rg_scene();
    RG_CK(cudaGetDevice(&s->device));
    if (desc) {
        s->desc = *desc;
    } else {
        s->desc.background[0] = 0.2f;
        s->desc.background[1] = 0.3f;
        s->desc.background[2] = 0.5f;
        s->desc.ambient = 0.1f;
        s->desc.flags = 0;
    }
    rg_status r = dev_alloc(reinterpret_cast<void**>(&s->st), sizeof(DevStatus), "status");
    if (r) {
        delete s;
        return r;
    }
    if ((r = s->counters.ensure(4 + kMaxLights, "counters")) ||
        (r = s->trace_ctr.ensure((size_t)kTraceSlots * 32, "trace counters"))) {
        cudaFree(s->st);
        s->counters.release();
        delete s;
        return r;
    }
    cudaError_t e = cudaMemset(s->st, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s->h_counts), 16 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->count_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaFree(s->st);
        s->counters.release();
        s->trace_ctr.release();
        delete s;
        return cuda_fail(e, "scene setup");
    }
    *out = s;
    return RG_OK;
}

rg_status rg_scene_create_shared(rg_scene** out, rg_scene* src) {
    if (!out) return fail(RG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    rg_status r;
    if ((r = check_scene(src))) return r;
    if ((r = set_device(src))) return r;
    rg_scene* s = nullptr;
    if ((r = rg_scene_create(&s, &src->desc))) return r;
    s->B = src->B;
    // materials and lights as the source has them now
    if (src->n_mats) {
        if ((r = s->mats.ensure(src->n_mats, "materials"))) {
            rg_scene_destroy(s);
            return r;
        }
        cudaError_t e = cudaMemcpy(s->mats.p, src->mats.p, src->n_mats * sizeof(rg_material), cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            rg_scene_destroy(s);
            return cuda_fail(e, "copying materials");
        }
        s->n_mats = src->n_mats;
    }
    if ((r = s->lights.ensure(src->n_lights ? src->n_lights : 1, "lights"))) {
        rg_scene_destroy(s);
        return r;
    }
    if (src->n_lights) {
        cudaError_t e = cudaMemcpy(s->lights.p, src->lights.p, src->n_lights * sizeof(rg_light), cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            rg_scene_destroy(s);
            return cuda_fail(e, "copying lights");
        }
    }
    s->n_lights = src->n_lights;
    *out = s;
    return RG_OK;
}

rg_status rg_scene_destroy(rg_scene* s) {
    if (!s) return RG_OK;
    set_device(s);
    cudaDeviceSynchronize();
    s->tlas8.release();
    s->inst8.release();
    s->src8.release();
    s->item_src8.release();
    s->counts8.release();
    s->tasks8.release();
    s->tlas_nodes.release();
    s->inst.release();
    s->leaf_of_inst.release();
    s->inst_tmp.release();
    s->wbox.release();
    s->perm.release();
    s->parents.release();
    s->flags.release();
    s->mats.release();
    s->lights.release();
    for (int k = 0; k < 2; ++k) {
        s->q_rays[k].release();
        s->q_pay[k].release();
    }
    s->s_rays.release();
    s->s_pay.release();
    s->hits.release();
    s->seg_count.release();
    s->counters.release();
    s->trace_ctr.release();
    if (s->st) cudaFree(s->st);
    if (s->h_counts) cudaFreeHost(s->h_counts);
    if (s->count_ev) cudaEventDestroy(s->count_ev);
    for (EventPair& ep : s->events) {
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    for (EventPair& ep : s->free_events) {
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    delete s;
    return RG_OK;
}

rg_status rg_blas_build(rg_scene* s, const float* d_vtx, uint32_t nv, const uint32_t* d_idx, uint32_t nt,
                        uint32_t flags, uint32_t* blas_id, void* stream) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (s->B.use_count() > 1) return fail(RG_ERR_INVALID_ARG, "the scene's BLAS are shared with another scene");
    if (!d_vtx || !d_idx || !blas_id) return fail(RG_ERR_INVALID_ARG, "NULL geometry or id pointer");
    if (nt == 0 || nv == 0) return fail(RG_ERR_INVALID_ARG, "empty mesh");
    if (flags & ~(RG_MORTON63 | RG_COMPRESSED | RG_WIDE_LEAF(3) | RG_BLAS_SAH))
        return fail(RG_ERR_INVALID_ARG, "unknown BLAS flags");
    const uint32_t leaf_max = ((flags >> 8) & 3u) ? ((flags >> 8) & 3u) : 2u;
    if (nt > (1u << 30)) return fail(RG_ERR_INVALID_ARG, "too many triangles");
    if ((r = set_device(s))) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int bits = (flags & RG_MORTON63) ? 21 : 10;
    const bool wide = (flags & RG_COMPRESSED) || (s->desc.flags & RG_SCENE_COMPRESSED);
    const size_t n_int = nt > 1 ? nt - 1 : 1;

    BlasHost b;
    b.nt = nt;
    b.root = nt == 1 ? kLeaf : 0u;
    if ((r = dev_alloc(reinterpret_cast<void**>(&b.nodes), n_int * 64, "BLAS nodes"))) return r;
    if ((r = dev_alloc(reinterpret_cast<void**>(&b.tris), (size_t)nt * kTriRecord, "BLAS triangles")) ||
        (r = dev_alloc(reinterpret_cast<void**>(&b.leaf_of_prim), (size_t)nt * 4, "BLAS leaf map"))) {
        free_blas(b);
        return r;
    }
    if (wide) {
        if ((r = dev_alloc(reinterpret_cast<void**>(&b.nodes8), n_int * 80, "wide BLAS nodes")) ||
            (r = dev_alloc(reinterpret_cast<void**>(&b.tris8), (size_t)nt * kTriRecord, "wide BLAS triangles")) ||
            (r = dev_alloc(reinterpret_cast<void**>(&b.src8), n_int * 32, "wide BLAS slot sources")) ||
            (r = dev_alloc(reinterpret_cast<void**>(&b.item_src8), (size_t)nt * 4, "wide BLAS item sources")) ||
            (r = dev_alloc(reinterpret_cast<void**>(&b.counts8), 16, "wide BLAS counts"))) {
            free_blas(b);
            return r;
        }
    }
    uint32_t id = (uint32_t)s->B->blas.size();
    if ((r = [&]() -> rg_status {
             // grow the descriptor array, keeping the old entries
             if (id + 1 > s->B->d_blas.cap) {
                 size_t ncap = (id + 1) * 2;
                 BlasDev* np = nullptr;
                 rg_status rr = dev_alloc(reinterpret_cast<void**>(&np), ncap * sizeof(BlasDev), "BLAS table");
                 if (rr) return rr;
                 if (s->B->d_blas.p && id) RG_CK(cudaMemcpyAsync(np, s->B->d_blas.p, id * sizeof(BlasDev), cudaMemcpyDeviceToDevice, st));
                 if (s->B->d_blas.p) {
                     RG_CK(cudaStreamSynchronize(st));
                     cudaFree(s->B->d_blas.p);
                 }
                 s->B->d_blas.p = np;
                 s->B->d_blas.cap = ncap;
             }
             BlasDev hd{};
             hd.nodes = b.nodes;
             hd.tris = b.tris;
             hd.root = b.root;
             hd.nt = nt;
             hd.nodes8 = b.nodes8;
             hd.tris8 = b.tris8;
             hd.leaf_of_prim = b.leaf_of_prim;
             RG_CK(cudaMemcpyAsync(s->B->d_blas.p + id, &hd, sizeof hd, cudaMemcpyHostToDevice, st));
             RG_CK(cudaStreamSynchronize(st));  // hd lives on this stack frame

             TempAlloc tmp(st);
             void *lohi, *cb, *perm, *parents, *fl, *ranges = nullptr, *tasks = nullptr;
             rg_status q;
             if (wide) {
                 if ((q = tmp.get(&ranges, n_int * 8, "ranges"))) return q;
                 if ((q = tmp.get(&tasks, (size_t)nt * 16, "collapse tasks"))) return q;
             }
             if ((q = tmp.get(&lohi, (size_t)nt * 24, "triangle boxes"))) return q;
             if ((q = tmp.get(&cb, 64, "centroid bounds"))) return q;
             if ((q = tmp.get(&perm, (size_t)nt * 4, "permutation"))) return q;
             if ((q = tmp.get(&parents, (size_t)(2 * (size_t)nt - 1) * 4, "parents"))) return q;
             if ((q = tmp.get(&fl, (size_t)(nt > 1 ? nt - 1 : 1) * 4, "refit flags"))) return q;
             RG_CK(launch_init_bounds(static_cast<int*>(cb), st));
             RG_CK(launch_tri_bounds(d_vtx, nv, d_idx, nt, static_cast<float*>(lohi), static_cast<int*>(cb), s->st, st));
             if (nt > 1) {
                 if (flags & RG_BLAS_SAH)
                     q = sah_topology(ScratchAlloc{temp_get, &tmp}, static_cast<float*>(lohi), nt,
                                      static_cast<int*>(cb), bits, b.nodes, static_cast<uint32_t*>(perm),
                                      static_cast<uint32_t*>(parents), st, static_cast<uint32_t*>(ranges));
                 else
                     q = lbvh_topology(tmp, static_cast<float*>(lohi), nt, static_cast<int*>(cb), bits, b.nodes,
                                       static_cast<uint32_t*>(perm), static_cast<uint32_t*>(parents), st,
                                       static_cast<uint32_t*>(ranges));
                 if (q) return q;
                 RG_CK(cudaMemsetAsync(fl, 0, (size_t)(nt - 1) * 4, st));
             } else {
                 RG_CK(cudaMemsetAsync(perm, 0, 4, st));
             }
             RG_CK(launch_blas_leaves_refit(d_vtx, d_idx, static_cast<uint32_t*>(perm), static_cast<float*>(lohi), nt,
                                            static_cast<uint32_t*>(parents), b.nodes, static_cast<uint32_t*>(fl), b.tris,
                                            s->B->d_blas.p + id, s->st, st));
             RG_CK(launch_bound_sphere(d_vtx, nv, s->B->d_blas.p + id, st));
             RG_CK(launch_invert_perm(static_cast<uint32_t*>(perm), nt, b.leaf_of_prim, st));
             if (wide) {
                 WideOut out{b.nodes8, b.src8, b.item_src8, b.counts8, static_cast<uint2*>(tasks)};
                 const float* leaf_box = reinterpret_cast<const float*>(reinterpret_cast<const char*>(s->B->d_blas.p + id) +
                                                                        offsetof(BlasDev, lo));
                 RG_CK(launch_collapse(b.nodes, static_cast<uint32_t*>(ranges), nt, leaf_box, b.tris, b.tris8, nullptr,
                                       nullptr, s->B->d_blas.p, out, s->st, st, leaf_max));
             }
             return RG_OK;
         }())) {
        cudaStreamSynchronize(st);
        free_blas(b);
        return r;
    }
    s->B->blas.push_back(b);
    if (nt > s->B->max_nt) s->B->max_nt = nt;
    *blas_id = id;
    return RG_OK;
}

static rg_status tlas_common(rg_scene* s, const rg_instance* d_inst, uint32_t n, cudaStream_t st, bool refit) {
    rg_status r;
    TempAlloc tmp(st);
    // the SAH hierarchy (one block) when asked for, else the LBVH; a one-launch
    // build or refit of a small TLAS when its topology is the LBVH's or fixed
    const bool sah = (s->desc.flags & RG_SCENE_SAH_TLAS) && n >= 2 && n <= kSahOneMax;
    if (n <= kTlasSmallMax && !(sah && !refit)) {
        // one single-block launch for the whole build or refit
        void* ranges = nullptr;
        if (!refit && s->wide && n > 1 && (r = tmp.get(&ranges, (size_t)(n - 1) * 8, "ranges"))) return r;
        RG_CK(launch_tlas_small(d_inst, n, s->B->d_blas.p, (uint32_t)s->B->blas.size(), s->inst_tmp.p, s->wbox.p, refit,
                                s->tlas_nodes.p, s->perm.p, s->parents.p, s->flags.p, static_cast<uint32_t*>(ranges),
                                s->inst.p, s->st, st));
        if (s->wide) {
            WideOut out{s->tlas8.p, s->src8.p, s->item_src8.p, s->counts8.p, s->tasks8.p};
            if (refit)
                RG_CK(launch_wide_refit(s->tlas_nodes.p, s->wbox.p, s->perm.p, n, s->inst.p, s->inst8.p, s->B->d_blas.p,
                                        out, s->st, st));
            else
                RG_CK(launch_collapse(s->tlas_nodes.p, static_cast<uint32_t*>(ranges), n, s->wbox.p, nullptr, nullptr,
                                      s->inst.p, s->inst8.p, s->B->d_blas.p, out, s->st, st, 1u));
        }
        return RG_OK;
    }
    void* cb;
    if ((r = tmp.get(&cb, 64, "centroid bounds"))) return r;
    if (!refit) RG_CK(launch_init_bounds(static_cast<int*>(cb), st));
    RG_CK(launch_instance_prep(d_inst, n, s->B->d_blas.p, (uint32_t)s->B->blas.size(), s->inst_tmp.p, s->wbox.p,
                               refit ? nullptr : static_cast<int*>(cb), refit, s->st, st));
    void* ranges = nullptr;
    void* boxes_done = nullptr;  // set by the SAH build when it wrote every node's boxes
    if (!refit) {
        if (n > 1) {
            if (s->wide && (r = tmp.get(&ranges, (size_t)(n - 1) * 8, "ranges"))) return r;
            if (sah && (r = tmp.get(&boxes_done, 16, "box flag"))) return r;
            if (sah)
                r = sah_one_topology(ScratchAlloc{temp_get, &tmp}, s->wbox.p, n, static_cast<int*>(cb), 10,
                                     s->tlas_nodes.p, s->perm.p, s->parents.p, st, static_cast<uint32_t*>(ranges),
                                     static_cast<uint32_t*>(boxes_done));
            else
                r = lbvh_topology(tmp, s->wbox.p, n, static_cast<int*>(cb), 10, s->tlas_nodes.p, s->perm.p,
                                  s->parents.p, st, static_cast<uint32_t*>(ranges));
            if (r) return r;
        } else {
            RG_CK(cudaMemsetAsync(s->perm.p, 0, 4, st));
        }
    }
    if (n > 1) RG_CK(cudaMemsetAsync(s->flags.p, 0, (size_t)(n - 1) * 4, st));
    RG_CK(launch_tlas_leaves_refit(s->inst_tmp.p, s->wbox.p, s->perm.p, n, s->parents.p, s->tlas_nodes.p, s->flags.p,
                                   s->inst.p, s->st, st, static_cast<const uint32_t*>(boxes_done)));
    if (s->wide) {
        WideOut out{s->tlas8.p, s->src8.p, s->item_src8.p, s->counts8.p, s->tasks8.p};
        if (refit)
            RG_CK(launch_wide_refit(s->tlas_nodes.p, s->wbox.p, s->perm.p, n, s->inst.p, s->inst8.p, s->B->d_blas.p, out,
                                    s->st, st));
        else
            RG_CK(launch_collapse(s->tlas_nodes.p, static_cast<uint32_t*>(ranges), n, s->wbox.p, nullptr, nullptr,
                                  s->inst.p, s->inst8.p, s->B->d_blas.p, out, s->st, st, 1u));
    }
    return RG_OK;
}

rg_status rg_tlas_build(rg_scene* s, const rg_instance* d_inst, uint32_t n, void* stream) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!d_inst || n == 0) return fail(RG_ERR_INVALID_ARG, "no instances");
    if (n > (1u << 28)) return fail(RG_ERR_INVALID_ARG, "too many instances");
    if (s->B->blas.empty()) return fail(RG_ERR_NOT_BUILT, "no BLAS built");
    if ((r = set_device(s))) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s->tlas_built = false;
    s->leaf_of_inst_valid = false;
    if ((r = s->tlas_nodes.ensure((size_t)(n > 1 ? n - 1 : 1) * 4, "TLAS nodes"))) return r;
    if ((r = s->inst.ensure(n, "instances"))) return r;
    if ((r = s->inst_tmp.ensure(n, "instance staging"))) return r;
    if ((r = s->wbox.ensure((size_t)n * 6, "instance boxes"))) return r;
    if ((r = s->perm.ensure(n, "TLAS order"))) return r;
    if ((r = s->parents.ensure(2 * (size_t)n, "TLAS parents"))) return r;
    if ((r = s->flags.ensure(n, "TLAS flags"))) return r;
    s->wide = false;
    if (s->desc.flags & RG_SCENE_COMPRESSED) {
        for (const BlasHost& b : s->B->blas)
            if (!b.nodes8) return fail(RG_ERR_NOT_BUILT, "a BLAS of this compressed scene has no wide form");
        const size_t n_int = n > 1 ? n - 1 : 1;
        if ((r = s->tlas8.ensure(n_int * 5, "wide TLAS nodes"))) return r;
        if ((r = s->inst8.ensure(n, "wide TLAS instances"))) return r;
        if ((r = s->src8.ensure(n_int * 8, "wide TLAS slot sources"))) return r;
        if ((r = s->item_src8.ensure(n, "wide TLAS item sources"))) return r;
        if ((r = s->counts8.ensure(4, "wide TLAS counts"))) return r;
        if ((r = s->tasks8.ensure(2 * (size_t)n, "collapse tasks"))) return r;
        s->wide = true;
    }
    if ((r = tlas_common(s, d_inst, n, st, false))) return r;
    s->n_inst = n;
    s->tlas_root = n == 1 ? kLeaf : 0u;
    s->tlas_built = true;
    return RG_OK;
}

rg_status rg_tlas_refit(rg_scene* s, const rg_instance* d_inst, uint32_t n, void* stream) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!s->tlas_built) return fail(RG_ERR_NOT_BUILT, "refit before rg_tlas_build");
    if (!d_inst || n != s->n_inst) return fail(RG_ERR_INVALID_ARG, "refit needs the instance count of the build");
    if ((r = set_device(s))) return r;
    return tlas_common(s, d_inst, n, static_cast<cudaStream_t>(stream), true);
}

rg_status rg_scene_set_materials(rg_scene* s, const rg_material* h, uint32_t n) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!h || n == 0) return fail(RG_ERR_INVALID_ARG, "no materials");
    for (uint32_t i = 0; i < n; ++i)
        if (h[i].type > RG_MAT_GLASS || (h[i].type == RG_MAT_GLASS && !(h[i].ior > 0.0f)))
            return fail(RG_ERR_INVALID_ARG, "bad material type or ior");
    if ((r = set_device(s))) return r;
    if ((r = s->mats.ensure(n, "materials"))) return r;
    RG_CK(cudaMemcpy(s->mats.p, h, n * sizeof(rg_material), cudaMemcpyHostToDevice));
    s->n_mats = n;
    return RG_OK;
}

rg_status rg_scene_set_lights(rg_scene* s, const rg_light* h, uint32_t n) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (n && !h) return fail(RG_ERR_INVALID_ARG, "NULL lights");
    if (n > kMaxLights) return fail(RG_ERR_INVALID_ARG, "more than 64 lights");
    if ((r = set_device(s))) return r;
    if ((r = s->lights.ensure(n ? n : 1, "lights"))) return r;
    if (n) RG_CK(cudaMemcpy(s->lights.p, h, n * sizeof(rg_light), cudaMemcpyHostToDevice));
    s->n_lights = n;
    return RG_OK;
}

rg_status rg_trace_rays(rg_scene* s, const rg_ray* d_rays, uint32_t n, uint32_t flags, rg_hit* d_hits, void* stream) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!s->tlas_built) return fail(RG_ERR_NOT_BUILT, "trace before rg_tlas_build");
    if (flags & ~(RG_ANY | RG_TRACE_BRUTE | RG_TRACE_STATS | RG_TRACE_PLAIN))
        return fail(RG_ERR_INVALID_ARG, "unknown trace flags");
    if ((flags & RG_TRACE_BRUTE) && (flags & RG_TRACE_STATS))
        return fail(RG_ERR_INVALID_ARG, "brute force and statistics are exclusive");
    if (n == 0) return RG_OK;
    if (!d_rays || !d_hits) return fail(RG_ERR_INVALID_ARG, "NULL ray or hit buffer");
    if ((r = set_device(s))) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TraceArgs a = base_trace_args(s, !(flags & RG_TRACE_PLAIN));
    a.rays = reinterpret_cast<const float4*>(d_rays);
    a.n = n;
    a.hits_abi = d_hits;
    // a work counter of its own, so calls on other streams may run at the same time
    uint32_t* ctr = s->trace_ctr.p + 32 * (size_t)(s->trace_slot++ % kTraceSlots);
    a.work_counter = ctr;
    a.iter_cap = iter_cap_for(s, flags & RG_TRACE_BRUTE);
    RG_CK(cudaMemsetAsync(ctr, 0, 4, st));
    const bool any = flags & RG_ANY;
    EventPair* ev;
    if ((r = event_begin(s, any ? 1 : 0, st, &ev))) return r;
    RG_CK(launch_trace(any ? kModeAnyAbi : kModeClosestAbi, flags & RG_TRACE_BRUTE, flags & RG_TRACE_STATS, a, st));
    if ((r = event_end(s, st))) return r;
    // closest hit: exact t, u, v of the hits and the tie decisions (the
    // traversal wrote provisional records that refer to the instance array it
    // walked)
    if (!any) {
        if (!s->leaf_of_inst_valid) {
            if ((r = s->leaf_of_inst.ensure(s->n_inst, "instance leaf map"))) return r;
            RG_CK(launch_invert_perm(s->perm.p, s->n_inst, s->leaf_of_inst.p, st));
            s->leaf_of_inst_valid = true;
        }
        if ((r = event_begin(s, 3, st, &ev))) return r;
        RG_CK(launch_refine_hits(a.rays, d_hits, n, s->inst.p, s->leaf_of_inst.p, s->B->d_blas.p, st));
        if ((r = event_end(s, st))) return r;
    }
    if (any)
        s->shadow_rays_host += n;
    else
        s->closest_rays += n;
    return RG_OK;
}

rg_status rg_render(rg_scene* s, const rg_camera* cam, uint32_t w, uint32_t h, uint32_t max_depth, float* d_rgba,
                    void* stream) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!s->tlas_built) return fail(RG_ERR_NOT_BUILT, "render before rg_tlas_build");
    if (!cam || !d_rgba || w == 0 || h == 0 || max_depth == 0) return fail(RG_ERR_INVALID_ARG, "bad render arguments");
    if ((uint64_t)w * h > (1ull << 28)) return fail(RG_ERR_INVALID_ARG, "image too large");
    if (s->n_mats == 0) return fail(RG_ERR_NOT_BUILT, "no materials set");
    if ((r = set_device(s))) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t N = w * h;
    const uint32_t L = s->n_lights;
    // Per depth level: closest-hit traversal, shading, shadow traversal.  The
    // shadow rays of a level and the closest-hit rays of the next depend only
    // on the level's shading and share one launch (k_trace_pair) unless
    // RG_SCENE_NO_PAIR is set or the BVH is the compressed one.  Every launch
    // reads its ray count on the device.  Counters: one block per level, [0]
    // closest work, [1] rays of the next level, [2] shadow work (and the
    // pair's), [4 + l] shadow rays toward light l.
    const size_t CB = 4 + kMaxLights;
    if ((r = s->counters.ensure(CB * ((size_t)max_depth + 1), "counters"))) return r;
    // Queue room (before anything is written to the queues: growing one
    // frees its contents).  Level d holds at most N 2^(d-1) rays (a ray spawns at most
    // two).  When that worst case for the whole frame fits the budget it is
    // allocated once and the frame is enqueued without the host waiting:
    // every count is read on the device.  Otherwise the host learns each
    // level's count one level late (copied back while the GPU traces) and
    // sizes the next queues from it.
    auto cap_of = [&](uint32_t d) { return (uint64_t)N << (d - 1); };
    bool async = !(s->desc.flags & RG_SCENE_FRUGAL) && max_depth <= 24;
    uint64_t cap_q[2] = {0, 0}, cap_max = 0;
    if (async) {
        for (uint32_t d = 1; d <= max_depth; ++d) {
            cap_q[(d - 1) & 1] = std::max(cap_q[(d - 1) & 1], cap_of(d));
            cap_max = std::max(cap_max, cap_of(d));
        }
        const uint64_t bytes = (cap_q[0] + cap_q[1]) * 48 + cap_max * 16 + cap_max * L * 48;
        async = cap_max <= 0xFFFFFFFFull && bytes <= kAsyncQueueBudget;
    }
    if (async) {
        if ((r = s->q_rays[0].ensure(2 * cap_q[0], "ray queue")) || (r = s->q_pay[0].ensure(cap_q[0], "payload queue")) ||
            (max_depth > 1 && ((r = s->q_rays[1].ensure(2 * cap_q[1], "ray queue")) ||
                               (r = s->q_pay[1].ensure(cap_q[1], "payload queue")))) ||
            (r = s->hits.ensure(cap_max, "hit queue")) ||
            (L && ((r = s->s_rays.ensure(2 * cap_max * L, "shadow queue")) ||
                   (r = s->s_pay.ensure(cap_max * L, "shadow payload")))))
            return r;
    }

    if ((r = s->q_rays[0].ensure(2 * (size_t)N, "ray queue"))) return r;
    if ((r = s->q_pay[0].ensure(N, "payload queue"))) return r;
    if ((r = s->hits.ensure(N, "hit queue"))) return r;
    if (!s->seg_count.p) {
        if ((r = s->seg_count.ensure(kShadowSplitMax, "shadow segment counts"))) return r;
        RG_CK(cudaMemsetAsync(s->seg_count.p, 0, (size_t)kShadowSplitMax * sizeof(uint32_t), st));
    }
    RG_CK(cudaMemsetAsync(s->counters.p, 0, CB * ((size_t)max_depth + 1) * sizeof(uint32_t), st));
    RG_CK(cudaMemsetAsync(d_rgba, 0, (size_t)N * 16, st));
    CameraDev cd;
    std::memcpy(&cd, cam, sizeof cd);
    RG_CK(launch_raygen(cd, w, h, s->q_rays[0].p, s->q_pay[0].p, st));

    // shading of depth level `depth` (its rays in queue q, spawns into 1 - q)
    auto shade_args = [&](uint32_t depth, int q, uint32_t* c, bool last, uint32_t n_stride) {
        ShadeArgs sa{};
        sa.rays = s->q_rays[q].p;
        sa.payload = s->q_pay[q].p;
        sa.hits = s->hits.p;
        sa.inst = s->wide ? s->inst8.p : s->inst.p;
        sa.mats = s->mats.p;
        sa.n_mats = s->n_mats;
        sa.lights = s->lights.p;
        sa.n_lights = L;
        sa.bg[0] = s->desc.background[0];
        sa.bg[1] = s->desc.background[1];
        sa.bg[2] = s->desc.background[2];
        sa.ambient = s->desc.ambient;
        sa.depth = depth;
        sa.max_depth = max_depth;
        sa.image = d_rgba;
        sa.next_rays = last ? nullptr : s->q_rays[1 - q].p;
        sa.next_payload = last ? nullptr : s->q_pay[1 - q].p;
        sa.next_count = c + 1;
        sa.shadow_rays = s->s_rays.p;
        sa.shadow_payload = s->s_pay.p;
        sa.shadow_count = c + 4;
        sa.shadow_stride = n_stride;
        sa.st = s->st;
        return sa;
    };

    // closest-hit traversal of level d (count on the host, or on the device)
    auto trace_closest = [&](int q, uint32_t n_host, const uint32_t* d_count, uint32_t* c) -> rg_status {
        TraceArgs a = base_trace_args(s, true);
        a.rays = s->q_rays[q].p;
        a.n = n_host;
        a.d_count = d_count;
        a.hits_render = s->hits.p;
        a.work_counter = c + 0;
        EventPair* ev;
        rg_status rr;
        if ((rr = event_begin(s, 0, st, &ev))) return rr;
        RG_CK(launch_trace(kModeClosestRender, false, s->desc.flags & RG_SCENE_COUNT, a, st));
        return event_end(s, st);
    };

    uint32_t n = N;  // this level's rays (a bound on them when async)
    int cur = 0;
    if ((r = trace_closest(cur, N, nullptr, s->counters.p))) return r;
    for (uint32_t depth = 1; depth <= max_depth; ++depth) {
        const bool last = depth == max_depth;
        uint32_t* c = s->counters.p + CB * (depth - 1);
        if (async) {
            n = (uint32_t)cap_of(depth);
        } else {
            // room for what this level's shading writes (growing a buffer waits for the device)
            if (L && (r = s->s_rays.ensure(2 * (size_t)n * L, "shadow queue"))) return r;
            if (L && (r = s->s_pay.ensure((size_t)n * L, "shadow payload"))) return r;
            if (!last) {
                if ((r = s->q_rays[1 - cur].ensure(4 * (size_t)n, "ray queue"))) return r;
                if ((r = s->q_pay[1 - cur].ensure(2 * (size_t)n, "payload queue"))) return r;
            }
        }

        ShadeArgs sa = shade_args(depth, cur, c, last, n);
        if (async && depth > 1) sa.d_count = c - CB + 1;  // written by the previous level's shading
        RG_CK(launch_shade(sa, n, st));
        if (!last && !async) {
            RG_CK(cudaMemcpyAsync(s->h_counts, c + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            RG_CK(cudaEventRecord(s->count_ev, st));
        }

        TraceArgs b{};
        if (L) {
            b = base_trace_args(s, true);
            b.rays = s->s_rays.p;
            b.sub_counts = c + 4;
            b.n_sub = L;
            b.sub_stride = n;
            b.payload = s->s_pay.p;
            b.image = d_rgba;
            b.work_counter = c + 2;
        }
        const bool pair = L && !last && !s->wide && !(s->desc.flags & RG_SCENE_NO_PAIR);
        if (L && last && !s->wide) {
            // the last level's shadow rays, traced on their own: when few, each
            // as segments side by side (in a pair the closest-hit rays fill
            // the lanes); the same rule with and without pairs
            b.seg_count = s->seg_count.p;
            b.split = kShadowSplit;
            b.split_max = kShadowSplitMax;
        }
        if (L && !pair) {
            EventPair* ev;
            if ((r = event_begin(s, 1, st, &ev))) return r;
            RG_CK(launch_trace(kModeShadowRender, false, s->desc.flags & RG_SCENE_COUNT, b, st));
            if ((r = event_end(s, st))) return r;
        }
        if (last) break;
        // the next level's rays (at most 2 per ray of this level) are traced
        // before the host knows how many there are
        if (!async && (r = s->hits.ensure(2 * (size_t)n, "hit queue"))) return r;
        if (pair) {
            TraceArgs a = base_trace_args(s, true);
            a.rays = s->q_rays[1 - cur].p;
            a.d_count = c + 1;
            a.hits_render = s->hits.p;
            EventPair* ev;
            if ((r = event_begin(s, 2, st, &ev))) return r;
            RG_CK(launch_trace_pair(false, s->desc.flags & RG_SCENE_COUNT, b, a, st));
            if ((r = event_end(s, st))) return r;
        } else if ((r = trace_closest(1 - cur, 0, c + 1, c + CB))) {
            return r;
        }
        cur = 1 - cur;
        if (!async) {
            RG_CK(cudaEventSynchronize(s->count_ev));
            n = s->h_counts[0];
            if (n == 0) break;
        }
    }
    return RG_OK;
}

rg_status rg_fxaa(const float* d_in, uint32_t w, uint32_t h, float* d_out, void* stream) {
    if (w == 0 || h == 0) return RG_OK;
    if (!d_in || !d_out) return fail(RG_ERR_INVALID_ARG, "NULL image");
    if (d_in == d_out) return fail(RG_ERR_INVALID_ARG, "FXAA is out-of-place: input and output alias");
    if ((uint64_t)w * h > (1ull << 28) || w > (1u << 24) || h > (1u << 24))
        return fail(RG_ERR_INVALID_ARG, "image too large");
    if (reinterpret_cast<uintptr_t>(d_in) % 16 || reinterpret_cast<uintptr_t>(d_out) % 16)
        return fail(RG_ERR_INVALID_ARG, "images must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TempAlloc tmp(st);
    void* lum;
    rg_status r;
    if ((r = tmp.get(&lum, (size_t)w * h * sizeof(float), "luma image"))) return r;
    RG_CK(launch_fxaa(reinterpret_cast<const float4*>(d_in), w, h, static_cast<float*>(lum),
                      reinterpret_cast<float4*>(d_out), st));
    return RG_OK;
}

rg_status rg_sync(rg_scene* s) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if ((r = set_device(s))) return r;
    RG_CK(cudaDeviceSynchronize());
    int err = 0;
    RG_CK(cudaMemcpy(&err, &s->st->error, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        RG_CK(cudaMemset(&s->st->error, 0, sizeof(int)));
        const char* what = err == RG_ERR_STACK       ? "traversal stack overflow"
                           : err == RG_ERR_TIMEOUT   ? "device loop iteration cap reached"
                           : err == RG_ERR_SINGULAR  ? "singular instance transform"
                           : err == RG_ERR_INVALID_ARG ? "invalid index or id found on the device"
                                                       : "device error";
        return fail(err, what);
    }
    return RG_OK;
}

rg_status rg_get_stats(rg_scene* s, rg_stats* out) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!out) return fail(RG_ERR_INVALID_ARG, "out is NULL");
    if ((r = set_device(s))) return r;
    RG_CK(cudaDeviceSynchronize());
    if ((r = collect_events(s))) return r;
    DevStatus d;
    RG_CK(cudaMemcpy(&d, s->st, sizeof d, cudaMemcpyDeviceToHost));
    out->closest_rays = s->closest_rays + d.closest_rays;  // rg_trace_rays + the renderer's launches
    out->shadow_rays = s->shadow_rays_host + d.shadow_rays;
    out->trace_launches = s->trace_launches;
    out->trace_ms = s->trace_ms;
    out->any_launches = s->any_launches;
    out->any_ms = s->any_ms;
    out->node_visits = d.count[0][0];
    out->tri_tests = d.count[0][1];
    out->inst_entries = d.count[0][2];
    out->any_node_visits = d.count[1][0];
    out->any_tri_tests = d.count[1][1];
    out->any_inst_entries = d.count[1][2];
    out->kernel_launches = launches_so_far() - s->launch_base;
    out->pair_launches = s->pair_launches;
    out->pair_ms = s->pair_ms;
    out->refine_launches = s->refine_launches;
    out->refine_ms = s->refine_ms;
    return RG_OK;
}

rg_status rg_reset_stats(rg_scene* s) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if ((r = set_device(s))) return r;
    RG_CK(cudaDeviceSynchronize());
    if ((r = collect_events(s))) return r;
    s->closest_rays = s->shadow_rays_host = 0;
    s->trace_ms = s->any_ms = s->pair_ms = s->refine_ms = 0;
    s->trace_launches = s->any_launches = s->pair_launches = s->refine_launches = 0;
    s->launch_base = launches_so_far();
    RG_CK(cudaMemset(reinterpret_cast<char*>(s->st) + offsetof(DevStatus, closest_rays), 0,
                     sizeof(DevStatus) - offsetof(DevStatus, closest_rays)));
    return RG_OK;
}

rg_status rg_tri_bounds(const float* d_vtx, uint32_t nv, const uint32_t* d_idx, uint32_t nt, float* d_lohi,
                        void* stream) {
    if (nt == 0) return RG_OK;
    if (!d_vtx || !d_idx || !d_lohi || nv == 0) return fail(RG_ERR_INVALID_ARG, "bad arguments");
    RG_CK(launch_tri_bounds(d_vtx, nv, d_idx, nt, d_lohi, nullptr, nullptr, static_cast<cudaStream_t>(stream)));
    return RG_OK;
}

rg_status rg_morton_codes(const float* d_lohi, uint32_t n, uint32_t bits, void* d_codes, float* d_cbounds,
                          void* stream) {
    if (bits != 10 && bits != 21) return fail(RG_ERR_INVALID_ARG, "bits must be 10 or 21");
    if (n == 0) return RG_OK;
    if (!d_lohi || !d_codes) return fail(RG_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TempAlloc tmp(st);
    void* cb;
    rg_status r;
    if ((r = tmp.get(&cb, 64, "centroid bounds"))) return r;
    RG_CK(launch_init_bounds(static_cast<int*>(cb), st));
    RG_CK(launch_centroid_bounds(d_lohi, n, static_cast<int*>(cb), st));
    RG_CK(launch_morton(d_lohi, n, static_cast<int*>(cb), (int)bits, d_codes, nullptr, d_cbounds, st));
    return RG_OK;
}

rg_status rg_radix_sort_pairs(const void* d_keys, const uint32_t* d_vals, uint32_t n, uint32_t key_bits,
                              void* d_keys_out, uint32_t* d_vals_out, void* stream) {
    if (key_bits != 32 && key_bits != 64) return fail(RG_ERR_INVALID_ARG, "key_bits must be 32 or 64");
    if (n == 0) return RG_OK;
    if (!d_keys || !d_vals || !d_keys_out || !d_vals_out) return fail(RG_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TempAlloc tmp(st);
    void* scratch;
    rg_status r;
    if ((r = tmp.get(&scratch, radix_sort_scratch_bytes(n, (int)key_bits), "sort scratch"))) return r;
    RG_CK(radix_sort_pairs(d_keys, d_vals, n, (int)key_bits, d_keys_out, d_vals_out, scratch, st));
    return RG_OK;
}

rg_status rg_karras(const void* d_sorted_keys, uint32_t n, uint32_t key_bits, uint32_t* d_children,
                    uint32_t* d_parents, void* stream) {
    if (key_bits != 32 && key_bits != 64) return fail(RG_ERR_INVALID_ARG, "key_bits must be 32 or 64");
    if (n < 2 || !d_sorted_keys || !d_children) return fail(RG_ERR_INVALID_ARG, "bad arguments");
    RG_CK(launch_karras(d_sorted_keys, n, (int)key_bits, d_children, 2, d_parents, static_cast<cudaStream_t>(stream)));
    return RG_OK;
}

rg_status rg_blas_export(rg_scene* s, uint32_t blas_id, void* h_nodes, void* h_tris, uint32_t* h_root) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (blas_id >= s->B->blas.size()) return fail(RG_ERR_INVALID_ARG, "no such BLAS");
    if ((r = set_device(s))) return r;
    RG_CK(cudaDeviceSynchronize());
    const BlasHost& b = s->B->blas[blas_id];
    if (h_nodes && b.nt > 1) RG_CK(cudaMemcpy(h_nodes, b.nodes, (size_t)(b.nt - 1) * 64, cudaMemcpyDeviceToHost));
    // the (x, y, z) order of each triangle record
    if (h_tris) RG_CK(cudaMemcpy2D(h_tris, 48, b.tris, kTriRecord, 48, b.nt, cudaMemcpyDeviceToHost));
    if (h_root) *h_root = b.root;
    return RG_OK;
}

rg_status rg_wide_export(rg_scene* s, uint32_t blas_id, void* h_nodes, uint32_t* h_src, uint32_t* h_item_src,
                         uint32_t* h_counts) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if ((r = set_device(s))) return r;
    const float4* nodes;
    const uint32_t *src, *item_src, *counts;
    if (blas_id == RG_TLAS_ID) {
        if (!s->tlas_built || !s->wide) return fail(RG_ERR_NOT_BUILT, "no wide TLAS");
        nodes = s->tlas8.p;
        src = s->src8.p;
        item_src = s->item_src8.p;
        counts = s->counts8.p;
    } else {
        if (blas_id >= s->B->blas.size()) return fail(RG_ERR_INVALID_ARG, "no such BLAS");
        const BlasHost& b = s->B->blas[blas_id];
        if (!b.nodes8) return fail(RG_ERR_NOT_BUILT, "this BLAS has no wide form");
        nodes = b.nodes8;
        src = b.src8;
        item_src = b.item_src8;
        counts = b.counts8;
    }
    RG_CK(cudaDeviceSynchronize());
    uint32_t c[2];
    RG_CK(cudaMemcpy(c, counts, sizeof c, cudaMemcpyDeviceToHost));
    if (h_counts) {
        h_counts[0] = c[0];
        h_counts[1] = c[1];
    }
    if (h_nodes) RG_CK(cudaMemcpy(h_nodes, nodes, (size_t)c[0] * 80, cudaMemcpyDeviceToHost));
    if (h_src) RG_CK(cudaMemcpy(h_src, src, (size_t)c[0] * 32, cudaMemcpyDeviceToHost));
    if (h_item_src) RG_CK(cudaMemcpy(h_item_src, item_src, (size_t)c[1] * 4, cudaMemcpyDeviceToHost));
    return RG_OK;
}

rg_status rg_tlas_export(rg_scene* s, void* h_nodes, float* h_wbox, float* h_inv, uint32_t* h_order,
                         uint32_t* h_root) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!s->tlas_built) return fail(RG_ERR_NOT_BUILT, "no TLAS");
    if ((r = set_device(s))) return r;
    RG_CK(cudaDeviceSynchronize());
    const uint32_t n = s->n_inst;
    if (h_nodes && n > 1) RG_CK(cudaMemcpy(h_nodes, s->tlas_nodes.p, (size_t)(n - 1) * 64, cudaMemcpyDeviceToHost));
    if (h_wbox) RG_CK(cudaMemcpy(h_wbox, s->wbox.p, (size_t)n * 24, cudaMemcpyDeviceToHost));
    if (h_order) RG_CK(cudaMemcpy(h_order, s->perm.p, (size_t)n * 4, cudaMemcpyDeviceToHost));
    if (h_inv) {
        std::vector<InstDev> v(n);
        RG_CK(cudaMemcpy(v.data(), s->inst.p, (size_t)n * sizeof(InstDev), cudaMemcpyDeviceToHost));
        for (uint32_t j = 0; j < n; ++j) {
            uint32_t k = v[j].id;
            if (k >= n) return fail(RG_ERR_CUDA, "corrupt instance table");
            for (int row = 0; row < 3; ++row) {
                h_inv[12 * (size_t)k + 4 * row + 0] = v[j].inv[row].x;
                h_inv[12 * (size_t)k + 4 * row + 1] = v[j].inv[row].y;
                h_inv[12 * (size_t)k + 4 * row + 2] = v[j].inv[row].z;
                h_inv[12 * (size_t)k + 4 * row + 3] = v[j].inv[row].w;
            }
        }
    }
    if (h_root) *h_root = s->tlas_root;
    return RG_OK;
}

}  // extern "C"

namespace rg {
rg_status scene_view(rg_scene* s, SceneView* v) {
    rg_status r;
    if ((r = check_scene(s))) return r;
    if (!s->tlas_built) return fail(RG_ERR_NOT_BUILT, "scene has no TLAS");
    if (s->n_mats == 0) return fail(RG_ERR_NOT_BUILT, "scene has no materials");
    v->device = s->device;
    v->d_blas = s->B->d_blas.p;
    v->n_blas = (uint32_t)s->B->blas.size();
    v->tlas_nodes = s->tlas_nodes.p;
    v->perm = s->perm.p;
    v->parents = s->parents.p;
    v->inst = s->inst.p;
    v->n_inst = s->n_inst;
    v->tlas_root = s->tlas_root;
    v->mats = s->mats.p;
    v->n_mats = s->n_mats;
    v->lights = s->lights.p;
    v->n_lights = s->n_lights;
    for (int k = 0; k < 3; ++k) v->bg[k] = s->desc.background[k];
    v->ambient = s->desc.ambient;
    v->iter_cap = iter_cap_for(s, false);
    return RG_OK;
}
}  // namespace rg

namespace rg {
rg_status report_error(rg_status code, const char* msg) { return fail(code, msg); }

static std::atomic<unsigned long long> g_launches{0};
static thread_local bool g_capturing = false;
void count_launches(unsigned n) {
    if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
void set_capturing(bool on) { g_capturing = on; }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

int device_sm_count() {
    // looked up once per process; concurrent first callers store the same value
    static std::atomic<int> cached{0};
    int sms = cached.load(std::memory_order_relaxed);
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        cached.store(sms, std::memory_order_relaxed);
    }
    return sms;
}
}  // namespace rg
