// Continuous-batching render server (include/rg.h, "continuous-batching
// render server").  The per-ray work is the renderer's (Sec. 1 and 2.1 of
// "Running on Raygun": closest hit, shadow rays, reflection and refraction to
// a fixed depth); what this file adds is the batching around it:
//
//  * one ring of 2^k path rays (ray 32 B + payload 16 B) shared by every
//    request in flight; the payload's pixel word carries the request slot and
//    the ray depth, so one launch traces rays of many requests;
//  * a step traces the m oldest rays of the ring (closest hit), shades them
//    (shadow rays into a dense queue, reflected / refracted rays appended to
//    the ring), and advances the ring head; the shadow rays a step makes are
//    traced by the next step, in one launch with its closest-hit rays (or,
//    with RG_SERVER_NO_PAIR, by the same step after shading), so a request
//    completes one step after its last path ray;
//  * per-slot live counts (path rays still in the ring) tell the host which
//    requests finished;
//  * per-request TLAS: on admission, a slot's private copy of the scene's TLAS
//    is refit with the request's instance transforms;
//  * the step's launches and copies are one CUDA graph; each slot's refit
//    sequence per scene is another;
//  * lanes: a server holds one or more independent rings (lanes), each with
//    its own queues, request slots, stream and step graph; a request lives in
//    one lane (admitted to the least loaded), and one server step runs a step
//    of every lane with work at the same time, so that the idle tails of one
//    lane's launches (the last rays of a launch, a few long ones) are filled
//    by the others' work, as frames in flight are for rg_render.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "rg_internal.cuh"

using namespace rg;

namespace {

// Ring positions are free-running 32-bit counters; entry = position & mask.
// A step consumes m rays, the oldest (from head) or, when the ring is nearly
// full, the newest (from the tail: the deepest rays, so the work proceeds
// depth first and the live rays stay bounded); spawned rays are appended.
struct RingState {
    uint32_t head, tail;        // oldest live ray, one past the newest
    uint32_t gen_base;          // where this step's primary rays start
    uint32_t next_base;         // where this step's spawned rays start (the tail after ray generation)
    uint32_t cons;              // first ray consumed by this step
    uint32_t work_closest, next_count, work_shadow;
    uint32_t pad[4];
    int slot_live[kMaxSlots];   // path rays of each slot in the ring
    uint32_t shadow_count[kMaxLights];       // shadow rays toward each light made by this step (one sub-queue each)
    uint32_t prev_shadow_count[kMaxLights];  // the same for the previous step (traced by this one when paired)
};

// Host -> device once per step.
struct __align__(16) StepHdr {
    uint32_t n_reqs;            // requests admitted this step
    uint32_t n_new_rays;        // their primary rays (sum of w h)
    uint32_t m;                 // rays traced this step
    uint32_t new_mask;          // slots (re)started this step
    uint32_t newest_first;      // consume the m newest rays instead of the m oldest
    uint32_t pad[3];
    int live_init[kMaxSlots];
    RaygenReq reqs[kMaxSlots];  // offsets ascending
    SlotDev slots[kMaxSlots];
};

// Device -> host once per step.
struct __align__(16) StepOut {
    uint32_t head, tail, next_count, shadow_count;
    int error, pad[3];
    int slot_live[kMaxSlots];
};

// begin, raygen, closest + previous shadow (paired) or closest and shadow, shade, close gap, end
constexpr unsigned kStepKernelsPaired = 6, kStepKernelsApart = 7;
constexpr unsigned kRefitKernels = 2;  // instance prep, TLAS leaf refit

__global__ void k_step_begin(const StepHdr* __restrict__ hdr, RingState* __restrict__ rs) {
    const uint32_t l = threadIdx.x;
    if (l < kMaxSlots && ((hdr->new_mask >> l) & 1u)) rs->slot_live[l] = hdr->live_init[l];
    if (l == 0) {
        const uint32_t t = rs->tail;
        const uint32_t T = t + hdr->n_new_rays;
        rs->gen_base = t;
        rs->tail = T;
        rs->next_base = T;
        rs->cons = hdr->newest_first ? T - hdr->m : rs->head;
        rs->work_closest = 0;
        rs->next_count = 0;
        rs->work_shadow = 0;
    }
    for (uint32_t k = l; k < kMaxLights; k += blockDim.x) {
        rs->prev_shadow_count[k] = rs->shadow_count[k];
        rs->shadow_count[k] = 0;
    }
}

// Newest-first steps leave the consumed rays [T - m, T) as a gap below the
// spawned ones [T, T + next): the last min(m, next) spawned rays move into it
// (order in the ring does not matter; source and target do not overlap).
__global__ void k_close_gap(const StepHdr* __restrict__ hdr, const RingState* __restrict__ rs, uint32_t mask,
                            float4* __restrict__ rays, Payload* __restrict__ payload) {
    if (!hdr->newest_first) return;
    const uint32_t m = hdr->m, T = rs->next_base, next = rs->next_count;
    const uint32_t k = min(m, next);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint32_t src = (T + next - k + i) & mask, dst = (T - m + i) & mask;
        rays[2 * (size_t)dst] = rays[2 * (size_t)src];
        rays[2 * (size_t)dst + 1] = rays[2 * (size_t)src + 1];
        payload[dst] = payload[src];
    }
}

__global__ void k_step_end(const StepHdr* __restrict__ hdr, RingState* __restrict__ rs, StepOut* __restrict__ out,
                           const DevStatus* __restrict__ st) {
    const uint32_t l = threadIdx.x;
    if (l < kMaxSlots) out->slot_live[l] = rs->slot_live[l];
    if (l == 0) {
        if (hdr->newest_first) {
            rs->tail = rs->next_base - hdr->m + rs->next_count;
        } else {
            rs->head += hdr->m;
            rs->tail = rs->next_base + rs->next_count;
        }
        out->head = rs->head;
        out->tail = rs->tail;
        out->next_count = rs->next_count;
        uint32_t shadow = 0;
        for (uint32_t k = 0; k < kMaxLights; ++k) shadow += rs->shadow_count[k];
        out->shadow_count = shadow;
        out->error = st->error;
    }
}

rg_status sfail(rg_status code, const std::string& msg) { return report_error(code, msg.c_str()); }

// An empty ring whose positions (head, tail) start at `start`.  Positions are
// free-running 32-bit counters (ring entries are positions masked by the
// capacity, sizes are differences of positions), so any start is valid; the
// tests start near 2^32 to make a run wrap the counters (RG_TEST_RING_START,
// read when a server is created; 0 otherwise).
cudaError_t reset_ring(RingState* d_rs, uint32_t start) {
    RingState rs;
    std::memset(&rs, 0, sizeof rs);
    rs.head = rs.tail = rs.gen_base = rs.next_base = rs.cons = start;
    return cudaMemcpy(d_rs, &rs, sizeof rs, cudaMemcpyHostToDevice);
}

uint32_t ring_start_for_tests() {
    const char* v = std::getenv("RG_TEST_RING_START");
    return (v && *v) ? (uint32_t)std::strtoul(v, nullptr, 0) : 0u;
}

rg_status scuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    return sfail(e == cudaErrorMemoryAllocation ? RG_ERR_OOM : RG_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define SV_CK(call)                                      \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return scuda(e_, #call);  \
    } while (0)

template <class T>
rg_status salloc(T** p, size_t n, const char* what) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return scuda(e, what);
    }
    return RG_OK;
}

struct SceneEntry {
    rg_scene* scene;
    SceneView v;
    std::vector<rg_instance> base;  // build order
};

struct SlotBufs {
    float4* tlas_nodes = nullptr;
    InstDev* inst = nullptr;
    InstDev* inst_tmp = nullptr;
    float* wbox = nullptr;
    uint32_t* flags = nullptr;
    rg_instance* d_inst = nullptr;
    rg_instance* h_inst = nullptr;            // pinned staging
    std::vector<cudaGraphExec_t> refit_exec;  // per scene
};

struct Pending {
    uint64_t id;
    rg_request r;
    std::vector<float> transforms;  // empty: the scene's own
};

struct Active {
    bool on = false;
    bool flushing = false;  // no path rays left; its last shadow rays are traced by the next step
    uint64_t id = 0, tag = 0;
    uint32_t scene = 0, admitted_step = 0;
};

const char* device_error_text(int err) {
    return err == RG_ERR_STACK      ? "traversal stack overflow"
           : err == RG_ERR_TIMEOUT  ? "device loop iteration cap reached"
           : err == RG_ERR_SINGULAR ? "singular instance transform"
           : err == RG_ERR_INVALID_ARG ? "invalid instance BLAS id or material index"
                                       : "device error";
}

}  // namespace

// One lane by default: on the serving stream (200 requests/s, one or two in
// flight at a time) four lanes measured 2 % more busy throughput and a worse
// tail latency, since most of the time only one request, in one lane, has work.
constexpr uint32_t kDefaultLanes = 1;

// One lane: a ring of path rays with its queues, request slots, status word,
// stream and step graph.
struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    DevStatus* st = nullptr;
    float4* ring_rays = nullptr;
    Payload* ring_pay = nullptr;
    HitDev* hits = nullptr;
    float4* s_rays = nullptr;
    Payload* s_pay = nullptr;
    RingState* d_rs = nullptr;
    StepHdr* d_hdr = nullptr;
    StepOut* d_out = nullptr;
    StepHdr* h_hdr = nullptr;
    StepOut* h_out = nullptr;
    SlotBufs slots[kMaxSlots];
    Active active[kMaxSlots];
    uint32_t ring_rays_now = 0;  // tail - head after the lane's last step
    uint32_t admitted = 0;       // primary rays admitted for the lane's coming step
    cudaGraphExec_t step_exec = nullptr;
    bool in_flight = false;      // a step launched and not yet booked
    uint64_t launch_seq = 0;     // order of the launches in flight (the oldest is waited for)
};

struct rg_server {
    int device = 0;
    uint32_t ring_cap = 0, ring_mask = 0, batch = 0, max_lights = 0, flags = 0, admit = 0;
    size_t shadow_cap = 0;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    uint32_t* d_tune_count = nullptr;
    std::vector<Lane> lanes;
    std::vector<SceneEntry> scenes;
    uint32_t max_inst = 0, iter_cap = 64;
    std::deque<Pending> pending;
    std::deque<rg_completion> done;
    uint64_t next_id = 1;
    uint32_t ring_start = 0;     // ring position of an empty ring at creation (a test hook; 0)
    uint64_t launches = 0;       // lane steps launched so far
    TraceShape shape[2];
    rg_server_stats stats{};
};

namespace {

rg_status set_dev(rg_server* s) {
    SV_CK(cudaSetDevice(s->device));
    return RG_OK;
}

// Shadow rays traced by the next step, with its closest-hit rays.
bool paired(const rg_server* s) { return !(s->flags & RG_SERVER_NO_PAIR); }

// Whether a lane's step must run although its ring is empty: paired steps
// leave the last shadow rays of finished requests to the next step.
bool shadow_flush_due(const Lane& L) {
    for (const Active& a : L.active)
        if (a.on && a.flushing) return true;
    return false;
}

void free_slot_bufs(SlotBufs& b) {
    cudaFree(b.tlas_nodes);
    cudaFree(b.inst);
    cudaFree(b.inst_tmp);
    cudaFree(b.wbox);
    cudaFree(b.flags);
    cudaFree(b.d_inst);
    if (b.h_inst) cudaFreeHost(b.h_inst);
    for (cudaGraphExec_t g : b.refit_exec)
        if (g) cudaGraphExecDestroy(g);
    b = SlotBufs();
}

void drop_step_graph(rg_server* s) {
    for (Lane& L : s->lanes) {
        if (L.step_exec) cudaGraphExecDestroy(L.step_exec);
        L.step_exec = nullptr;
    }
}

rg_status alloc_slot_bufs(SlotBufs& b, uint32_t n, size_t n_scenes) {
    rg_status r;
    const size_t n_int = n > 1 ? n - 1 : 1;
    if ((r = salloc(&b.tlas_nodes, n_int * 4, "slot TLAS nodes"))) return r;
    if ((r = salloc(&b.inst, n, "slot instances"))) return r;
    if ((r = salloc(&b.inst_tmp, n, "slot instance staging"))) return r;
    if ((r = salloc(&b.wbox, (size_t)n * 6, "slot instance boxes"))) return r;
    if ((r = salloc(&b.flags, n_int, "slot refit flags"))) return r;
    if ((r = salloc(&b.d_inst, n, "slot instance records"))) return r;
    SV_CK(cudaMallocHost(reinterpret_cast<void**>(&b.h_inst), (size_t)n * sizeof(rg_instance)));
    b.refit_exec.assign(n_scenes, nullptr);
    return RG_OK;
}

// The refit of slot k's TLAS copy for a request of scene e (transforms already
// in the slot's pinned staging).
rg_status enqueue_refit(rg_server* s, Lane& L, uint32_t k, uint32_t e) {
    const SceneView& v = s->scenes[e].v;
    SlotBufs& b = L.slots[k];
    const uint32_t n = v.n_inst;
    SV_CK(cudaMemcpyAsync(b.d_inst, b.h_inst, (size_t)n * sizeof(rg_instance), cudaMemcpyHostToDevice, L.stream));
    SV_CK(launch_instance_prep(b.d_inst, n, v.d_blas, v.n_blas, b.inst_tmp, b.wbox, nullptr, false, L.st, L.stream));
    if (n > 1) {
        SV_CK(cudaMemcpyAsync(b.tlas_nodes, v.tlas_nodes, (size_t)(n - 1) * 64, cudaMemcpyDeviceToDevice, L.stream));
        SV_CK(cudaMemsetAsync(b.flags, 0, (size_t)(n - 1) * 4, L.stream));
    }
    SV_CK(launch_tlas_leaves_refit(b.inst_tmp, b.wbox, v.perm, n, v.parents, b.tlas_nodes, b.flags, b.inst, L.st,
                                   L.stream));
    return RG_OK;
}

TraceArgs closest_args(rg_server* s, Lane& L, const uint32_t* d_count) {
    TraceArgs a{};
    a.rays = L.ring_rays;
    a.d_count = d_count;
    a.payload = L.ring_pay;
    a.hits_render = L.hits;
    a.work_counter = &L.d_rs->work_closest;
    a.st = L.st;
    a.iter_cap = s->iter_cap;
    a.slots = L.d_hdr->slots;
    a.ring_head = &L.d_rs->cons;
    a.ring_mask = s->ring_mask;
    return a;
}

TraceArgs shadow_args(rg_server* s, Lane& L, const uint32_t* counts) {
    TraceArgs b{};
    b.rays = L.s_rays;
    b.sub_counts = counts;
    b.n_sub = s->max_lights;
    b.sub_stride = s->batch;
    b.payload = L.s_pay;
    b.work_counter = &L.d_rs->work_shadow;
    b.st = L.st;
    b.iter_cap = s->iter_cap;
    b.slots = L.d_hdr->slots;
    return b;
}

ShadeArgs shade_args(rg_server* s, Lane& L, const uint32_t* d_count) {
    ShadeArgs a{};
    a.rays = L.ring_rays;
    a.payload = L.ring_pay;
    a.hits = L.hits;
    a.d_count = d_count;
    a.next_rays = L.ring_rays;
    a.next_payload = L.ring_pay;
    a.next_count = &L.d_rs->next_count;
    a.shadow_rays = L.s_rays;
    a.shadow_payload = L.s_pay;
    a.shadow_count = L.d_rs->shadow_count;
    a.shadow_stride = s->batch;
    a.max_lights = s->max_lights;
    a.st = L.st;
    a.slots = L.d_hdr->slots;
    a.slot_live = L.d_rs->slot_live;
    a.ring_head = &L.d_rs->cons;
    a.next_base = &L.d_rs->next_base;
    a.ring_mask = s->ring_mask;
    return a;
}

// Everything one step of a lane puts on the lane's stream, graph-capturable
// (all counts are read on the device).
rg_status enqueue_step(rg_server* s, Lane& L) {
    SV_CK(cudaMemcpyAsync(L.d_hdr, L.h_hdr, sizeof(StepHdr), cudaMemcpyHostToDevice, L.stream));
    k_step_begin<<<1, 32, 0, L.stream>>>(L.d_hdr, L.d_rs);
    count_launches(1);
    SV_CK(cudaGetLastError());
    SV_CK(launch_raygen_batch(L.d_hdr->reqs, &L.d_hdr->n_reqs, s->ring_cap / 2, &L.d_hdr->n_new_rays,
                              &L.d_rs->gen_base, s->ring_mask, L.ring_rays, L.ring_pay, L.stream));
    if (paired(s)) {
        // the previous step's shadow rays with this step's closest-hit rays;
        // shading then refills the shadow queue
        SV_CK(launch_trace_pair(true, false, shadow_args(s, L, L.d_rs->prev_shadow_count),
                                closest_args(s, L, &L.d_hdr->m), L.stream, s->shape[0]));
        SV_CK(launch_shade_batch(shade_args(s, L, &L.d_hdr->m), L.stream));
    } else {
        SV_CK(launch_trace(kModeClosestBatch, false, false, closest_args(s, L, &L.d_hdr->m), L.stream, s->shape[0]));
        SV_CK(launch_shade_batch(shade_args(s, L, &L.d_hdr->m), L.stream));
        SV_CK(launch_trace(kModeShadowBatch, false, false, shadow_args(s, L, L.d_rs->shadow_count), L.stream,
                           s->shape[1]));
    }
    k_close_gap<<<device_sm_count() * 4, 256, 0, L.stream>>>(L.d_hdr, L.d_rs, s->ring_mask, L.ring_rays, L.ring_pay);
    count_launches(1);
    SV_CK(cudaGetLastError());
    k_step_end<<<1, 32, 0, L.stream>>>(L.d_hdr, L.d_rs, L.d_out, L.st);
    count_launches(1);
    SV_CK(cudaGetLastError());
    SV_CK(cudaMemcpyAsync(L.h_out, L.d_out, sizeof(StepOut), cudaMemcpyDeviceToHost, L.stream));
    return RG_OK;
}

// Captures `body` on `stream` into an executable graph.
template <class F>
rg_status capture(rg_server* s, cudaStream_t stream, F body, cudaGraphExec_t* out) {
    *out = nullptr;
    SV_CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed));
    set_capturing(true);
    rg_status r = body();
    set_capturing(false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(stream, &g);
    if (r != RG_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return scuda(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return scuda(e, "cudaGraphInstantiate");
    }
    s->stats.graph_captures++;
    return RG_OK;
}

rg_status run_step_work(rg_server* s, Lane& L) {
    if (s->flags & RG_SERVER_NO_GRAPH) {
        const unsigned long long before = launches_so_far();
        rg_status r = enqueue_step(s, L);
        s->stats.kernel_launches += launches_so_far() - before;
        return r;
    }
    rg_status r;
    if (!L.step_exec && (r = capture(s, L.stream, [&] { return enqueue_step(s, L); }, &L.step_exec))) return r;
    SV_CK(cudaGraphLaunch(L.step_exec, L.stream));
    const unsigned k = paired(s) ? kStepKernelsPaired : kStepKernelsApart;
    count_launches(k);
    s->stats.kernel_launches += k;
    s->stats.graph_launches++;
    return RG_OK;
}

rg_status run_refit(rg_server* s, Lane& L, uint32_t k, uint32_t e) {
    if (s->flags & RG_SERVER_NO_GRAPH) {
        const unsigned long long before = launches_so_far();
        rg_status r = enqueue_refit(s, L, k, e);
        s->stats.kernel_launches += launches_so_far() - before;
        return r;
    }
    rg_status r;
    cudaGraphExec_t& g = L.slots[k].refit_exec[e];
    if (!g && (r = capture(s, L.stream, [&] { return enqueue_refit(s, L, k, e); }, &g))) return r;
    SV_CK(cudaGraphLaunch(g, L.stream));
    count_launches(kRefitKernels);
    s->stats.kernel_launches += kRefitKernels;
    s->stats.graph_launches++;
    return RG_OK;
}

rg_status check_server(rg_server* s) {
    if (!s) return sfail(RG_ERR_INVALID_ARG, "null server");
    return RG_OK;
}

rg_status check_request(rg_server* s, const rg_request* q) {
    if (!q) return sfail(RG_ERR_INVALID_ARG, "null request");
    if (q->scene >= s->scenes.size()) return sfail(RG_ERR_INVALID_ARG, "unknown scene id");
    const uint64_t px = (uint64_t)q->width * q->height;
    if (q->width == 0 || q->height == 0 || px > RG_SERVER_MAX_PIXELS)
        return sfail(RG_ERR_INVALID_ARG, "request size out of range");
    if (px > s->ring_cap / 2) return sfail(RG_ERR_INVALID_ARG, "request larger than half the ray ring");
    if (q->max_depth < 1 || q->max_depth > RG_SERVER_MAX_DEPTH)
        return sfail(RG_ERR_INVALID_ARG, "max_depth out of range");
    if (!q->d_rgba) return sfail(RG_ERR_INVALID_ARG, "null image");
    if (reinterpret_cast<uintptr_t>(q->d_rgba) % 16) return sfail(RG_ERR_INVALID_ARG, "image not 16-byte aligned");
    return RG_OK;
}

// Admission: in arrival order, each request into the least loaded lane (the
// fewest rays in its ring plus those admitted to it this step) that has a
// free slot and room: the lane's rays stay within the admission bound, or the
// request runs alone in an empty lane (within half the ring).  The first
// request no lane takes stops admission (no overtaking).
rg_status admit(rg_server* s) {
    for (Lane& L : s->lanes) {
        if (L.in_flight) continue;
        L.h_hdr->n_reqs = 0;
        L.h_hdr->new_mask = 0;
        L.admitted = 0;
    }
    while (!s->pending.empty()) {
        Pending& p = s->pending.front();
        const uint32_t px = p.r.width * p.r.height;
        Lane* best = nullptr;
        uint32_t best_k = 0;
        uint64_t best_load = 0;
        for (Lane& L : s->lanes) {
            if (L.in_flight) continue;  // its header is in use by the step in flight
            const uint64_t load = (uint64_t)L.ring_rays_now + L.admitted;
            const bool alone = load == 0 && px <= s->ring_cap / 2;
            if (load + px > s->admit && !alone) continue;
            uint32_t k = 0;
            while (k < kMaxSlots && L.active[k].on) ++k;
            if (k == kMaxSlots) continue;
            if (!best || load < best_load) {
                best = &L;
                best_k = k;
                best_load = load;
            }
        }
        if (!best) break;
        Lane& L = *best;
        const uint32_t k = best_k;
        StepHdr& H = *L.h_hdr;
        const SceneEntry& E = s->scenes[p.r.scene];
        const uint32_t n = E.v.n_inst;
        rg_instance* hi = L.slots[k].h_inst;
        std::memcpy(hi, E.base.data(), (size_t)n * sizeof(rg_instance));
        if (!p.transforms.empty())
            for (uint32_t i = 0; i < n; ++i) std::memcpy(hi[i].m, &p.transforms[12 * (size_t)i], 48);
        rg_status r;
        if ((r = run_refit(s, L, k, p.r.scene))) return r;
        RaygenReq& q = H.reqs[H.n_reqs++];
        std::memcpy(&q.cam, &p.r.camera, sizeof(CameraDev));
        q.w = p.r.width;
        q.h = p.r.height;
        q.slot = k;
        q.offset = L.admitted;
        q.image = p.r.d_rgba;
        SlotDev& D = H.slots[k];
        D.tlas_nodes = L.slots[k].tlas_nodes;
        D.inst = L.slots[k].inst;
        D.tlas_root = E.v.tlas_root;
        D.mats = E.v.mats;
        D.n_mats = E.v.n_mats;
        D.lights = E.v.lights;
        D.n_lights = E.v.n_lights;
        D.image = p.r.d_rgba;
        D.max_depth = p.r.max_depth;
        for (int c = 0; c < 3; ++c) D.bg[c] = E.v.bg[c];
        D.ambient = E.v.ambient;
        H.live_init[k] = (int)px;
        H.new_mask |= 1u << k;
        Active& A = L.active[k];
        A.on = true;
        A.id = p.id;
        A.tag = p.r.tag;
        A.scene = p.r.scene;
        A.admitted_step = (uint32_t)(s->stats.steps + 1);
        L.admitted += px;
        s->stats.admitted++;
        s->pending.pop_front();
    }
    for (Lane& L : s->lanes)
        if (!L.in_flight) L.h_hdr->n_new_rays = L.admitted;
    return RG_OK;
}

// Rays one step traces with `avail` rays in the ring, and from which end.
// Oldest first while the free ring F takes the worst case (two spawned rays
// per traced ray) of at least a quarter of a full batch; else newest first
// with m <= F / (2 (RG_SERVER_MAX_DEPTH + 1)): a newest-first descent grows
// the ring by at most m per step until its rays reach their depth limit, so
// it always finds room.  0: no room at all (F < 2 (RG_SERVER_MAX_DEPTH + 1)).
uint32_t step_batch(const rg_server* s, uint32_t avail, bool* newest_first) {
    uint64_t want = std::min<uint64_t>(avail, s->batch);
    if (s->max_lights) want = std::min<uint64_t>(want, s->shadow_cap / s->max_lights);
    const uint64_t F = s->ring_cap - (uint64_t)avail;
    const uint64_t m_old = std::min<uint64_t>(want, F / 2);
    *newest_first = false;
    if (4 * m_old >= want) return (uint32_t)m_old;
    *newest_first = true;
    return (uint32_t)std::min<uint64_t>(want, F / (2 * (RG_SERVER_MAX_DEPTH + 1)));
}

// Waits for a lane's step and books its results: ring count, completed
// requests (their images are final), device errors.
rg_status finish_step(rg_server* s, Lane& L, uint32_t* n_completed) {
    SV_CK(cudaEventSynchronize(L.done_ev));
    L.in_flight = false;
    s->stats.lane_steps++;
    const StepOut& O = *L.h_out;
    s->stats.closest_rays += L.h_hdr->m;
    s->stats.shadow_rays += O.shadow_count;
    L.ring_rays_now = O.tail - O.head;
    s->stats.ring_peak = std::max(s->stats.ring_peak, L.ring_rays_now);
    int64_t live_sum = 0;
    uint32_t completed = 0;
    for (uint32_t k = 0; k < kMaxSlots; ++k) {
        if (!L.active[k].on) {
            if (O.slot_live[k] != 0) return sfail(RG_ERR_CUDA, "render server: rays of a free slot in the ring");
            continue;
        }
        if (O.slot_live[k] < 0) return sfail(RG_ERR_CUDA, "render server: negative live ray count");
        live_sum += O.slot_live[k];
        if (O.slot_live[k] == 0 && paired(s) && s->max_lights && !L.active[k].flushing) {
            L.active[k].flushing = true;  // complete after the next step traces its last shadow rays
            continue;
        }
        if (O.slot_live[k] == 0) {
            rg_completion c;
            c.id = L.active[k].id;
            c.tag = L.active[k].tag;
            c.admitted_step = L.active[k].admitted_step;
            c.completed_step = (uint32_t)s->stats.steps;
            s->done.push_back(c);
            L.active[k] = Active();
            s->stats.completed++;
            ++completed;
        }
    }
    if (n_completed) *n_completed += completed;
    if (O.error) {
        // the step completed (a ray that failed counts as a miss); report it
        SV_CK(cudaMemset(&L.st->error, 0, sizeof(int)));
        return sfail(O.error, std::string("render server step: ") + device_error_text(O.error));
    }
    if (live_sum != (int64_t)L.ring_rays_now) return sfail(RG_ERR_CUDA, "render server: ring count mismatch");
    return RG_OK;
}

uint32_t n_active(const rg_server* s) {
    uint32_t c = 0;
    for (const Lane& L : s->lanes)
        for (const Active& a : L.active) c += a.on ? 1u : 0u;
    return c;
}

uint32_t ring_rays_total(const rg_server* s) {
    uint32_t c = 0;
    for (const Lane& L : s->lanes) c += L.ring_rays_now;
    return c;
}

// ---- autotuner cache: a JSON array, one object per line ---------------------
std::string device_key(int dev, int* sms) {
    cudaDeviceProp p{};
    cudaGetDeviceProperties(&p, dev);
    *sms = p.multiProcessorCount;
    return std::string(p.name);
}

bool read_num(const std::string& line, const std::string& key, long* v) {
    size_t p = line.find("\"" + key + "\"");
    if (p == std::string::npos) return false;
    p = line.find(':', p);
    if (p == std::string::npos) return false;
    *v = std::strtol(line.c_str() + p + 1, nullptr, 10);
    return true;
}

bool parse_shape(const std::string& obj, TraceShape* sh) {
    long b, bps, g, st = 0;
    if (!read_num(obj, "block", &b) || !read_num(obj, "blocks_per_sm", &bps) || !read_num(obj, "refill", &g)) return false;
    read_num(obj, "stack", &st);  // absent in caches written before the short stack: 0
    if ((b != 64 && b != 128 && b != 256) || bps < 0 || bps > 64 || g < 0 || g > 32) return false;
    if (!(st == 0 || (b == 128 && (st == 8 || st == 16)))) return false;
    sh->block = (int)b;
    sh->blocks_per_sm = (int)bps;
    sh->refill = (int)g;
    sh->stack = (int)st;
    return true;
}

std::vector<std::string> read_lines(const char* path) {
    std::vector<std::string> out;
    FILE* f = std::fopen(path, "r");
    if (!f) return out;
    char buf[4096];
    std::string cur;
    while (std::fgets(buf, sizeof buf, f)) {
        cur += buf;
        if (!cur.empty() && cur.back() == '\n') {
            out.push_back(cur);
            cur.clear();
        }
    }
    if (!cur.empty()) out.push_back(cur);
    std::fclose(f);
    return out;
}

bool cache_lookup(const char* path, const std::string& dev, int sms, TraceShape sh[2]) {
    for (const std::string& line : read_lines(path)) {
        if (line.find("\"device\": \"" + dev + "\"") == std::string::npos) continue;
        long n;
        if (!read_num(line, "sms", &n) || n != sms) continue;
        const size_t c = line.find("\"closest\""), d = line.find("\"shadow\"");
        if (c == std::string::npos || d == std::string::npos || d < c) continue;
        TraceShape a, b;
        if (parse_shape(line.substr(c, d - c), &a) && parse_shape(line.substr(d), &b)) {
            sh[0] = a;
            sh[1] = b;
            return true;
        }
    }
    return false;
}

std::string shape_json(const TraceShape& t, float ms) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "{\"block\": %d, \"blocks_per_sm\": %d, \"refill\": %d, \"stack\": %d, \"ms\": %.4f}",
                  t.block, t.blocks_per_sm, t.refill, t.stack, ms);
    return buf;
}

rg_status cache_store(const char* path, const std::string& dev, int sms, const TraceShape sh[2], const float ms[2]) {
    std::vector<std::string> keep;
    for (const std::string& line : read_lines(path)) {
        if (line.find("\"device\"") == std::string::npos) continue;
        long n = -1;
        read_num(line, "sms", &n);
        if (line.find("\"device\": \"" + dev + "\"") != std::string::npos && n == sms) continue;
        std::string l = line;
        while (!l.empty() && (l.back() == '\n' || l.back() == ',' || l.back() == ' ' || l.back() == ']')) l.pop_back();
        if (!l.empty() && l.front() == '[') l.erase(0, 1);
        keep.push_back(l);
    }
    char head[256];
    std::snprintf(head, sizeof head, "{\"device\": \"%s\", \"sms\": %d, ", dev.c_str(), sms);
    keep.push_back(std::string(head) + "\"closest\": " + shape_json(sh[0], ms[0]) + ", \"shadow\": " +
                   shape_json(sh[1], ms[1]) + "}");
    FILE* f = std::fopen(path, "w");
    if (!f) return sfail(RG_ERR_INVALID_ARG, std::string("cannot write ") + path);
    std::fputs("[\n", f);
    for (size_t i = 0; i < keep.size(); ++i) std::fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    std::fputs("]\n", f);
    std::fclose(f);
    return RG_OK;
}

}  // namespace

extern "C" {

rg_status rg_server_create(rg_server** out, const rg_server_desc* desc) {
    if (!out) return sfail(RG_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    rg_server_desc d{};
    if (desc) d = *desc;
    const uint32_t lg = d.ring_log2 ? d.ring_log2 : 25u;
    if (lg < 16 || lg > 30) return sfail(RG_ERR_INVALID_ARG, "ring_log2 must be in 16..30");
    rg_server* s = new rg_server();
    s->ring_cap = 1u << lg;
    s->ring_mask = s->ring_cap - 1;
    s->batch = d.batch_rays ? d.batch_rays : (1u << 23);
    s->batch = std::min(s->batch, s->ring_cap / 2);
    s->max_lights = d.max_lights ? d.max_lights : 4u;
    if (s->max_lights > kMaxLights) {
        delete s;
        return sfail(RG_ERR_INVALID_ARG, "max_lights above 64");
    }
    s->shadow_cap = (size_t)s->batch * s->max_lights;
    s->flags = d.flags;
    s->admit = std::min(d.admit_rays ? d.admit_rays : s->batch, s->ring_cap / 2);
    const uint32_t n_lanes = d.lanes ? d.lanes : kDefaultLanes;
    if (n_lanes > RG_SERVER_MAX_LANES) {
        delete s;
        return sfail(RG_ERR_INVALID_ARG, "lanes above RG_SERVER_MAX_LANES");
    }
    rg_status r = RG_OK;
    auto bail = [&](rg_status code) {
        rg_server_destroy(s);
        return code;
    };
    if (cudaGetDevice(&s->device) != cudaSuccess) return bail(scuda(cudaGetLastError(), "cudaGetDevice"));
    if (cudaEventCreate(&s->t0) != cudaSuccess || cudaEventCreate(&s->t1) != cudaSuccess)
        return bail(sfail(RG_ERR_CUDA, "cudaEventCreate failed"));
    if ((r = salloc(&s->d_tune_count, 1, "tuning count"))) return bail(r);
    s->ring_start = ring_start_for_tests();
    s->lanes.resize(n_lanes);
    for (Lane& L : s->lanes) {
        if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(sfail(RG_ERR_CUDA, "cudaStreamCreate failed"));
        if (cudaEventCreateWithFlags(&L.done_ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(sfail(RG_ERR_CUDA, "cudaEventCreate failed"));
        if ((r = salloc(&L.st, 1, "server status"))) return bail(r);
        if ((r = salloc(&L.ring_rays, 2 * (size_t)s->ring_cap, "ray ring"))) return bail(r);
        if ((r = salloc(&L.ring_pay, (size_t)s->ring_cap, "payload ring"))) return bail(r);
        if ((r = salloc(&L.hits, (size_t)s->batch, "hit queue"))) return bail(r);
        if ((r = salloc(&L.s_rays, 2 * s->shadow_cap, "shadow queue"))) return bail(r);
        if ((r = salloc(&L.s_pay, s->shadow_cap, "shadow payload"))) return bail(r);
        if ((r = salloc(&L.d_rs, 1, "ring state"))) return bail(r);
        if ((r = salloc(&L.d_hdr, 1, "step header"))) return bail(r);
        if ((r = salloc(&L.d_out, 1, "step result"))) return bail(r);
        if (cudaMallocHost(reinterpret_cast<void**>(&L.h_hdr), sizeof(StepHdr)) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&L.h_out), sizeof(StepOut)) != cudaSuccess)
            return bail(sfail(RG_ERR_OOM, "pinned host buffers"));
        std::memset(L.h_hdr, 0, sizeof(StepHdr));
        std::memset(L.h_out, 0, sizeof(StepOut));
        if (cudaMemset(L.st, 0, sizeof(DevStatus)) != cudaSuccess || reset_ring(L.d_rs, s->ring_start) != cudaSuccess ||
            cudaMemset(L.d_hdr, 0, sizeof(StepHdr)) != cudaSuccess)
            return bail(scuda(cudaGetLastError(), "cudaMemset"));
    }
    *out = s;
    return RG_OK;
}

rg_status rg_server_destroy(rg_server* s) {
    if (!s) return RG_OK;
    cudaSetDevice(s->device);
    for (Lane& L : s->lanes)
        if (L.stream) cudaStreamSynchronize(L.stream);
    drop_step_graph(s);
    for (Lane& L : s->lanes) {
        for (SlotBufs& b : L.slots) free_slot_bufs(b);
        cudaFree(L.st);
        cudaFree(L.ring_rays);
        cudaFree(L.ring_pay);
        cudaFree(L.hits);
        cudaFree(L.s_rays);
        cudaFree(L.s_pay);
        cudaFree(L.d_rs);
        cudaFree(L.d_hdr);
        cudaFree(L.d_out);
        if (L.h_hdr) cudaFreeHost(L.h_hdr);
        if (L.h_out) cudaFreeHost(L.h_out);
        if (L.done_ev) cudaEventDestroy(L.done_ev);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    cudaFree(s->d_tune_count);
    if (s->t0) cudaEventDestroy(s->t0);
    if (s->t1) cudaEventDestroy(s->t1);
    delete s;
    return RG_OK;
}

rg_status rg_server_add_scene(rg_server* s, rg_scene* scene, uint32_t* scene_id) {
    rg_status r;
    if ((r = check_server(s))) return r;
    if (!scene || !scene_id) return sfail(RG_ERR_INVALID_ARG, "null scene or id");
    if (!s->pending.empty() || n_active(s)) return sfail(RG_ERR_INVALID_ARG, "add scenes while the server is idle");
    SceneEntry E;
    E.scene = scene;
    if ((r = scene_view(scene, &E.v))) return r;
    if (E.v.device != s->device) return sfail(RG_ERR_INVALID_ARG, "scene on another device");
    if (E.v.n_lights > s->max_lights) return sfail(RG_ERR_INVALID_ARG, "scene has more lights than max_lights");
    if ((r = set_dev(s))) return r;
    // the scene's own instance records, back in build order
    const uint32_t n = E.v.n_inst;
    SV_CK(cudaDeviceSynchronize());  // the scene may have been built on any stream
    std::vector<InstDev> leaf(n);
    SV_CK(cudaMemcpy(leaf.data(), E.v.inst, (size_t)n * sizeof(InstDev), cudaMemcpyDeviceToHost));
    E.base.assign(n, rg_instance{});
    std::vector<char> seen(n, 0);
    for (const InstDev& D : leaf) {
        if (D.id >= n || seen[D.id]) return sfail(RG_ERR_INVALID_ARG, "scene TLAS is inconsistent");
        seen[D.id] = 1;
        rg_instance& I = E.base[D.id];
        for (int row = 0; row < 3; ++row) {
            I.m[row][0] = D.m[row].x;
            I.m[row][1] = D.m[row].y;
            I.m[row][2] = D.m[row].z;
            I.m[row][3] = D.m[row].w;
        }
        I.blas_id = D.blas;
        I.material_id = D.material;
        I.mask = 0xFFu;
    }
    // slot buffers sized for the largest scene; every refit graph is per scene
    const size_t n_scenes = s->scenes.size() + 1;
    if (n > s->max_inst) {
        for (Lane& L : s->lanes)
            for (SlotBufs& b : L.slots) free_slot_bufs(b);
        for (Lane& L : s->lanes)
            for (SlotBufs& b : L.slots)
                if ((r = alloc_slot_bufs(b, n, n_scenes))) return r;
        s->max_inst = n;
        drop_step_graph(s);
    } else {
        for (Lane& L : s->lanes)
            for (SlotBufs& b : L.slots) b.refit_exec.resize(n_scenes, nullptr);
    }
    s->iter_cap = std::max(s->iter_cap, E.v.iter_cap);
    drop_step_graph(s);
    s->scenes.push_back(std::move(E));
    *scene_id = (uint32_t)(s->scenes.size() - 1);
    return RG_OK;
}

rg_status rg_server_submit(rg_server* s, const rg_request* q, uint64_t* id) {
    rg_status r;
    if ((r = check_server(s))) return r;
    if ((r = check_request(s, q))) return r;
    Pending p;
    p.id = s->next_id++;
    p.r = *q;
    if (q->h_transforms) {
        const size_t n = 12 * (size_t)s->scenes[q->scene].v.n_inst;
        p.transforms.assign(q->h_transforms, q->h_transforms + n);
    }
    p.r.h_transforms = nullptr;
    s->pending.push_back(std::move(p));
    s->stats.submitted++;
    if (id) *id = s->pending.back().id;
    return RG_OK;
}

bool any_in_flight(const rg_server* s) {
    for (const Lane& L : s->lanes)
        if (L.in_flight) return true;
    return false;
}

// Books every lane whose step has finished, waiting first for the oldest
// launch in flight when none has.
rg_status book_finished(rg_server* s, uint32_t* n_completed) {
    Lane* oldest = nullptr;
    bool any_done = false;
    for (Lane& L : s->lanes) {
        if (!L.in_flight) continue;
        if (!oldest || L.launch_seq < oldest->launch_seq) oldest = &L;
        const cudaError_t q = cudaEventQuery(L.done_ev);
        if (q == cudaSuccess) any_done = true;
        else if (q != cudaErrorNotReady) return scuda(q, "cudaEventQuery");
    }
    if (!oldest) return RG_OK;
    if (!any_done) SV_CK(cudaEventSynchronize(oldest->done_ev));
    rg_status r = RG_OK;
    for (Lane& L : s->lanes) {
        if (!L.in_flight || cudaEventQuery(L.done_ev) != cudaSuccess) continue;
        const rg_status q = finish_step(s, L, n_completed);
        if (!r) r = q;
    }
    return r;
}

rg_status rg_server_step(rg_server* s, uint32_t* n_completed) {
    rg_status r;
    if (n_completed) *n_completed = 0;
    if ((r = check_server(s))) return r;
    if ((r = set_dev(s))) return r;
    if ((r = admit(s))) return r;
    // a step on every idle lane with work, each on its own stream
    for (Lane& L : s->lanes) {
        if (L.in_flight) continue;
        const uint32_t avail = L.ring_rays_now + L.admitted;
        // an empty ring still takes a step while finished requests wait for their last shadow rays
        if (avail == 0 && !shadow_flush_due(L)) continue;
        bool newest = false;
        const uint32_t m = avail ? step_batch(s, avail, &newest) : 0u;
        if (avail && m == 0) {
            r = sfail(RG_ERR_OOM, "ray ring full: no room for the rays a step spawns");
            break;
        }
        L.h_hdr->m = m;
        L.h_hdr->newest_first = newest ? 1u : 0u;
        if (newest) s->stats.newest_first_steps++;
        if ((r = run_step_work(s, L))) break;
        SV_CK(cudaEventRecord(L.done_ev, L.stream));
        L.in_flight = true;
        L.launch_seq = ++s->launches;
    }
    if (!any_in_flight(s)) return r;
    s->stats.steps++;
    // returns once at least one lane's step is booked (the others run on)
    const rg_status q = book_finished(s, n_completed);
    return r ? r : q;
}

rg_status rg_server_drain(rg_server* s) {
    rg_status r;
    if ((r = check_server(s))) return r;
    while (!s->pending.empty() || n_active(s) || any_in_flight(s)) {
        const uint64_t before = s->stats.steps;
        if ((r = rg_server_step(s, nullptr))) return r;
        if (s->stats.steps == before) return sfail(RG_ERR_INVALID_ARG, "render server cannot make progress");
    }
    return RG_OK;
}

// Waits for (and books) every lane's step in flight.
rg_status settle(rg_server* s) {
    rg_status r = RG_OK;
    while (any_in_flight(s)) {
        const rg_status q = book_finished(s, nullptr);
        if (!r) r = q;
    }
    return r;
}

rg_status rg_server_poll(rg_server* s, rg_completion* out, uint32_t max, uint32_t* n) {
    rg_status r;
    if ((r = check_server(s))) return r;
    if (!n || (max && !out)) return sfail(RG_ERR_INVALID_ARG, "null output");
    uint32_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return RG_OK;
}

rg_status rg_server_get_stats(rg_server* s, rg_server_stats* out) {
    rg_status r;
    if ((r = check_server(s))) return r;
    if (!out) return sfail(RG_ERR_INVALID_ARG, "null output");
    *out = s->stats;
    out->pending = (uint32_t)s->pending.size();
    out->active = n_active(s);
    out->ring_rays = ring_rays_total(s);
    return RG_OK;
}

rg_status rg_server_set_shape(rg_server* s, uint32_t which, const rg_trace_shape* sh) {
    rg_status r;
    if ((r = check_server(s))) return r;
    if (which > 1 || !sh) return sfail(RG_ERR_INVALID_ARG, "bad shape selector");
    if ((sh->block != 64 && sh->block != 128 && sh->block != 256) || sh->blocks_per_sm > 64 || sh->refill > 32)
        return sfail(RG_ERR_INVALID_ARG, "bad launch shape");
    if (!(sh->stack == 0 || (sh->block == 128 && (sh->stack == 8 || sh->stack == 16))))
        return sfail(RG_ERR_INVALID_ARG, "short stack: 0, or 8 or 16 entries with 128 threads per block");
    if ((r = settle(s))) return r;
    s->shape[which].block = (int)sh->block;
    s->shape[which].blocks_per_sm = (int)sh->blocks_per_sm;
    s->shape[which].refill = (int)sh->refill;
    s->shape[which].stack = (int)sh->stack;
    drop_step_graph(s);
    return RG_OK;
}

rg_status rg_server_get_shape(rg_server* s, uint32_t which, rg_trace_shape* out) {
    rg_status r;
    if ((r = check_server(s))) return r;
    if (which > 1 || !out) return sfail(RG_ERR_INVALID_ARG, "bad shape selector");
    out->block = (uint32_t)s->shape[which].block;
    out->blocks_per_sm = (uint32_t)s->shape[which].blocks_per_sm;
    out->refill = (uint32_t)s->shape[which].refill;
    out->stack = (uint32_t)s->shape[which].stack;
    out->ms = -1.0f;
    return RG_OK;
}

rg_status rg_server_autotune(rg_server* s, const rg_request* sample, const char* cache_path, uint32_t flags,
                             rg_trace_shape out[2]) {
    rg_status r;
    if ((r = check_server(s))) return r;
    if ((r = check_request(s, sample))) return r;
    if (!s->pending.empty() || n_active(s) || any_in_flight(s))
        return sfail(RG_ERR_INVALID_ARG, "autotune needs an idle server");
    if ((r = set_dev(s))) return r;
    int sms = 0;
    const std::string dev = device_key(s->device, &sms);
    TraceShape best[2] = {s->shape[0], s->shape[1]};
    float best_ms[2] = {-1.0f, -1.0f};
    const bool cached = cache_path && !(flags & RG_TUNE_FORCE) && cache_lookup(cache_path, dev, sms, best);
    if (!cached) {
        // the sample's primary rays into the ring of lane 0 (the least loaded of
        // an idle server): a step that traces nothing
        Lane& L = s->lanes[0];
        const uint32_t px = sample->width * sample->height;
        bool newest = false;
        const uint32_t m = std::min(px, step_batch(s, px, &newest));
        if ((r = rg_server_submit(s, sample, nullptr))) return r;
        if ((r = admit(s))) return r;
        L.h_hdr->m = 0;
        L.h_hdr->newest_first = 0;
        const uint32_t saved_flags = s->flags;
        s->flags |= RG_SERVER_NO_GRAPH;
        r = enqueue_step(s, L);
        s->flags = saved_flags;
        if (r) return r;
        SV_CK(cudaMemcpyAsync(s->d_tune_count, &m, 4, cudaMemcpyHostToDevice, L.stream));
        SV_CK(cudaStreamSynchronize(L.stream));
        const int blocks[3] = {64, 128, 256}, bps[3] = {0, 4, 8}, refills[4] = {8, 16, 24, 32}, stacks[3] = {0, 8, 16};
        auto time_one = [&](int which, const TraceShape& t, float* ms) -> rg_status {
            float best_t = 1e30f;
            for (int rep = 0; rep < 4; ++rep) {
                uint32_t* wc = which == 0 ? &L.d_rs->work_closest : &L.d_rs->work_shadow;
                SV_CK(cudaMemsetAsync(wc, 0, 4, L.stream));
                SV_CK(cudaEventRecord(s->t0, L.stream));
                if (which == 0)
                    SV_CK(launch_trace(kModeClosestBatch, false, false, closest_args(s, L, s->d_tune_count), L.stream,
                                       t));
                else
                    SV_CK(launch_trace(kModeShadowBatch, false, false, shadow_args(s, L, L.d_rs->shadow_count),
                                       L.stream, t));
                SV_CK(cudaEventRecord(s->t1, L.stream));
                SV_CK(cudaEventSynchronize(s->t1));
                float e = 0;
                SV_CK(cudaEventElapsedTime(&e, s->t0, s->t1));
                if (rep > 0) best_t = std::min(best_t, e);
            }
            *ms = best_t;
            return RG_OK;
        };
        for (int which = 0; which < 2; ++which) {
            if (which == 1) {
                // one shading pass makes the shadow rays (its spawned rays are discarded below)
                SV_CK(cudaMemsetAsync(&L.d_rs->work_closest, 0, 4, L.stream));
                SV_CK(launch_trace(kModeClosestBatch, false, false, closest_args(s, L, s->d_tune_count), L.stream,
                                   best[0]));
                SV_CK(launch_shade_batch(shade_args(s, L, s->d_tune_count), L.stream));
            }
            best_ms[which] = 1e30f;
            for (int b : blocks)
                for (int q : bps)
                    for (int g : refills)
                        for (int sd : stacks) {
                            if (sd && b != 128) continue;  // short stacks are compiled for 128 threads
                            TraceShape t;
                            t.block = b;
                            t.blocks_per_sm = q;
                            t.refill = g;
                            t.stack = sd;
                            float ms;
                            if ((r = time_one(which, t, &ms))) return r;
                            if (ms < best_ms[which]) {
                                best_ms[which] = ms;
                                best[which] = t;
                            }
                        }
        }
        // back to an empty ring and a free slot
        SV_CK(cudaStreamSynchronize(L.stream));
        int err = 0;
        SV_CK(cudaMemcpy(&err, &L.st->error, sizeof(int), cudaMemcpyDeviceToHost));
        SV_CK(reset_ring(L.d_rs, s->ring_start));
        SV_CK(cudaMemset(&L.st->error, 0, sizeof(int)));
        L.ring_rays_now = 0;
        L.admitted = 0;
        for (Active& a : L.active) a = Active();
        s->stats.admitted--;
        s->stats.submitted--;
        if (err) return sfail(err, std::string("autotune: ") + device_error_text(err));
        if (cache_path && (r = cache_store(cache_path, dev, sms, best, best_ms))) return r;
    }
    s->shape[0] = best[0];
    s->shape[1] = best[1];
    drop_step_graph(s);
    if (out)
        for (int w = 0; w < 2; ++w) {
            out[w].block = (uint32_t)best[w].block;
            out[w].blocks_per_sm = (uint32_t)best[w].blocks_per_sm;
            out[w].refill = (uint32_t)best[w].refill;
            out[w].stack = (uint32_t)best[w].stack;
            out[w].ms = best_ms[w];
        }
    return RG_OK;
}

}  // extern "C"
