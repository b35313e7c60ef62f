// Internal layout and launcher declarations of librg (not part of the ABI).
//
// Device data layout (all arrays 16-byte aligned, read with 16-byte vector
// loads on the traversal path):
//
//   BVH node, 64 B (BLAS and TLAS alike), binary, both child boxes inline:
//     float4 n0 = {lo0.x, lo0.y, lo0.z, hi0.x}
//     float4 n1 = {hi0.y, hi0.z, lo1.x, lo1.y}
//     float4 n2 = {lo1.z, hi1.x, hi1.y, hi1.z}
//     uint4  n3 = {child0, child1, 0, 0}      bit 31 set = leaf index, else node index
//   Internal node i is Karras's node i; the root is node 0 (a one-leaf tree has
//   no nodes and its root reference is the leaf itself).
//
//   Triangle, 48 B, stored in BLAS leaf order (sorted by Morton code):
//     float4 {v0.xyz, prim (uint32 bits)}  float4 {v1.xyz, 0}  float4 {v2.xyz, 0}
//
//   Instance, 128 B, stored in TLAS leaf order (InstDev below): float32
//   world-to-object rows, BLAS pointers, ids, object-to-world rows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rg.h"

namespace rg {

constexpr uint32_t kLeaf = 0x80000000u;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kMiss = 0xFFFFFFFFu;

// A BLAS triangle record: the three vertices (float4 each, prim in the first
// one's w) in the axis orders (x, y, z), (y, z, x) and (z, x, y), 144 B.  The
// watertight test reads the order whose last axis is the ray's dominant one,
// so it needs no per-coordinate selection; shading reads the first.
constexpr size_t kTriRecord = 144;
constexpr uint32_t kTriStride = 9;  // float4s per triangle record

struct __align__(16) InstDev {
    float4 inv[3];          // world -> object rows (float32 of the float64 inverse)
    const float4* nodes;    // BLAS nodes
    const float4* tris;     // BLAS triangle records (kTriRecord each)
    uint32_t root;          // BLAS root reference
    uint32_t id;            // index in the caller's instance array
    uint32_t material;
    uint32_t blas;
    float4 m[3];            // object -> world rows (as given)
};
static_assert(sizeof(InstDev) == 128, "instance record is 128 B");

struct __align__(16) BlasDev {
    const float4* nodes;
    const float4* tris;
    uint32_t root;
    uint32_t nt;
    float lo[3];
    float hi[3];
    const float4* nodes8;   // compressed 8-wide BVH (null if not built)
    const float4* tris8;    // its triangles, in wide-leaf order
    // bound on |v - c|^2 over the vertices, c = (lo + hi) * 0.5, every
    // operation rounded upward (bits of a non-negative float, atomicMax-able)
    uint32_t r2_bits;
    uint32_t pad;
    const uint32_t* leaf_of_prim;  // BLAS leaf (triangle record) of each triangle index
};
static_assert(sizeof(BlasDev) == 80, "BLAS descriptor is 80 B");

// ---------------------------------------------------------------- wide BVH
// Compressed 8-wide node, 80 B (five 16 B words):
//   w0 = {p.x, p.y, p.z, bits(ex | ey << 8 | ez << 16 | imask << 24)}
//   w1 = {child_base, item_base, meta[0..3], meta[4..7]}
//   w2 = {qlo.x[0..3], qlo.x[4..7], qlo.y[0..3], qlo.y[4..7]}
//   w3 = {qlo.z[0..3], qlo.z[4..7], qhi.x[0..3], qhi.x[4..7]}
//   w4 = {qhi.y[0..3], qhi.y[4..7], qhi.z[0..3], qhi.z[4..7]}
// Child box of slot s along axis a: [p_a + qlo_a[s] * 2^e_a, p_a + qhi_a[s] * 2^e_a]
// (e_a a signed byte), rounded outward at build time so that it contains the
// exact float32 box.  imask bit s = slot s is an internal child; internal
// children are stored consecutively from child_base in slot order.  A leaf slot
// has meta = count << 5 | offset: items item_base + offset .. + count - 1; an
// empty slot has meta = 0 and no imask bit.  Slot s holds a child lying toward
// octant s of the node (bit a of s set: the negative side of axis a), so a ray
// visits children in the order of (s ^ its direction-sign bits), highest first.
constexpr int kWideLeafMax = 3;  // largest number of items a leaf slot may hold (count is 2 bits)

struct WideOut {
    float4* nodes;      // 5 float4 per node
    uint32_t* src;      // 8 per node: binary-tree reference of each slot (kNone if empty)
    uint32_t* item_src; // per item: binary leaf index it was copied from
    uint32_t* counts;   // [0] nodes, [1] items (written at the end)
    uint2* tasks;       // scratch: 2 x n task entries
};

// Per-ray payload of the wavefront renderer, 16 B: pixel index and the RGB
// weight (throughput for path rays, unshadowed contribution for shadow rays).
struct __align__(16) Payload {
    uint32_t pixel;
    float r, g, b;
};

// Batched wavefront (serving): rays of several requests share the queues; the
// payload's pixel word packs the request slot, the ray depth and the pixel.
constexpr uint32_t kPixelBits = 23, kDepthBits = 4, kSlotBits = 5;
constexpr uint32_t kMaxSlots = 1u << kSlotBits;
constexpr uint32_t kMaxBatchDepth = (1u << kDepthBits) - 1;
__host__ __device__ __forceinline__ uint32_t pack_pixel(uint32_t pixel, uint32_t depth, uint32_t slot) {
    return pixel | (depth << kPixelBits) | (slot << (kPixelBits + kDepthBits));
}
__host__ __device__ __forceinline__ uint32_t px_of(uint32_t w) { return w & ((1u << kPixelBits) - 1u); }
__host__ __device__ __forceinline__ uint32_t depth_of(uint32_t w) { return (w >> kPixelBits) & ((1u << kDepthBits) - 1u); }
__host__ __device__ __forceinline__ uint32_t slot_of_px(uint32_t w) { return w >> (kPixelBits + kDepthBits); }

// One request slot of the batched wavefront: its TLAS (a per-request copy
// refit with the request's transforms), its scene's shading tables, and its
// image.
struct __align__(16) SlotDev {
    const float4* tlas_nodes;
    const InstDev* inst;
    const rg_material* mats;
    const rg_light* lights;
    float* image;
    uint32_t tlas_root;
    uint32_t n_mats;
    uint32_t n_lights;
    uint32_t max_depth;
    float bg[3];
    float ambient;
};

// Internal closest-hit record of the renderer, 16 B: TLAS leaf of the
// instance, BLAS leaf of the triangle, t.
struct __align__(16) HitDev {
    uint32_t inst_leaf;
    uint32_t tri_leaf;
    float t;
    uint32_t pad;
};

// Device-side status word and statistics of one scene.
struct DevStatus {
    int error;                 // first rg_status recorded by a kernel
    int pad;
    unsigned long long closest_rays;
    unsigned long long shadow_rays;
    unsigned long long count[2][3];  // [closest, any][node visits, triangle tests, instance entries]
};

// Kernels launched by the library since process start (host counter).
void count_launches(unsigned n);
// While set (per host thread), count_launches ignores launches: they are
// being captured into a CUDA graph, whose replays are counted instead.
void set_capturing(bool on);
unsigned long long launches_so_far();

__device__ __forceinline__ void record_error(DevStatus* st, int code) {
    if (st) atomicCAS(&st->error, 0, code);
}

// Monotone map of float32 to int32 (for atomicMin/atomicMax on floats).
__device__ __forceinline__ int f2ord(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

// ---------------------------------------------------------------- launchers
// build.cu
cudaError_t launch_tri_bounds(const float* vtx, uint32_t nv, const uint32_t* idx, uint32_t nt, float* lohi,
                              int* cb_ord, DevStatus* st, cudaStream_t s);
cudaError_t launch_init_bounds(int* cb_ord, cudaStream_t s);
cudaError_t launch_centroid_bounds(const float* lohi, uint32_t n, int* cb_ord, cudaStream_t s);
cudaError_t launch_morton(const float* lohi, uint32_t n, const int* cb_ord, int bits, void* codes, uint32_t* vals,
                          float* cb_out, cudaStream_t s);
// Radix sort; scratch must hold radix_sort_scratch_bytes(n, key_bits) bytes:
// ping-pong keys and values, and 256 digit counts per tile of kSortTilePairs
// pairs, each part 256-byte aligned.
constexpr uint32_t kSortTilePairs = 2048;
constexpr size_t radix_sort_scratch_bytes(uint32_t n, int key_bits) {
    return ((((size_t)n * (key_bits == 64 ? 8 : 4)) + 255) & ~(size_t)255) + ((((size_t)n * 4) + 255) & ~(size_t)255) +
           ((((size_t)256 * ((n + kSortTilePairs - 1) / kSortTilePairs) * 4) + 255) & ~(size_t)255);
}
cudaError_t radix_sort_pairs(const void* keys_in, const uint32_t* vals_in, uint32_t n, int key_bits, void* keys_out,
                             uint32_t* vals_out, void* scratch, cudaStream_t s);
// ranges (optional, 2 per internal node): first and last leaf of node i.
cudaError_t launch_karras(const void* keys, uint32_t n, int key_bits, uint32_t* child_base, int child_stride_words,
                          uint32_t* parents, cudaStream_t s, uint32_t* ranges = nullptr);
cudaError_t launch_blas_leaves_refit(const float* vtx, const uint32_t* idx, const uint32_t* perm, const float* lohi,
                                     uint32_t n, const uint32_t* parents, float4* nodes, uint32_t* flags,
                                     float4* tris, BlasDev* blas_out, DevStatus* st, cudaStream_t s);
// Bounding sphere of a mesh about its root box centre (after the BLAS refit
// wrote the root box): blas->r2_bits = max over the vertices.
cudaError_t launch_bound_sphere(const float* vtx, uint32_t nv, BlasDev* blas, cudaStream_t s);
// inv[perm[j]] = j for j < n (perm a permutation of 0..n-1).
cudaError_t launch_invert_perm(const uint32_t* perm, uint32_t n, uint32_t* inv, cudaStream_t s);
cudaError_t launch_instance_prep(const rg_instance* in, uint32_t n, const BlasDev* blas, uint32_t nblas,
                                 InstDev* tmp, float* wbox, int* cb_ord, bool check_blas, DevStatus* st,
                                 cudaStream_t s);
// The whole TLAS build (refit = false) or refit of n <= kTlasSmallMax
// instances in one single-block launch; same results as instance prep +
// bounds + Morton + sort + Karras + leaves refit.  ranges may be NULL.
constexpr uint32_t kTlasSmallMax = 1024;
cudaError_t launch_tlas_small(const rg_instance* in, uint32_t n, const BlasDev* blas, uint32_t nblas, InstDev* tmp,
                              float* wbox, bool refit, float4* nodes, uint32_t* perm, uint32_t* parents,
                              uint32_t* flags, uint32_t* ranges, InstDev* inst_out, DevStatus* st, cudaStream_t s);
// The instances in leaf order and the bottom-up refit of the node boxes; with
// boxes_done set (device memory, may be null) the boxes are already in place
// and only the instances are copied.
cudaError_t launch_tlas_leaves_refit(const InstDev* tmp, const float* wbox, const uint32_t* perm, uint32_t n,
                                     const uint32_t* parents, float4* nodes, uint32_t* flags, InstDev* inst_out,
                                     DevStatus* st, cudaStream_t s, const uint32_t* boxes_done = nullptr);

// Karras hierarchies over segments of the sorted keys (the bottom of the SAH
// build): segment k spans leaves begin .. begin + count - 1 and its internal
// nodes are node .. node + count - 2 (its root is `node`, whose parent entry
// the caller writes); `first` numbers its internal nodes in one flat range of
// n_threads threads (ascending over the segments).
struct KarrasSeg {
    uint32_t begin, count, node, first;
};
cudaError_t launch_karras_segments(const void* keys, int key_bits, const KarrasSeg* segs, uint32_t n_segs,
                                   uint32_t n_threads, uint32_t n_leaves, float4* nodes, uint32_t* parents,
                                   uint32_t* ranges, cudaStream_t s);

// sah.cu: binned-SAH topology, one level of segments per launch sequence.
constexpr int kSahBins = 16;            // bins per axis
constexpr uint32_t kSahChunk = 2048;    // triangles per block of a level's kernels
constexpr uint32_t kSahSmall = 2;       // segments of at most this many triangles get the Karras hierarchy
constexpr uint32_t kSahMaxLevels = 40;  // deeper segments get the Karras hierarchy whatever their size
constexpr uint32_t kSahSliceTasks = 65536;  // segments per launch sequence (bounds the scratch)
constexpr uint32_t kSahOneMax = 4096;       // items of the build without host round trips (launch_sah_small)
constexpr uint32_t kSahAccInts = 6 + 3 * kSahBins * 7;  // per task: centroid bounds, then 7 values per bin and axis
struct SahTask {                        // one segment split at this level
    uint32_t begin, count, node;        // leaves begin .. begin + count - 1, internal node `node`
    uint32_t first_block, n_blocks;     // its blocks in the level's block list
    uint32_t pad[3];
};
struct SahParam {                       // per task: binning frame and the chosen split
    float cmin[3], scale[3];
    int axis, split;                    // axis -1: halved by position
    uint32_t nl;                        // triangles on the left
    uint32_t pad[3];
};
struct SahLevel {
    const float* lohi;                  // triangle boxes (lo xyz, hi xyz)
    uint32_t n_leaves, m, n_blocks;     // triangles of the mesh, tasks, blocks
    const SahTask* tasks;
    const uint2* blk;                   // per block: task, first position of its chunk
    int* acc;                           // per task: centroid bounds and bins (scratch)
    SahParam* par;
    uint32_t* prim_at;                  // triangle at each position (updated)
    void* key_at;                       // its Morton code (updated)
    uint32_t* prim_out;                 // scratch, n
    void* key_out;                      // scratch, n
    uint32_t *blk_left, *blk_off;       // scratch, per block
    uint32_t* out_nl;                   // per task: triangles on the left
    float4* nodes;
    uint32_t* parents;
    uint32_t* ranges;                   // may be null
};
cudaError_t launch_sah_level(const SahLevel& L, int key_bits, cudaStream_t s);
// The same binned-SAH hierarchy for 2 <= n <= kSahOneMax items from their
// 30-bit Morton codes, in three launches without host round trips (the sort
// and the top levels in one block, then the subtrees of at most 128 items in
// a block each, then the leaf order): perm_out (the item of each leaf),
// children, parents, (optional) leaf ranges, and the boxes of every node's
// children where the splits give them; *boxes_done is 1 when every node's
// boxes were written, 0 when the bottom-up refit must compute them.
struct SahSmallScratch {
    uint32_t* keys;       // n: the sorted codes
    uint32_t* perm0;      // n: the Morton order
    uint32_t* rank;       // n
    void* pending;        // n / 3 + 1 entries of 16 B
    uint32_t* n_pending;  // 1
    uint32_t* boxes_done; // 1
};
cudaError_t launch_sah_small(const float* lohi, uint32_t n, const uint32_t* codes, uint32_t* perm_out, float4* nodes,
                             uint32_t* parents, uint32_t* ranges, const SahSmallScratch& w, cudaStream_t s);
// Device temporaries of one library call (stream-ordered, freed when the call
// returns); get() reports its own failures.
struct ScratchAlloc {
    rg_status (*get)(void* ctx, void** p, size_t bytes, const char* what);
    void* ctx;
};
// The binned-SAH topology over n triangle boxes: Morton sort into perm, then
// the SAH levels (one host round trip each) and the Karras hierarchy inside
// the remaining segments; children, parents and (optional) leaf ranges as the
// LBVH emits them.
rg_status sah_topology(const ScratchAlloc& tmp, const float* lohi, uint32_t n, const int* cb_ord, int bits,
                       float4* nodes, uint32_t* perm, uint32_t* parents, cudaStream_t s, uint32_t* ranges);
// The same, for 2 <= n <= kSahOneMax and bits 10, without host round trips
// (launch_sah_small); it also writes the node boxes it can, and sets
// *boxes_done (device memory) as launch_sah_small says.
rg_status sah_one_topology(const ScratchAlloc& tmp, const float* lohi, uint32_t n, const int* cb_ord, int bits,
                           float4* nodes, uint32_t* perm, uint32_t* parents, cudaStream_t s, uint32_t* ranges,
                           uint32_t* boxes_done);

// wide.cu
// Collapse a binary LBVH (n leaves) into a compressed 8-wide BVH in one
// single-block launch.  Items are triangles (tris2 -> tris8) or instances
// (inst2 -> inst8, whose BLAS pointers are switched to the wide ones).
// leaf_max (1..kWideLeafMax): a subtree with at most that many items becomes a leaf slot.
cudaError_t launch_collapse(const float4* nodes2, const uint32_t* ranges, uint32_t n, const float* leaf_box,
                            const float4* tris2, float4* tris8, const InstDev* inst2, InstDev* inst8,
                            const BlasDev* blas, const WideOut& out, DevStatus* st, cudaStream_t s,
                            uint32_t leaf_max);
// Re-quantize the wide TLAS after a binary refit and refresh its instance copies.
cudaError_t launch_wide_refit(const float4* nodes2, const float* wbox, const uint32_t* perm, uint32_t n,
                              const InstDev* inst2, InstDev* inst8, const BlasDev* blas, const WideOut& out,
                              DevStatus* st, cudaStream_t s);

// trace.cu
enum TraceMode {
    kModeClosestAbi = 0,
    kModeAnyAbi = 1,
    kModeClosestRender = 2,
    kModeShadowRender = 3,
    kModeClosestBatch = 4,  // like kModeClosestRender, TLAS chosen per ray by the payload's slot
    kModeShadowBatch = 5    // like kModeShadowRender, image chosen per ray by the payload's slot
};
// Launch shape of a traversal (picked by the autotuner): threads per block
// (64, 128 or 256), resident blocks per SM (0: as many as fit), and how many
// lanes of a warp must be idle before the warp fetches new rays (1..32; 32:
// the whole warp; 0: the traversal mode's default).
struct TraceShape {
    int block = 128;
    int blocks_per_sm = 0;
    int refill = 0;
    int stack = 0;  // batched modes at 128 threads: short-stack entries in shared memory (0, 8 or 16)
};
struct TraceArgs {
    const float4* rays;          // n x 2 float4 {o, tmin}, {d, tmax}
    uint32_t n;                  // ray count, or
    const uint32_t* d_count;     // device ray count (if not null)
    const float4* tlas_nodes;
    uint32_t tlas_root;
    const InstDev* inst;
    uint32_t n_inst;
    rg_hit* hits_abi;            // kModeClosestAbi / kModeAnyAbi
    HitDev* hits_render;         // kModeClosestRender
    const Payload* payload;      // kModeShadowRender
    float* image;                // kModeShadowRender: RGBA32F accumulation
    uint32_t* work_counter;      // persistent-thread work queue head (zeroed before launch)
    DevStatus* st;
    uint32_t iter_cap;           // bound on the loop steps of one ray (a valid traversal needs fewer)
    const float4* tlas_nodes8;   // compressed 8-wide TLAS (null: binary path)
    const InstDev* inst8;        // its instances, in wide-leaf order (BLAS pointers to wide BLAS)
    const SlotDev* slots;        // batched modes: request slots
    uint32_t refill;             // binary traversal: idle lanes that make a warp fetch new rays (1..32)
    const uint32_t* ring_head;   // kModeClosestBatch: ray i is ring entry (*ring_head + i) & ring_mask
    uint32_t ring_mask;
    // shadow modes: the rays sit in n_sub sub-queues (one per light) of
    // sub_stride entries, sub_counts[l] rays in sub-queue l (then n, d_count unused)
    const uint32_t* sub_counts;
    uint32_t n_sub, sub_stride;
    // kModeShadowRender: when the queue holds at most split_max rays, each
    // ray is traced as `split` segments of its interval by `split` lanes, and
    // seg_count[i] (zero before the launch) counts ray i's unoccluded
    // segments; null: no splitting
    uint32_t* seg_count;
    uint32_t split, split_max;
    // binary traversal with counting (RG_TRACE_STATS, RG_SCENE_COUNT): stack
    // entries a ray may use (0: all kTraceStack); a smaller limit only makes
    // failure-path tests reach RG_ERR_STACK
    uint32_t stack_max;
};
constexpr uint32_t kTraceStack = 64;  // binary traversal stack entries per thread

constexpr uint32_t kMaxLights = 64;  // lights per scene (one shadow sub-queue each)
cudaError_t launch_trace(int mode, bool brute, bool stats, const TraceArgs& a, cudaStream_t s,
                         const TraceShape& shape = TraceShape());
// Completes the provisional hit records that a closest-hit ABI traversal
// (kModeClosestAbi) wrote: exact t, u, v of the chosen triangle and the tie
// decision.
// Records carry (instance index, prim) of the best and the runner-up; the
// binary TLAS's instances (inst, TLAS leaf order, with leaf_of_inst mapping an
// instance index to its leaf) and the BLAS table locate them.
cudaError_t launch_refine_hits(const float4* rays, rg_hit* hits, uint32_t n, const InstDev* inst,
                               const uint32_t* leaf_of_inst, const BlasDev* blas, cudaStream_t s);
// The shadow rays of sa and the closest-hit rays of ca in one launch
// (kModeShadowRender + kModeClosestRender, or with batch the two batched
// modes, whose launch takes shape.block and shape.blocks_per_sm);
// sa.work_counter serves both.  Binary BVH only.
cudaError_t launch_trace_pair(bool batch, bool stats, const TraceArgs& sa, const TraceArgs& ca, cudaStream_t s,
                              const TraceShape& shape = TraceShape());

// render.cu
struct CameraDev {
    float eye[3], target[3], up[3], vfov_deg;
};
struct ShadeArgs {
    const float4* rays;
    const Payload* payload;
    const HitDev* hits;
    const uint32_t* d_count;     // rays in this wavefront
    const InstDev* inst;
    const rg_material* mats;
    uint32_t n_mats;
    const rg_light* lights;
    uint32_t n_lights;
    float bg[3];
    float ambient;
    uint32_t depth, max_depth;
    float* image;
    float4* next_rays;
    Payload* next_payload;
    uint32_t* next_count;
    float4* shadow_rays;         // one sub-queue of shadow_stride rays per light
    Payload* shadow_payload;
    uint32_t* shadow_count;      // per light
    uint32_t shadow_stride;
    uint32_t max_lights;         // batched: lights of the scene with the most (loop bound)
    DevStatus* st;
    // batched wavefront only: ray i is ring entry (*ring_head + i) & ring_mask,
    // spawned path rays go to ring entries from *next_base, and each ray adds
    // (path rays spawned - 1) to the live count of its slot
    const SlotDev* slots;
    int* slot_live;
    const uint32_t* ring_head;
    const uint32_t* next_base;
    uint32_t ring_mask;
};
cudaError_t launch_raygen(const CameraDev& cam, uint32_t w, uint32_t h, float4* rays, Payload* payload,
                          cudaStream_t s);
cudaError_t launch_shade(const ShadeArgs& a, uint32_t n_max, cudaStream_t s);
// Batched wavefront: primary rays of newly admitted requests, written to ring
// entries (*gen_base + req[k].offset + pixel) & ring_mask for request k; each
// pixel of the request's image is cleared on the way.
struct RaygenReq {
    CameraDev cam;
    uint32_t w, h, slot, offset;
    float* image;
};
cudaError_t launch_raygen_batch(const RaygenReq* reqs, const uint32_t* n_reqs, uint32_t max_rays,
                                const uint32_t* n_rays, const uint32_t* gen_base, uint32_t ring_mask, float4* rays,
                                Payload* payload, cudaStream_t s);
// Shading of a mixed queue: count read on the device (*a.d_count), per-ray
// slot, depth and pixel from the payload, per-slot tables from a.slots.
cudaError_t launch_shade_batch(const ShadeArgs& a, cudaStream_t s);
// FXAA of a w x h RGBA32F image into out (out-of-place); lum: w*h floats of
// scratch (the luma image).
cudaError_t launch_fxaa(const float4* in, uint32_t w, uint32_t h, float* lum, float4* out, cudaStream_t s);

int device_sm_count();

// Record `msg` as this thread's rg_last_error() and return `code`.
rg_status report_error(rg_status code, const char* msg);

// Read-only view of a built scene (api.cu), for the serving loop.
struct SceneView {
    int device;
    const BlasDev* d_blas;
    uint32_t n_blas;
    const float4* tlas_nodes;   // binary TLAS (n_inst - 1 nodes)
    const uint32_t* perm;       // TLAS leaf -> instance index
    const uint32_t* parents;
    const InstDev* inst;        // instances in TLAS leaf order
    uint32_t n_inst, tlas_root;
    const rg_material* mats;
    uint32_t n_mats;
    const rg_light* lights;
    uint32_t n_lights;
    float bg[3];
    float ambient;
    uint32_t iter_cap;
};
rg_status scene_view(rg_scene* s, SceneView* v);

}  // namespace rg
