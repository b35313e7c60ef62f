/*
 * rg.h -- C ABI of the GB300 ray tracer (librg.so).
 *
 * The method is the two-step ray tracing model of "Running on Raygun"
 * (Hirsch & Thoman, Sec. 1): first a two-layered acceleration structure is
 * built from the models' vertices and their transformation matrices (here:
 * one bottom-level BVH per mesh, rg_blas_build, and a top-level BVH over
 * transformed instances, rg_tlas_build / rg_tlas_refit); then rays are
 * dispatched, and per ray a closest-hit, any-hit or miss result is produced
 * (rg_trace_rays).  rg_render runs the paper's Whitted-style renderer on top
 * (Sec. 2.1: multiple objects, shadow casting, reflection and refraction;
 * Sec. 1: recursion to a fixed depth, per-ray payload).
 *
 * Conventions shared by every call:
 *  - Every call returns rg_status (RG_OK = 0).  On failure the call leaves
 *    its outputs unspecified and rg_last_error() returns a message for the
 *    calling thread.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work is asynchronous on it.  Errors detected by a
 *    kernel (stack overflow, iteration cap, singular transform) are recorded
 *    in the scene and returned by the next rg_sync() on that scene.
 *  - Pointers named d_* are device pointers, h_* are host pointers.  The
 *    caller owns every buffer it passes; the library never frees them and
 *    keeps no pointer to them after the call returns (rg_blas_build copies
 *    the geometry it needs).  The library owns the acceleration structures,
 *    ray queues and counters it allocates; rg_scene_destroy frees them.
 *  - All device geometry is float32.  float64 is used on the device only to
 *    invert instance transforms.
 *  - Calls on one scene must not run concurrently from several host threads.
 *  - A scene lives on the CUDA device that was current when it was created.
 *    Every call on it makes that device current for the calling thread (and
 *    leaves it current); the device buffers and the stream passed to it must
 *    belong to that device.
 */
#ifndef RG_H
#define RG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rg_status;
enum {
    RG_OK = 0,
    RG_ERR_INVALID_ARG = 1, /* bad pointer, size, id or flag */
    RG_ERR_OOM = 2,         /* device allocation failed */
    RG_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    RG_ERR_NOT_BUILT = 4,   /* trace/render/refit before rg_tlas_build */
    RG_ERR_STACK = 5,       /* traversal stack overflow (ray abandoned as a miss) */
    RG_ERR_TIMEOUT = 6,     /* a device loop hit its iteration cap */
    RG_ERR_SINGULAR = 7     /* an instance transform is not invertible */
};

typedef struct rg_scene rg_scene;

/* A ray: origin, parametric interval [tmin, tmax] (closed), direction.  The
 * direction need not be unit length; t is measured in units of |d|.  32 B. */
typedef struct { float o[3]; float tmin; float d[3]; float tmax; } rg_ray;

/* A hit record, 20 B.  instance = index into the array given to
 * rg_tlas_build; prim = triangle index within that instance's mesh; t the
 * ray parameter; u, v the barycentric weights of the triangle's second and
 * third vertex (the first has 1-u-v).  Miss: instance = prim = 0xFFFFFFFF,
 * t = +inf, u = v = 0. */
typedef struct { uint32_t instance, prim; float t, u, v; } rg_hit;

/* An instance: row-major 3x4 object-to-world matrix [A | t] applied as
 * world = A * object + t; the mesh (BLAS id) it places; its material; mask is
 * reserved (ignored). 64 B. */
typedef struct { float m[3][4]; uint32_t blas_id, material_id, mask, pad; } rg_instance;

/* Pinhole camera: vertical field of view in degrees, aspect = w/h. */
typedef struct { float eye[3], target[3], up[3], vfov_deg; } rg_camera;

enum { RG_MAT_DIFFUSE = 0, RG_MAT_MIRROR = 1, RG_MAT_GLASS = 2 };
/* Material: diffuse albedo / mirror tint; glass uses ior (tint ignored). */
typedef struct { uint32_t type; float albedo[3]; float ior; float pad[3]; } rg_material;

/* Point light: position and RGB intensity (no distance falloff). */
typedef struct { float pos[3]; float intensity[3]; } rg_light;

/* Scene-wide shading constants.  flags: RG_SCENE_TIMING records CUDA events
 * around every traversal launch; RG_SCENE_COUNT makes rg_render's traversals
 * count node visits, triangle tests and instance entries (slower; see
 * rg_get_stats); RG_SCENE_COMPRESSED builds, next to every binary BVH, a
 * compressed 8-wide BVH whose child boxes are 8-bit integers against a
 * float32 parent origin and per-axis power-of-two scale, rounded outward (80 B
 * per 8 children instead of 64 B per 2), and traces and renders with it; hit
 * records are bit-identical to the binary float32 path.  rg_render traces
 * each depth level's shadow rays and the next level's closest-hit rays in one
 * launch (binary BVH); RG_SCENE_NO_PAIR makes them two launches.
 * RG_SCENE_FRUGAL sizes rg_render's queues from each depth level's ray count
 * (the host waits once per level) instead of the frame's worst case.
 * RG_SCENE_SAH_TLAS builds a TLAS of 2 to 4,096 instances for trace speed:
 * the hierarchy of rg_blas_build's RG_BLAS_SAH, built in one single-block
 * launch without host round trips (larger TLAS keep the LBVH); the same hit
 * records, a slower build. */
enum {
    RG_SCENE_TIMING = 1u,
    RG_SCENE_COUNT = 2u,
    RG_SCENE_COMPRESSED = 4u,
    RG_SCENE_NO_PAIR = 8u,
    RG_SCENE_FRUGAL = 16u,
    RG_SCENE_SAH_TLAS = 32u
};
typedef struct { float background[3]; float ambient; uint32_t flags; } rg_scene_desc;

/* Counters since the last rg_reset_stats. */
typedef struct {
    uint64_t closest_rays;    /* rays traced by closest-hit traversal */
    uint64_t shadow_rays;     /* rays traced by any-hit traversal */
    uint64_t trace_launches;  /* timed closest-hit traversal launches */
    double trace_ms;          /* summed device time of those launches (RG_SCENE_TIMING) */
    uint64_t any_launches;    /* timed any-hit traversal launches */
    double any_ms;            /* summed device time of those launches */
    uint64_t node_visits;     /* counting traversals only (RG_TRACE_STATS, RG_SCENE_COUNT), */
    uint64_t tri_tests;       /*   closest-hit: BVH nodes fetched, triangles tested, */
    uint64_t inst_entries;    /*   instance (BLAS) entries */
    uint64_t any_node_visits; /*   the same for any-hit traversals */
    uint64_t any_tri_tests;
    uint64_t any_inst_entries;
    uint64_t kernel_launches; /* kernels launched by the library (all scenes of the process) */
    uint64_t pair_launches;   /* timed launches that trace one level's shadow rays together with */
    double pair_ms;           /*   the next level's closest-hit rays, and their summed device time */
    uint64_t refine_launches; /* timed launches that complete rg_trace_rays' hit records (exact t, u, v */
    double refine_ms;         /*   and tie decisions), and their summed device time */
} rg_stats;

/* ---- scene lifetime ---------------------------------------------------- */

/* Create an empty scene on the current CUDA device.  desc may be NULL
 * (background (0.2,0.3,0.5), ambient 0.1, no flags). */
rg_status rg_scene_create(rg_scene** out, const rg_scene_desc* desc);
/* A new scene on src's device that shares src's BLAS (by reference: they
 * stay allocated until the last scene holding them is destroyed) and starts
 * with a copy of src's description, materials and lights; its TLAS, queues,
 * counters and statistics are its own.  Renders of the two scenes on
 * different streams may run at the same time, e.g. two frames in flight,
 * each with its own instance transforms.  Once shared, neither scene can
 * build another BLAS (RG_ERR_INVALID_ARG). */
rg_status rg_scene_create_shared(rg_scene** out, rg_scene* src);
/* Free every device allocation of the scene (synchronises the device); BLAS
 * shared with another scene stay until the last of them is destroyed. */
rg_status rg_scene_destroy(rg_scene* scene);

/* ---- step 1 of the paper's model: the two-layered structure (Sec. 1) ---- */

enum { RG_MORTON30 = 0u, RG_MORTON63 = 1u, RG_COMPRESSED = 2u, RG_BLAS_SAH = 4u };
/* Largest number of triangles in one leaf slot of the wide BLAS (1..3;
 * default 2), as a flag of rg_blas_build.  (TLAS leaf slots hold one
 * instance each.) */
#define RG_WIDE_LEAF(n) ((uint32_t)(n) << 8)
/* Bottom-level BVH of one triangle mesh (LBVH: Morton codes of triangle
 * centroids, radix sort, Karras hierarchy, atomic bottom-up box refit).
 * d_vtx: nv x float3 (12 B each); d_idx: nt x uint3 vertex indices (CCW =
 * outward).  flags: RG_MORTON30 (10 bits/axis, u32 keys) or RG_MORTON63 (21
 * bits/axis, u64 keys), plus RG_COMPRESSED to also build the compressed
 * 8-wide BVH (always built in an RG_SCENE_COMPRESSED scene), plus
 * RG_BLAS_SAH to build for trace speed rather than build speed: every split
 * is chosen by the binned surface-area heuristic (16 bins per axis; below 40
 * levels the Karras hierarchy of the Morton codes takes over); same node
 * layout, any query gives the same results, and the build takes one host
 * round trip per tree level.  Writes the new
 * BLAS id to *blas_id.  nt >= 1;
 * indices must be < nv (checked on the device: RG_ERR_INVALID_ARG at
 * rg_sync).  The mesh is copied; d_vtx/d_idx may be freed after the call
 * once the stream has passed it. */
rg_status rg_blas_build(rg_scene* scene, const float* d_vtx, uint32_t nv, const uint32_t* d_idx, uint32_t nt,
                        uint32_t flags, uint32_t* blas_id, void* stream);

/* Top-level BVH over n instances (device array of rg_instance).  Inverts
 * every transform in float64 (RG_ERR_SINGULAR at rg_sync if |det| is 0),
 * bounds each instance with Arvo's method in outward-rounded float32, and
 * builds an LBVH over the instance boxes (30-bit Morton). */
rg_status rg_tlas_build(rg_scene* scene, const rg_instance* d_inst, uint32_t n, void* stream);

/* Update the instance transforms of the last rg_tlas_build (the
 * "update" mode of an acceleration structure): same n (checked on the host,
 * RG_ERR_INVALID_ARG) and the same blas_id per instance (checked on the
 * device, RG_ERR_INVALID_ARG at rg_sync).  Recomputes the instance inverses
 * and boxes and the node boxes; the topology is unchanged. */
rg_status rg_tlas_refit(rg_scene* scene, const rg_instance* d_inst, uint32_t n, void* stream);

/* Shading tables of the renderer (Sec. 2.1: the render system shows multiple
 * objects with shadow casting, reflection and refraction; the materials say
 * which surface reflects or refracts, the lights which shadows are cast).
 * Materials: host array, copied.  Point lights: host array, copied; at most
 * 64, else RG_ERR_INVALID_ARG. */
rg_status rg_scene_set_materials(rg_scene* scene, const rg_material* h_mat, uint32_t n);
rg_status rg_scene_set_lights(rg_scene* scene, const rg_light* h_lights, uint32_t n);

/* ---- step 2: dispatch rays (Sec. 1) ------------------------------------ */

enum {
    RG_CLOSEST = 0u,       /* nearest hit in [tmin, tmax]; ties: smaller instance, then smaller prim */
    RG_ANY = 1u,           /* any hit in [tmin, tmax] (shadow query); record of some hit or a miss */
    RG_TRACE_BRUTE = 2u,   /* test every triangle of every instance (no BVH); for validation */
    RG_TRACE_STATS = 4u,   /* count node visits / triangle tests into rg_stats (slower) */
    RG_TRACE_PLAIN = 8u    /* in an RG_SCENE_COMPRESSED scene: use the binary float32 BVH */
};
/* Trace n rays (device array d_rays) and write n hit records to d_hits.
 * n may be 0.  Closest hit: the nearest triangle is chosen by a float32
 * traversal; a second pass then recomputes t, u, v of that triangle in
 * float-float arithmetic (about 44 bits) from the float32 inputs, so they are
 * the exact values rounded to float32 up to a few units in the last place
 * (far inside 1e-5 relative, also for small triangles seen from afar), and
 * t is kept within [tmin, tmax].  When the float32 distances of the two
 * nearest candidates lie within a relative 2^-14, the two are decided again
 * on their exact distances rounded to float32 (then instance, then prim), so
 * exact ties such as coplanar surfaces have one answer.  Any hit: only
 * occluded / not is defined; the record of some hit carries the float32 t,
 * u, v of the watertight test.  Calls on one scene from one host thread may
 * run at the same time on different streams (each takes a work counter of its
 * own; at most 64 calls in flight), provided no rg_tlas_build or
 * rg_tlas_refit of the scene runs meanwhile. */
rg_status rg_trace_rays(rg_scene* scene, const rg_ray* d_rays, uint32_t n, uint32_t flags, rg_hit* d_hits,
                        void* stream);

/* Whitted render into d_rgba (w*h*4 float32, row 0 = top, RGB linear
 * radiance, A = 1 where the primary ray hit).  Primary rays through pixel
 * centres; diffuse: ambient + unshadowed Lambert per light; mirror: tinted
 * reflection; glass: Schlick-weighted reflection + refraction (total internal
 * reflection beyond the critical angle); misses: background.  Reflection and
 * refraction rays are spawned while the ray depth (primary = 1) is below
 * max_depth.  Asynchronous on `stream`: the scene's queues are sized once
 * for the frame's worst case (level d holds at most w h 2^(d-1) rays) when
 * that takes at most 16 GB, and every launch reads its ray count on the
 * device, so the call returns without waiting for the GPU; beyond that size
 * the host waits once per depth level to size the next queues.  Renders of
 * one scene on different streams must not overlap (its queues are shared);
 * scenes made with rg_scene_create_shared may render concurrently. */
rg_status rg_render(rg_scene* scene, const rg_camera* h_cam, uint32_t w, uint32_t h, uint32_t max_depth,
                    float* d_rgba, void* stream);

/* FXAA (Sec. 2.1: the engine's compute passes include fast approximate
 * anti-aliasing; the method is Lottes' FXAA, 2009) of a w x h RGBA32F image,
 * row 0 at the top, into d_out (same layout, must not alias d_in; both
 * 16-byte aligned).  Per pixel, float32: gamma-2 luma; pixels whose local
 * luma range is below max(0.0312, 0.125 x local max) are copied; otherwise
 * the edge orientation, the side of the edge and its two ends (searched up
 * to 26.5 pixels each way) give an offset across the edge, at least the
 * sub-pixel offset 0.75 s^2 of the 3x3 contrast, and the colour is
 * resampled bilinearly there (clamp-to-edge); alpha is copied.  Needs no
 * scene; w or h = 0 does nothing.  Takes w*h*4 bytes of stream-ordered
 * temporary device memory (the luma image) for the duration of the call. */
rg_status rg_fxaa(const float* d_in, uint32_t w, uint32_t h, float* d_out, void* stream);

/* rg_sync waits for all of the device's work and returns the first error a
 * kernel of this scene recorded since the last rg_sync (RG_ERR_STACK,
 * RG_ERR_TIMEOUT, RG_ERR_SINGULAR, RG_ERR_INVALID_ARG for a bad index found on
 * the device), clearing it; the rays concerned came back as misses and the
 * scene stays usable.  rg_get_stats waits for the device and fills *out with
 * the counters since the last rg_reset_stats (rays traced, timed launches and
 * their device time with RG_SCENE_TIMING, node / triangle / instance counts of
 * counting traversals); rg_reset_stats waits and zeroes them.  RG_ERR_INVALID_ARG
 * for a NULL scene or output. */
rg_status rg_sync(rg_scene* scene);
rg_status rg_get_stats(rg_scene* scene, rg_stats* out);
rg_status rg_reset_stats(rg_scene* scene);
/* Message of the last failed call on this thread ("" if none). */
const char* rg_last_error(void);

/* ---- the build steps, exposed one by one (for validation) -------------- */

/* Per-triangle box: d_lohi[6*i] = {lo.xyz, hi.xyz}, exact float32 min/max of
 * the triangle's vertices. */
rg_status rg_tri_bounds(const float* d_vtx, uint32_t nv, const uint32_t* d_idx, uint32_t nt, float* d_lohi,
                        void* stream);
/* Morton code of each box centroid c = (lo+hi)*0.5 on one cubic grid: a single
 * scale s = 2^b / max over the axes of (cmax-cmin) (q = 0 on an axis with
 * cmax == cmin), q = clamp(floor((c-cmin)*s), 0, 2^b-1), bits interleaved x
 * (most significant), y, z.  bits = 10 writes uint32 codes,
 * bits = 21 uint64 codes.  d_cbounds (6 floats, may be NULL) receives the
 * centroid bounds {cmin.xyz, cmax.xyz}. */
rg_status rg_morton_codes(const float* d_lohi, uint32_t n, uint32_t bits, void* d_codes, float* d_cbounds,
                          void* stream);
/* Stable LSD radix sort (8-bit digits) of (key, value) pairs; key_bits = 32
 * (uint32 keys, 4 passes) or 64 (uint64 keys, 8 passes).  Inputs are not
 * modified.  Allocates temporary device memory on the stream. */
rg_status rg_radix_sort_pairs(const void* d_keys, const uint32_t* d_vals, uint32_t n, uint32_t key_bits,
                              void* d_keys_out, uint32_t* d_vals_out, void* stream);
/* Binary radix tree over n >= 2 sorted keys (Karras 2012, Sec. 4): for internal
 * node i (root 0) writes d_children[2i] / [2i+1]; a child with bit 31 set is
 * leaf (child & 0x7FFFFFFF), else internal node `child`.  d_parents (2n-1,
 * may be NULL): parent of internal node i at [i], of leaf j at [n-1+j]; the
 * root's parent is 0xFFFFFFFF. */
rg_status rg_karras(const void* d_sorted_keys, uint32_t n, uint32_t key_bits, uint32_t* d_children,
                    uint32_t* d_parents, void* stream);

/* Copy a built BLAS to host memory: h_nodes (nt-1) x 64 B nodes (float
 * lo0[3], hi0[3], lo1[3], hi1[3], uint32 child0, child1, 2 x pad), h_tris
 * nt x 48 B triangles in leaf order (v0.xyz, uint32 prim; v1.xyz, pad;
 * v2.xyz, pad), *h_root the root reference (leaf refs have bit 31 set).
 * Any output may be NULL.  Synchronises the device. */
rg_status rg_blas_export(rg_scene* scene, uint32_t blas_id, void* h_nodes, void* h_tris, uint32_t* h_root);
/* Copy the TLAS: h_nodes (n-1) x 64 B, h_wbox n x 6 floats (world box of
 * instance i, in input order), h_inv n x 12 floats (float32 world-to-object
 * 3x4 of instance i, input order), h_order n uint32 (input index of TLAS
 * leaf j), *h_root.  Any output may be NULL.  Synchronises the device. */
rg_status rg_tlas_export(rg_scene* scene, void* h_nodes, float* h_wbox, float* h_inv, uint32_t* h_order,
                         uint32_t* h_root);

/* Copy a compressed 8-wide BVH to host memory (blas_id, or RG_TLAS_ID for the
 * TLAS): h_counts[0] = nodes, [1] = items; h_nodes 80 B per node (layout in
 * csrc/rg_internal.cuh); h_src 8 uint32 per node, the binary-BVH reference of
 * each child slot (0xFFFFFFFF if empty; bit 31 = binary leaf); h_item_src one
 * uint32 per item, the binary leaf it copies.  Buffers must hold max(n-1,1)
 * nodes and n items for an n-leaf tree.  Any output may be NULL.
 * Synchronises the device.  RG_ERR_NOT_BUILT if that BVH has no wide form. */
#define RG_TLAS_ID 0xFFFFFFFFu
rg_status rg_wide_export(rg_scene* scene, uint32_t blas_id, void* h_nodes, uint32_t* h_src, uint32_t* h_item_src,
                         uint32_t* h_counts);

/* ---- sorting without allocation ---------------------------------------- */

/* The paper has no counterpart to this call; it is a service of the library.
 * Same result as rg_radix_sort_pairs (same arguments and order), but the call
 * makes no device allocation: its temporaries live in one fixed array inside
 * librg.so, sized for RG_NOALLOC_SORT_MAX_PAIRS pairs of 64-bit keys (about
 * 3.2 MB, held on every GPU that loads the library until the process exits).
 * It is meant for callers that cannot allocate device memory: code whose
 * device memory is owned by a caching allocator that has already reserved
 * what the GPU has free, and frame loops that must not stall on an
 * allocation.  The caller still provides inputs and outputs (d_keys_out and
 * d_vals_out hold n elements each, on the current device).
 *  - n > RG_NOALLOC_SORT_MAX_PAIRS returns RG_ERR_INVALID_ARG.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and keeps it for the process; make that first
 *    call before any stream capture.  The address is not looked up again
 *    after cudaDeviceReset.
 *  - All calls share the array and it keeps the last call's contents (every
 *    byte a call reads there it wrote first): calls whose GPU work overlaps
 *    (other streams, other host threads) race and must be serialised. */
#define RG_NOALLOC_SORT_MAX_PAIRS 262144u
rg_status rg_radix_sort_pairs_noalloc(const void* d_keys, const uint32_t* d_vals, uint32_t n, uint32_t key_bits,
                                      void* d_keys_out, uint32_t* d_vals_out, void* stream);

/* ---- continuous-batching render server --------------------------------- */

/* Serving many render requests at once over resident scenes.  The paper
 * renders one frame per dispatch (Sec. 1: a scene is set up, then rays are
 * dispatched and recursively traced); the server keeps that per-ray work and
 * batches it: the path rays (primary, reflected, refracted) of every request
 * in flight share one ring of rays; each rg_server_step traces and shades a
 * batch of them and appends the rays it spawns; the shadow rays the shading
 * spawns are traced by the next step, in one launch with its closest-hit
 * rays (RG_SERVER_NO_PAIR: by the same step, after shading), so a request
 * completes one step after its last path ray (an otherwise idle step traces
 * only those shadow rays).  Requests of different scenes, resolutions
 * and depths are traced in the same launches.  Requests join as earlier ones
 * complete (continuous batching).  Each request carries its own instance
 * transforms: on admission the server refits a private copy of the scene's
 * TLAS with them (same topology, new boxes), so the images equal those of
 * rg_tlas_refit + rg_render of the request alone, up to the order of the
 * float additions into a pixel.
 *
 * Admission is by free ring memory: a request of w*h pixels is admitted, in
 * arrival order, when a request slot is free (at most RG_SERVER_MAX_SLOTS in
 * flight) and the rays in the ring plus its w*h primary rays fit in the
 * admission bound (admit_rays, by default one batch; at most half the ring:
 * the other half takes the rays steps spawn, at most two per traced ray).  A
 * request larger than the bound is admitted alone, into an empty ring.  A step traces up to min(batch_rays, shadow capacity / max lights)
 * rays, oldest first, as many as the free ring takes in the worst case.  When
 * that is under a quarter of a batch (glass doubling the rays of deep ray
 * trees), steps take the newest rays instead (the deepest: the trees are then
 * finished depth first, which bounds the live rays), a batch of at most
 * free ring / (2 (RG_SERVER_MAX_DEPTH + 1)).  RG_ERR_OOM only if even that is
 * zero.
 *
 * The server holds one or more lanes (rg_server_desc.lanes): independent
 * rings, each with its own shadow and hit queues, request slots and stream.
 * A request is admitted to the least loaded lane and stays there; a step
 * runs one step of every lane with work, at the same time, so the idle tails
 * of one lane's launches are filled by the others'.  Every lane's step is
 * one CUDA graph on the lane's stream (captured on first use, re-captured
 * when buffers or launch shapes change); a lane takes new requests and
 * starts its next step only once its step in flight has been booked.  Calls
 * on one server must not run concurrently. */
typedef struct rg_server rg_server;

#define RG_SERVER_MAX_SLOTS 32u
#define RG_SERVER_MAX_PIXELS (1u << 23)   /* w*h of one request */
#define RG_SERVER_MAX_DEPTH 15u

typedef struct {
    uint32_t ring_log2;   /* the ray ring holds 2^ring_log2 rays (48 B each); 0 = 2^25; 16..30 */
    uint32_t batch_rays;  /* rays traced per step at most; 0 = 2^23 */
    uint32_t max_lights;  /* shadow queue = batch_rays * max_lights rays (48 B each); 0 = 4; scenes with
                             more lights are refused */
    uint32_t flags;       /* RG_SERVER_NO_GRAPH: launch each step's kernels directly, no CUDA graph;
                             RG_SERVER_NO_PAIR: trace a step's shadow rays in the step, after shading
                             (default: in the next step, one launch with its closest-hit rays, using
                             the closest-hit shape; a request then completes one step later) */
    uint32_t admit_rays;  /* admission bound on the rays in the ring plus a new request's primary rays;
                             0 = batch_rays (what one step can take); at most half the ring.  A
                             smaller bound keeps fewer requests in flight: large requests run closer
                             to one after another (shorter tail latency), small ones still share steps */
    uint32_t lanes;       /* independent rings (each with its own queues, request slots and stream) whose
                             steps run at the same time; a request lives in one lane, admitted to the
                             least loaded; 0 = 1; at most RG_SERVER_MAX_LANES.  Every lane holds a ring,
                             a shadow queue and a hit queue of the sizes above */
} rg_server_desc;
#define RG_SERVER_MAX_LANES 8u
#define RG_SERVER_NO_GRAPH 1u
#define RG_SERVER_NO_PAIR 2u

/* One render request.  h_transforms: n_inst 3x4 row-major object-to-world
 * matrices (12 floats each) in the order of the scene's rg_tlas_build, or
 * NULL for the scene's own; copied at submission.  d_rgba: caller-owned
 * device image of w*h RGBA32F (row 0 at the top), written by the server from
 * admission to completion; the caller keeps it alive until then. */
typedef struct {
    uint32_t scene;        /* id from rg_server_add_scene */
    rg_camera camera;
    uint32_t width, height; /* 1 <= w*h <= RG_SERVER_MAX_PIXELS, and w*h <= 2^(ring_log2-1) */
    uint32_t max_depth;     /* 1..RG_SERVER_MAX_DEPTH */
    const float* h_transforms;
    float* d_rgba;
    uint64_t tag;           /* returned with the completion */
} rg_request;

typedef struct {
    uint64_t id;          /* from rg_server_submit */
    uint64_t tag;
    uint32_t admitted_step, completed_step; /* step numbers (1-based) */
} rg_completion;

typedef struct {
    uint64_t steps, submitted, admitted, completed;
    uint64_t closest_rays, shadow_rays;     /* traced so far */
    uint32_t pending, active;               /* waiting for admission / in flight */
    uint32_t ring_rays, ring_peak;          /* rays in the ring now / at most so far */
    uint64_t graph_launches, graph_captures;
    uint64_t kernel_launches;               /* kernels launched by the server's steps (graph kernels included) */
    uint64_t newest_first_steps;            /* steps that took the newest rays (ring nearly full) */
    uint64_t lane_steps;                    /* steps of the individual lanes (a server step runs those of
                                               every lane with work) */
} rg_server_stats;

/* Creates a server on the current device (desc NULL: defaults).  Allocates the
 * ring, the hit and shadow queues and the per-slot buffers up front. */
rg_status rg_server_create(rg_server** out, const rg_server_desc* desc);
rg_status rg_server_destroy(rg_server* server);
/* Makes a built scene (rg_tlas_build and rg_scene_set_materials done)
 * available to requests; the scene must stay alive and must not be rebuilt
 * (rg_blas_build, rg_tlas_build) or destroyed while the server exists.  The
 * server traces the scene's binary float32 BVH, also for a scene made with
 * RG_SCENE_COMPRESSED (its hit records are the same in both forms).  Returns
 * RG_ERR_INVALID_ARG for a foreign-device scene or one with more lights than
 * max_lights. */
rg_status rg_server_add_scene(rg_server* server, rg_scene* scene, uint32_t* scene_id);
/* Queues a request; validated here (RG_ERR_INVALID_ARG on a bad size, depth,
 * scene id or pointer). */
rg_status rg_server_submit(rg_server* server, const rg_request* req, uint64_t* request_id);
/* One step: admits what fits into the idle lanes, refits the admitted
 * requests' TLAS copies, launches a step (trace and shade one batch) on every
 * idle lane with work, each on its own stream, and returns once at least one
 * lane's step has finished (the oldest launched is waited for; every finished
 * one is booked); the other lanes' steps run on and are booked by later
 * calls (rg_server_drain waits for all).  *n_completed (may be NULL)
 * = requests completed by this step; their images are final.  With nothing
 * queued or in flight the step does nothing.  Device errors (stack overflow,
 * iteration cap, singular transform, bad material) are returned here. */
rg_status rg_server_step(rg_server* server, uint32_t* n_completed);
/* Steps until nothing is queued or in flight. */
rg_status rg_server_drain(rg_server* server);
/* Moves up to `max` completions (oldest first) to out; *n = how many. */
rg_status rg_server_poll(rg_server* server, rg_completion* out, uint32_t max, uint32_t* n);
rg_status rg_server_get_stats(rg_server* server, rg_server_stats* out);

/* Launch shapes of the server's two traversals (which: 0 closest hit,
 * 1 shadow): threads per block 64 / 128 / 256, resident blocks per SM
 * (0 = as many as fit), how many of a warp's 32 lanes must have finished
 * their rays before the warp fetches new ones (1..32; 32 = only when all
 * have, a leaner loop; 0 = the default, 32), and the short traversal stack:
 * how many of a thread's stack entries live in shared memory, the rest in
 * local memory (the benchmark spec's short stack; 0, or 8 or 16 with 128 threads per
 * block; else RG_ERR_INVALID_ARG). */
typedef struct { uint32_t block, blocks_per_sm, refill, stack; float ms; } rg_trace_shape;
rg_status rg_server_set_shape(rg_server* server, uint32_t which, const rg_trace_shape* shape);
rg_status rg_server_get_shape(rg_server* server, uint32_t which, rg_trace_shape* out);
/* Autotuner: picks both shapes by timing every candidate (block x blocks per
 * SM x refill x short-stack depth) on the sample request's rays (its primary rays for the closest
 * traversal, the shadow rays their shading spawns for the shadow traversal),
 * sets them, and reports them in out[0..1] (ms = best time of that
 * traversal).  cache_path (may be NULL): a JSON file; if it holds shapes for
 * this device model they are taken without timing (unless flags has
 * RG_TUNE_FORCE), else the tuned shapes are written there.  Runs only on an
 * idle server (nothing queued or in flight: else RG_ERR_INVALID_ARG); the
 * sample's image is overwritten. */
#define RG_TUNE_FORCE 1u
rg_status rg_server_autotune(rg_server* server, const rg_request* sample, const char* cache_path, uint32_t flags,
                             rg_trace_shape out[2]);

#ifdef __cplusplus
}
#endif

#endif /* RG_H */
