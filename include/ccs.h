/*
 * ccs.h -- C ABI of the GB300 (sm_103a) library for closest-hit ray intersection with Catmull-Clark
 * subdivision surfaces given as bicubic Bezier (16 control points) and Gregory (20 control points)
 * patches, after Binder & Keller, "Massively Parallel Stackless Ray Tracing of Catmull-Clark
 * Subdivision Surfaces" (arXiv 1811.03510).
 *
 * Conventions shared by every entry point
 *  - All pointers are plain host or device addresses; no framework types cross this boundary.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is enqueued
 *    asynchronously on it unless the entry point says otherwise; caller-owned device buffers must stay
 *    valid until that work completes.  Launches on one scene may run at the same time on different
 *    streams (each takes its own work-queue head from a ring of 48, and the scratch of the work order
 *    and of the pair engine from a stream-ordered memory pool of the library), except
 *    ccs_intersect_host and ccs_intersect_host_batches calls, which share the scene's staging buffer.
 *  - Every call returns a ccs_status.  On failure, ccs_last_error() returns a message for the calling
 *    thread.  Errors detected on the device (traversal iteration cap reached) are latched in a status
 *    word of the scene and returned by ccs_scene_sync_status().
 *  - Rays and hits are structure-of-arrays float32 / uint32 planes with one element per ray.
 *  - A miss is patch_id = 0xFFFFFFFF, t = +INF, u = v = 0.  Rays with NaN components or tmin > tmax
 *    are misses, not errors.
 *
 * What a hit is (Sec. 3 and Algorithm 3 of the paper): the (u,v) domain of each patch is split
 * alternately along u and v, starting with u, down to leaf cells of 2^-L x 2^-L; a node's box is the
 * AABB of its control points (de Casteljau halves for Bezier patches, Sec. 3.1; the lower bounding
 * patch raised by the displacement d of Algorithm 2 for Gregory patches, Sec. 3.2); a node's ray
 * interval is its box's slab interval intersected with its parent's.  The hit is the leaf with the
 * smallest key (entry distance t, patch id, cell index); u, v are the centre of that leaf cell.
 */
#ifndef CCS_H
#define CCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CCS_OK = 0,
    CCS_ERR_INVALID_ARG = 1,     /* null pointer, size out of range, bad option value */
    CCS_ERR_CUDA = 2,            /* a CUDA runtime call failed; message in ccs_last_error() */
    CCS_ERR_OOM = 3,             /* device or host allocation failed */
    CCS_ERR_TRAVERSAL_LIMIT = 4, /* a ray hit the iteration cap; that ray was written as a miss */
    CCS_ERR_NOT_BUILT = 5        /* intersect called before ccs_bvh_build */
} ccs_status;

typedef enum { CCS_BEZIER = 0, CCS_GREGORY = 1 } ccs_patch_type;

typedef struct ccs_scene ccs_scene;   /* opaque; created and freed by the library */

/* Ray batch: eight caller-owned float32 planes of n elements (device addresses for ccs_intersect,
 * host addresses for ccs_intersect_host).  Directions need not be normalised; t is in units of d. */
typedef struct {
    const float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
} ccs_rays;

/* Hit output: caller-owned planes of n elements. */
typedef struct {
    float *t, *u, *v;
    uint32_t *patch_id;
} ccs_hits;

/* Launch and method options.  Zero-initialised fields take the defaults given in brackets (except
 * cache_slots, whose 0 is meaningful: pass CCS_CACHE_DEFAULT for the default).  Apart from leaf_depth and
 * pixel_spread, which define the hierarchy, none of them changes the answer: hits are bit-identical for
 * every launch configuration. */
typedef struct {
    uint32_t leaf_depth;      /* L, splits per axis of the (u,v) domain, 1..15 [8] */
    uint32_t block_threads;   /* threads per block, multiple of 32, 32..1024 [128] */
    uint32_t blocks_per_sm;   /* blocks per SM of the persistent launch, clamped to what fits [4] */
    uint32_t refill;          /* a warp hands new rays to its idle lanes once at least this many of its
                                 rays are idle, 1..32 [8] */
    uint32_t chunk;           /* rays a warp takes from the global work queue at a time, multiple of 32,
                                 32..4096 [32] */
    uint32_t bvh_burst;       /* BVH steps a traversing lane takes per subdivision step of the others,
                                 1..16 [8] */
    uint32_t cache_slots;     /* grids of pending Bezier siblings kept in shared memory per thread,
                                 0, 1 or 2 [2]; 0 re-derives every sibling by de Casteljau from the root
                                 (the ray-persistent kernel takes 1 as 2) */
    uint32_t min_blocks;      /* 0: kernel compiled for 3 blocks of 128 threads per SM (168 registers);
                                 4: compiled for 4 blocks (128 registers, spills to L1) [0] */
    uint32_t vote;            /* 0: every lane steps every iteration; v > 0: per iteration a warp steps
                                 only its lanes inside a patch while at least v of them are, else only
                                 its lanes traversing the BVH, 0..32 [0] */
    uint32_t lanes_per_ray;   /* 1: a lane holds all three components of its ray, 32 rays per warp;
                                 3: a group of three lanes holds one ray, one component per lane, and
                                 combines the per-axis slab results by shuffles (Sec. 3.5), 10 rays per
                                 warp; refill and vote then count rays, not lanes.  The trace export and
                                 learned entry points use 1 [1] */
    uint32_t iter_cap;        /* per-ray cap on traversal iterations [1 << 22] */
    float pixel_spread;       /* ccs_intersect / ccs_intersect_host: screen-space termination (Sec. 3.3).
                                 0: fixed depth (every leaf at level 2L).  > 0: the rays' angular size of
                                 one pixel in radians (pinhole camera: 2 tan(fov/2) / height); a node made
                                 by a split whose box has an L1 diagonal below pixel_spread / 2 times its
                                 entry distance is a leaf, reported with u, v at its domain's centre and
                                 the cell index of its lowest leaf cell.  Changes the answer (it is a
                                 method parameter, not a launch option); one lane per ray.  [0] */
    uint32_t flags;           /* CCS_TRACE_* bits */
    uint64_t *counters;       /* optional device array of CCS_NUM_COUNTERS uint64 (CCS_TRACE_COUNT) */
    uint32_t image_width;     /* the rays are an image of this width, ray y * width + x (the last row may
                                 be partial).  CCS_TRACE_ORDER: ordered in tiles of 8 x 8 pixels with
                                 every 4th pixel in x and y sampled; 0: tiles of 32 consecutive rays,
                                 every 4th ray sampled.  CCS_TRACE_PAIRS, a multiple of 8: each warp of
                                 the candidate pass takes a tile of 8 x 4 pixels (a host chunk is tiled
                                 from its own first ray); else 32 consecutive rays.  Never changes the
                                 answer [0] */
    uint32_t bvh_width;       /* the scene's BVH to traverse: 0 its default, 2 or 4 (INVALID_ARG when the
                                 scene was not built with that width) [0] */
    uint32_t host_chunk;      /* ccs_intersect_host: rays per chunk of its copy/trace pipeline, at most 8
                                 chunks (larger chunks then); 0: below 2^17 rays (2^19 with the pair
                                 engine) one chunk, else a short first and last chunk (n/8 rays, at most
                                 2^18) around middle chunks of about 2^20 rays [0] */
} ccs_trace_opts;

#define CCS_CACHE_DEFAULT 0xFFFFFFFFu
#define CCS_TRACE_COUNT 1u          /* accumulate traversal counters into opts->counters */
#define CCS_TRACE_HOST_MAPPED 4u    /* ccs_intersect_host: when every plane is mapped page-locked memory,
                                       read rays and write hits through the mapping instead of staging
                                       copies */
#define CCS_TRACE_ORDER 2u          /* work order: before the launch, count for sampled rays the BVH leaf
                                       boxes (candidate patches) they enter within [tmin, tmax]; the work
                                       queue then hands out tiles in descending order of their largest
                                       count (stable within a count, counts clamped to 15), so that the
                                       rays that subdivide most start first and the launch does not end
                                       on a few late, long rays.  Never changes an answer.  Three small
                                       kernels and a permutation of 4 bytes per ray in scratch of the
                                       launch, from a stream-ordered memory pool of the library (kept for
                                       reuse).  Used by ccs_intersect, ccs_intersect_host and
                                       ccs_occluded; the other entry points ignore it, and so does the
                                       pair engine. */
#define CCS_TRACE_PAIRS 8u          /* pair engine, for the plain closest hit and the any-hit query with one
                                       lane per ray (other modes ignore it): (1) one thread per ray walks
                                       the BVH and keeps the ray's 8 nearest candidate patches (by entry
                                       distance of the patch box); with local frames a Bezier patch whose
                                       root box in its own frame the ray does not come near is no
                                       candidate; (2) the rays with candidates are ordered by a cost
                                       class (a Gregory candidate first, then more candidates first);
                                       (3) persistent warps run Algorithm 3 on one (ray, patch) pair per
                                       lane, taking each ray's candidates in entry order until one enters
                                       beyond its best hit, so that every warp iteration is one or two
                                       subdivision steps of up to 32 pairs; once the queue is empty, idle
                                       lanes take pending subtrees of busy lanes of their warp; (4) a ray
                                       whose dropped candidates could still hold the answer has its lane
                                       walk the BVH again for the next ones.  Hits are bit-identical.  Uses
                                       about 200 bytes of scratch per ray from a stream-ordered memory
                                       pool of the library (kept for reuse), on the launch's stream; the
                                       work order, bvh_burst, vote, chunk and min_blocks do not apply, and
                                       blocks_per_sm is what fits.  Counters: slots 8..17 hold candidates
                                       listed, rays that dropped some, walks for dropped candidates,
                                       subtrees handed over, warp iterations of the subdivision pass and,
                                       per iteration, lanes splitting, helping, waiting and idle, then
                                       candidates culled by their root box. */
#define CCS_NUM_COUNTERS 23         /* work per ray, summed (0..7): bvh nodes, bezier splits, gregory
                                       splits, leaves, backtracks, re-descent levels, pruned siblings, pairs;
                                       schedule of the warps, summed over warp iterations (8..19): warp
                                       iterations, resident rays, then for each step kind (subdivision,
                                       Gregory bound, leaf, BVH burst) the rays doing it and the
                                       iterations in which any ray does it (the BVH pair is followed by
                                       the longest burst of the iteration), then warp refills.  The
                                       schedule counts depend on the launch options, the work counts do
                                       not.  Timeline of the launch in device-clock nanoseconds, kept as
                                       maxima (20..22): bitwise NOT of the first warp's start, bitwise
                                       NOT of the time a warp first found the work queue empty, the last
                                       warp's exit; meaningful for one launch per zeroed array. */

typedef struct {
    uint32_t bins;            /* SAH bins per axis, 4..64 [16] */
    uint32_t width;           /* children per node: 2 (the binary BVH of Sec. 4), 4 (the binary tree
                                 collapsed, each node opening its largest child until it holds four
                                 subtrees; a wider BVH is named as future work in Sec. 4), or
                                 CCS_BVH_BOTH (both trees: launches use the binary one unless
                                 opts->bvh_width asks for the other; refits update both).  Does not change
                                 any answer.  A 4-wide tree deeper than 21 levels is refused (INVALID_ARG:
                                 its traversal stack holds 64 entries) [2] */
} ccs_bvh_params;

#define CCS_BVH_BOTH 6u

/* Create a scene from n_patches patches.
 * x, y, z: control points, 20 float32 slots per patch, patch-major: x[20*p + s].  Slots 0..15 are the
 *   4x4 grid, slot 4*j + i with i along u and j along v (corner p_00 at (u,v) = (0,0)).  For Gregory
 *   patches (Sec. 3.2) slots 5, 6, 9, 10 (inner points (1,1), (2,1), (1,2), (2,2)) hold p^u and slots
 *   16..19 hold p^v in the same order; p^u is the point that the v = 0 / v = 1 edges use, i.e. the inner
 *   point is p^v + h (p^u - p^v) with h_11 = u/(u+v), h_21 = (1-u)/((1-u)+v), h_12 = u/(u+1-v),
 *   h_22 = (1-u)/((1-u)+(1-v)) (the convention of Algorithm 2).  Bezier patches ignore slots 16..19.
 * types: n_patches bytes, CCS_BEZIER or CCS_GREGORY.
 * flags: CCS_SCENE_DEVICE_PTRS if x, y, z, types are device addresses (else host addresses);
 *   CCS_SCENE_LOCAL_FRAMES to take the boxes below each patch root in the patch's own frame (Sec. 3.4:
 *   local frames shrink the overlap of the sub-domain boxes): z along the normal of the corner quad (the
 *   cross product of its diagonals p33 - p00 and p03 - p30), x along its u edge p30 - p00 made orthogonal
 *   to z, y = z x x (the world axes where that is degenerate).  The BVH and the patch root interval stay
 *   in world space.  The hits are those of the same method with boxes in these frames.
 * The library copies the data into its own device store (patch records anchored at their box centre,
 * Sec. 3.4); the caller keeps ownership of its arrays.  n_patches may be 0 (every ray misses).
 * Blocks until the copy has finished.  Errors: INVALID_ARG (null pointers, n_patches > 2^26),
 * OOM, CUDA. */
ccs_status ccs_scene_create(ccs_scene **out, const float *x, const float *y, const float *z, const uint8_t *types,
                            uint32_t n_patches, int flags, void *stream);

#define CCS_SCENE_DEVICE_PTRS 1
#define CCS_SCENE_LOCAL_FRAMES 2

/* Replace the control points (same layout, same patch count and types) from device addresses,
 * asynchronously on `stream`; a following ccs_bvh_refit updates the hierarchy, and intersections must
 * wait for it (before the refit, hits are undefined: the patch boxes are new, the BVH's are old).
 * Graph-capturable. */
ccs_status ccs_scene_update_points(ccs_scene *scene, const float *x, const float *y, const float *z, void *stream);

ccs_status ccs_scene_destroy(ccs_scene *scene);

/* BVH over whole-patch boxes (AABB of the 16 or 20 control points; convex hull property, Sec. 3.1),
 * built on the host with binned SAH (Sec. 4), one patch per leaf, binary or collapsed to 4-wide nodes
 * (params->width), and uploaded.  Uses the points given at creation (or copied back after an update).
 * Blocks.  params may be NULL.  Batches need every scene built with one width (not CCS_BVH_BOTH). */
ccs_status ccs_bvh_build(ccs_scene *scene, const ccs_bvh_params *params);

/* Recompute every box of the hierarchy bottom-up from the current control points, keeping its
 * topology.  Asynchronous on `stream`, graph-capturable. */
ccs_status ccs_bvh_refit(ccs_scene *scene, void *stream);

/* Closest hit of n rays (Algorithm 3 per candidate patch of a BVH traversal; see the file comment for
 * the exact answer).  rays, hits: device addresses, caller-owned.  opts may be NULL (defaults).
 * Asynchronous on `stream`.  n may be 0.  Errors: INVALID_ARG, NOT_BUILT, CUDA. */
ccs_status ccs_intersect(const ccs_scene *scene, const ccs_rays *rays, uint32_t n, ccs_hits *hits,
                         const ccs_trace_opts *opts, void *stream);

/* Same answer as ccs_intersect, for rays and hits in host memory.  The rays are copied to a device
 * staging buffer owned by the scene in chunks (opts->host_chunk; at most 8).  Chunk k is traced while chunk k+1 is copied in and chunk k-1's hits are copied out, on
 * streams the scene owns and orders after the work already on `stream`.  Planes that are rows of one
 * host block (equally spaced, in the order of the struct) move as one 2D copy per chunk; other planes
 * take one copy each.  With CCS_TRACE_HOST_MAPPED, when every plane is page-locked memory mapped into the
 * device (cudaHostAlloc / cudaHostRegister; both ends of each plane are checked with
 * cudaPointerGetAttributes), the launch instead reads the rays and writes the hits through that
 * mapping: one launch, no staging (on Grace systems over NVLink-C2C).  Synchronises `stream` before
 * returning.  Not thread-safe per scene (one staging
 * buffer); not graph-capturable.  Errors: INVALID_ARG, NOT_BUILT, OOM, CUDA. */
ccs_status ccs_intersect_host(ccs_scene *scene, const ccs_rays *host_rays, uint32_t n, ccs_hits *host_hits,
                              const ccs_trace_opts *opts, void *stream);

/* Several batches of host rays through one copy/trace pipeline: batch j has n[j] rays in host_rays[j],
 * its hits go to host_hits[j], traced with opts[j] (opts or opts[j] may be NULL: defaults; each batch
 * may have its own work order, BVH width or chunk size).  The answers are those of ccs_intersect_host
 * called for each batch in turn; the difference is that batch j+1's copies and launches start while
 * batch j's last chunks are traced and copied out, instead of after the call returns.  Every batch is
 * checked before anything is queued.  Batches always take the staged copies (CCS_TRACE_HOST_MAPPED is
 * ignored here); the staging buffer holds all batches at once (12 floats per ray).  Synchronises
 * `stream` before returning.  Not thread-safe per scene; not graph-capturable.  n_batches may be 0, and
 * any n[j] may be 0.  Errors: INVALID_ARG, NOT_BUILT, OOM, CUDA. */
ccs_status ccs_intersect_host_batches(ccs_scene *scene, uint32_t n_batches, const ccs_rays *host_rays,
                                      const uint32_t *n, ccs_hits *host_hits, const ccs_trace_opts *const *opts,
                                      void *stream);

/* Wait for `stream`, then return and clear the scene's latched device status (CCS_OK or
 * CCS_ERR_TRAVERSAL_LIMIT). */
ccs_status ccs_scene_sync_status(ccs_scene *scene, void *stream);

/* Number of patches and of BVH nodes of a scene (host-side values). */
ccs_status ccs_scene_info(const ccs_scene *scene, uint32_t *n_patches, uint32_t *n_nodes);

/* Secondary rays of a wavefront tracer (input generation, not part of the intersection): for every
 * slot i with a hit, a cosine-weighted diffuse ray leaves the surface point f(u_i, v_i) of the hit
 * patch (Gregory patches reduced at (u, v)), offset along the normal (flipped against the incoming
 * direction) by offset_abs + 2 * 2^-L * L1(diagonal of the patch box), which stays outside the hit
 * leaf box (Sec. 3.3 offsets by the L1 size of the last box).  Direction from two PCG32 draws
 * (pcg32_srandom_r(seed, i)), orthonormal basis of Duff et al. 2017.  Slots without a hit get the
 * empty interval tmin = 1, tmax = 0 (they miss).  in_rays (for the incoming direction), hits and
 * out_rays are device planes of n elements; out_rays planes are written (const is cast away).
 * Asynchronous on `stream`. */
ccs_status ccs_gen_diffuse(const ccs_scene *scene, const ccs_rays *in_rays, const ccs_hits *hits, uint32_t n,
                           uint64_t seed, uint32_t leaf_depth, float offset_abs, ccs_rays *out_rays, void *stream);

/* Any-hit query for shadow rays (Sec. 4 traces one shadow ray per path): occluded[i] = 1 if ray i enters
 * a leaf box of some patch within [tmin, tmax] (the condition under which ccs_intersect reports a hit),
 * else 0.  The traversal is the closest-hit one with the best distance held at tmax; it stops at the
 * first leaf it records, so occluded[i] equals (ccs_intersect's patch_id[i] != 0xFFFFFFFF) exactly,
 * whatever the launch options.  Invalid rays and rays that reach opts->iter_cap give 0 (the latter also
 * latch CCS_ERR_TRAVERSAL_LIMIT).  rays: device planes of n elements; occluded: a device array of n
 * bytes, written.  One lane per ray (lanes_per_ray is ignored).  Asynchronous on `stream`. */
ccs_status ccs_occluded(const ccs_scene *scene, const ccs_rays *rays, uint32_t n, uint8_t *occluded,
                        const ccs_trace_opts *opts, void *stream);

/* Shadow rays, as ccs_gen_diffuse but aimed at the point light light[0..2]: unit direction toward the
 * light, tmin = 0, tmax = the distance to it.  Slots without a hit, and slots whose light lies behind the
 * surface (normal flipped against the incoming direction), get the empty interval tmin = 1, tmax = 0. */
ccs_status ccs_gen_shadow(const ccs_scene *scene, const ccs_rays *in_rays, const ccs_hits *hits, uint32_t n,
                          const float *light, uint32_t leaf_depth, float offset_abs, ccs_rays *out_rays, void *stream);

/* ---- Batched scenes (many scenes and their rays per launch; CUDA-graph capturable) ---------------- */
typedef struct ccs_batch ccs_batch;   /* opaque; created and freed by the library */

#define CCS_BATCH_UPDATE 1u      /* repack new control points of every scene that has a point source */
#define CCS_BATCH_REFIT 2u       /* refit every scene's BVH */
#define CCS_BATCH_INTERSECT 4u   /* one persistent closest-hit launch over the rays of all scenes */

/* Group n_scenes built scenes with their rays (device planes, n_rays[s] rays for scene s) and hit
 * buffers.  The batch keeps pointers to the scenes and buffers, which must outlive it.  The rays of
 * all scenes share one work queue, so uneven scenes load-balance within a single launch.  Blocks. */
ccs_status ccs_batch_create(ccs_batch **out, ccs_scene *const *scenes, uint32_t n_scenes, const ccs_rays *rays,
                            const uint32_t *n_rays, const ccs_hits *hits);

/* Source of new control points of scene `scene_index` for the update stage: device planes in the
 * layout of ccs_scene_create (same patch count and types); NULL leaves the scene's points unchanged.
 * Host-side only: the batch's scene table is copied to the device at the start of every run (also
 * inside a captured graph), so a new source applies to every later run or graph launch.  Do not call
 * while a run of this batch may still be copying its table (synchronise the stream first). */
ccs_status ccs_batch_set_points(ccs_batch *b, uint32_t scene_index, const float *x, const float *y, const float *z);

/* Enqueue the selected stages (CCS_BATCH_* bits) on `stream`: the table copy, one repack launch,
 * one refit launch and one intersect launch (with CCS_TRACE_PAIRS in opts: the pair engine's three
 * launches over the rays of all scenes, whose scratch of about 200 bytes per ray the batch allocates
 * with cudaMalloc on its first such run and keeps).  Otherwise allocates nothing; does not synchronise.
 * Answers are bit-identical to ccs_intersect on each scene alone. */
ccs_status ccs_batch_run(ccs_batch *b, uint32_t stages, const ccs_trace_opts *opts, void *stream);

/* Run once, then capture ccs_batch_run(stages, opts) into a CUDA graph owned by the batch (on an
 * internal stream) and instantiate it.  Blocks. */
ccs_status ccs_batch_capture(ccs_batch *b, uint32_t stages, const ccs_trace_opts *opts);

/* Launch the captured graph on `stream` (asynchronous). */
ccs_status ccs_batch_launch(ccs_batch *b, void *stream);

/* Wait for `stream`, then return and clear the batch's latched device status. */
ccs_status ccs_batch_sync_status(ccs_batch *b, void *stream);

ccs_status ccs_batch_destroy(ccs_batch *b);

/* One-shot closest hit of several scenes' rays in one persistent launch (creates a temporary batch,
 * runs CCS_BATCH_INTERSECT and frees it; synchronises `stream`). */
ccs_status ccs_intersect_batched(ccs_scene *const *scenes, const ccs_rays *rays_per_scene, const uint32_t *n_per_scene,
                                 ccs_hits *hits_per_scene, uint32_t n_scenes, const ccs_trace_opts *opts, void *stream);

/* ---- Learned sub-domain proposal ----------------------------------------------------------------
 * A multilayer perceptron 24 -> 64 -> 64 -> 64 (ReLU) scores the 64 depth-3 cells (8 x 8) of a patch's
 * (u,v) domain for a (ray, patch) pair.  Inside ccs_intersect_learned the best-scoring cell is
 * searched first: straight descent to it, search of its subtree, then the full Algorithm 3 from the
 * root with that subtree skipped.  The network only changes the order, so hits are bit-identical to
 * ccs_intersect.  Inference runs on tensor cores (BF16 weights and activations, FP32 accumulation,
 * warp-level MMA); training keeps FP32 master weights and Adam state.
 * Parameters (CCS_PROPOSAL_PARAMS floats): W1 [64,24], b1 [64], W2 [64,64], b2, W3 [64,64], b3, each W
 * row-major [out, in].  Features (CCS_PROPOSAL_FEATURES per pair, see ccs_trace_export), labels =
 * depth-3 cell v3 * 8 + u3 of the pair's best leaf. */
#define CCS_PROPOSAL_PARAMS 9920
#define CCS_PROPOSAL_FEATURES 24
#define CCS_PROPOSAL_CELLS 64
typedef struct ccs_proposal ccs_proposal;   /* opaque; created and freed by the library */

/* He-normal weights from a PCG32 stream seeded with `seed`, zero biases, zero Adam state. */
ccs_status ccs_proposal_create(ccs_proposal **out, uint64_t seed);
ccs_status ccs_proposal_destroy(ccs_proposal *p);
/* Host copies of the FP32 parameters (set also resets the Adam state).  Blocking. */
ccs_status ccs_proposal_set_params(ccs_proposal *p, const float *host_params);
ccs_status ccs_proposal_get_params(const ccs_proposal *p, float *host_params);
/* File: 8-byte magic "CCSPROP1", 4 uint32 layer sizes (24, 64, 64, 64), 9920 float32 parameters. */
ccs_status ccs_proposal_save(const ccs_proposal *p, const char *path);
ccs_status ccs_proposal_load(ccs_proposal **out, const char *path);

/* Mean softmax cross-entropy gradient over a mini-batch (device features [batch, 24], labels [batch]);
 * writes CCS_PROPOSAL_PARAMS floats to grad and the mean loss to *loss (device, optional). */
ccs_status ccs_proposal_grad(ccs_proposal *p, const float *features, const uint8_t *labels, uint32_t batch,
                             float *grad, float *loss, void *stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on a mini-batch; refreshes the BF16
 * copy used by inference.  *loss (device, optional) receives the mini-batch loss before the step. */
ccs_status ccs_proposal_train_step(ccs_proposal *p, const float *features, const uint8_t *labels, uint32_t batch,
                                   float lr, float *loss, void *stream);
/* Tensor-core inference of n feature rows (device): logits [n, 64] (optional), argmax cell [n]
 * (optional; ties go to the lower cell), largest softmax probability [n] (optional). */
ccs_status ccs_proposal_infer(const ccs_proposal *p, const float *features, uint32_t n, float *logits,
                              uint8_t *cells, float *pmax, void *stream);

/* Closest hit as ccs_intersect, and a training trace: for every (ray, patch) pair whose best leaf is
 * the ray's best hit at the end of the pair, appends its 24 features and the depth-3 cell of that leaf
 * (atomic order).  The features, in the patch's anchored frame scaled by S = largest corner distance:
 * ray entry point into the patch box / S (3), unit direction (3), the 4 corners / S (12), unit normal
 * of the corner quad (3), length inside the box / S clamped to 4 (1), direction . normal (1), Gregory
 * flag (1).  *count (device) receives the number of pairs found, which may exceed `capacity` (only the
 * first `capacity` are stored).  leaf_depth >= 3. */
ccs_status ccs_trace_export(const ccs_scene *scene, const ccs_rays *rays, uint32_t n, ccs_hits *hits,
                            const ccs_trace_opts *opts, float *features, uint8_t *labels, uint32_t capacity,
                            uint32_t *count, void *stream);

/* Closest hit with the learned proposal (bit-identical to ccs_intersect).  Proposals whose largest
 * softmax probability is below min_confidence are ignored (plain order for that pair).  Needs
 * block_threads = 128 and leaf_depth >= 3; runs without the sibling cache. */
ccs_status ccs_intersect_learned(const ccs_scene *scene, const ccs_proposal *proposal, const ccs_rays *rays,
                                 uint32_t n, ccs_hits *hits, const ccs_trace_opts *opts, float min_confidence,
                                 void *stream);

/* Allocation-free variant of ccs_intersect_batched (the paper has no counterpart; this is an
 * integration entry point).  For callers that cannot call cudaMalloc at the time they trace: code
 * running under a host that owns all device memory through its own arena or pool, real-time loops
 * with a fixed memory budget, or threads that must not take the CUDA allocator's locks.  The caller
 * passes the built scenes, its rays and its hit buffers as for ccs_intersect_batched; the per-call
 * scratch that ccs_intersect_batched allocates (scene table, ray prefix, work-queue head, status word)
 * lives instead in one fixed file-scope device array sized for CCS_NOALLOC_MAX_SCENES scenes (about
 * 50 KB), which every GPU that loads the library holds until the process exits.
 *  - Every call looks up that array's device address in the current device's context
 *    (cudaGetSymbolAddress), so a device reset between calls does not leave a stale address; the first
 *    call on a device also loads the module there.
 *  - The call copies the scene table and synchronises `stream`, and reads the status word back with a
 *    blocking copy: it can never be called while `stream` (or the legacy stream) is being captured into
 *    a CUDA graph.
 *  - More than CCS_NOALLOC_MAX_SCENES scenes: CCS_ERR_INVALID_ARG with a message; nothing runs.
 *  - Calls no cudaMalloc / cudaFree; the queue head and status word are reset at every call.
 *    CCS_TRACE_PAIRS is ignored (the pair engine's scratch grows with the number of rays).
 *  - All calls share the one array: calls whose work overlaps on the GPU (other threads or streams)
 *    race on it.  The call synchronises `stream` before it returns, so calls from one thread do not.
 * Answers are bit-identical to ccs_intersect_batched and ccs_intersect. */
#define CCS_NOALLOC_MAX_SCENES 256
ccs_status ccs_intersect_batched_noalloc(ccs_scene *const *scenes, const ccs_rays *rays_per_scene,
                                         const uint32_t *n_per_scene, ccs_hits *hits_per_scene, uint32_t n_scenes,
                                         const ccs_trace_opts *opts, void *stream);

/* One measured candidate of ccs_autotune. */
typedef struct {
    ccs_trace_opts opts;
    float ms;                 /* mean time of one ccs_intersect launch */
} ccs_autotune_trial;

/* Autotuner: coordinate descent (two passes) over the BVH width (when the scene was built with
 * CCS_BVH_BOTH), the engine (the ray-persistent kernel without or with CCS_TRACE_ORDER, with the base's
 * image_width, or the pair engine CCS_TRACE_PAIRS), lanes_per_ray {1, 3}, vote {0, 4, 8, 12, 16, 20, 24},
 * threads per block {64, 96, 128}, blocks per SM {1..6}, refill {1, 2, 4, 8, 16, 24}, chunk {32..1024},
 * bvh_burst {1..16}, cache_slots {0, 1, 2} and min_blocks {0, 4}, starting from
 * `base` (NULL: defaults).  These options never change the answer (leaf_depth is kept as given), so
 * tuning is safe.  Each candidate is timed with CUDA events over `reps` launches (after one warm-up)
 * of ccs_intersect on the caller's device rays/hits on `stream`, which is synchronised.  The fastest
 * is written to *best and its mean launch time to *best_ms; if `trials` is given, up to max_trials
 * measurements are recorded and *n_trials receives the number made. */
ccs_status ccs_autotune(const ccs_scene *scene, const ccs_rays *rays, uint32_t n, ccs_hits *hits,
                        const ccs_trace_opts *base, uint32_t reps, ccs_trace_opts *best, float *best_ms,
                        ccs_autotune_trial *trials, uint32_t max_trials, uint32_t *n_trials, void *stream);

/* Mirror-reflection rays, as ccs_gen_diffuse but with direction d - 2 (d . n) n (the incoming direction
 * reflected about the hit normal). */
ccs_status ccs_gen_mirror(const ccs_scene *scene, const ccs_rays *in_rays, const ccs_hits *hits, uint32_t n,
                          uint32_t leaf_depth, float offset_abs, ccs_rays *out_rays, void *stream);

/* Message describing the last failure on the calling thread ("" if none). */
const char *ccs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CCS_H */
