// Internal declarations shared by the host API and the kernels of libccs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "ccs.h"

namespace ccs {

// One patch record = 20 float4 = 320 bytes, control points relative to the record's anchor and, in a
// scene with local frames, rotated into the patch's frame (Sec. 3.4):
//   [0..3] x of the 16 grid slots (slot 4*j + i), [4..7] y, [8..11] z,
//   [12] x of p^v (inner slots (1,1),(2,1),(1,2),(2,2)), [13] y, [14] z,
//   [15] anchor xyz (world box centre), w = 1 for Gregory, 0 for Bezier,
//   [16..18] rows of the frame (identity without local frames), [19] unused.
constexpr int kRecF4 = 20;

// BVH node = 4 float4 = 64 bytes (both children's boxes stored in the parent), one float4 per axis so
// that the lane of a component loads one vector:
//   [0] (c0.lo.x, c0.hi.x, c1.lo.x, c1.hi.x)
//   [1] (c0.lo.y, c0.hi.y, c1.lo.y, c1.hi.y)
//   [2] (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   [3] (child0, child1, parent, slot in parent) as int bits; child >= 0 is a node index,
//       child < 0 is the leaf of patch ~child.  Node 0 is the root (parent -1).
constexpr int kNodeF4 = 4;
constexpr int kEmptyChild = 0x7FFFFFFF;   // child slot without a subtree (single-patch scenes)

// 4-wide BVH node = 8 float4 = 128 bytes, two float4 per axis so that the lane of a component loads two:
//   [2a]   (c0.lo, c1.lo, c2.lo, c3.lo) along axis a,  [2a+1] (c0.hi, c1.hi, c2.hi, c3.hi)
//   [6]    (child0, child1, child2, child3) as int bits (empty slot: kEmptyChild, box lo > hi)
//   [7]    (parent, slot in parent, children present, 0) as int bits
constexpr int kNode4F4 = 8;

constexpr int kMaxLeafDepth = 15;
constexpr int kNumCounters = CCS_NUM_COUNTERS;
constexpr int kNumSumCounters = 20;   // summed counters; the last three are the launch's timeline

struct MlpWeights;

// Export buffers of the trace mode (features + depth-3 cell label of each pair's best leaf).
struct ModeCtx {
    float *ex_features;
    uint8_t *ex_labels;
    uint32_t *ex_count;
    uint32_t ex_capacity;
    uint8_t *occluded;   // any-hit mode: one byte per ray
    float spread;        // screen-space termination: radians per pixel of the ray (0: fixed depth)
};

struct LaunchCfg {
    uint32_t leaf_depth, block_threads, blocks_per_sm, refill, chunk, bvh_burst, cache_slots, min_blocks, vote,
        lanes_per_ray, iter_cap, flags, image_width, host_chunk, bvh_width;
    float pixel_spread;
    unsigned long long *counters;
    int mode = 0;                         // 0 plain, 1 trace export, 2 learned proposal, 3 any hit, 4 screen-space
    ModeCtx mc{};
    const MlpWeights *mlp = nullptr;
    float min_conf = 0.0f;
};

struct DevScene {
    const float4 *rec;       // n_patches records
    const float4 *nodes;     // n_nodes nodes
    const float4 *leaf_box;  // 2 float4 per patch: (lo.xyz, 0), (hi.xyz, 0), the exact patch AABB
    uint32_t n_patches, n_nodes;
    uint32_t local;          // records hold points in local frames (Sec. 3.4)
    uint32_t width;          // BVH node width: 2 or 4
    const uint8_t *types;    // n_patches bytes: 0 Bezier, 1 Gregory
    uint32_t n_greg;         // Gregory patches in the scene
};

struct DevRays {
    const float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
};

struct DevHits {
    float *t, *u, *v;
    uint32_t *pid;
};

// One scene of a batch (device table): where its data, rays and hits live.
struct BatchEntry {
    DevScene sc;
    DevRays rays;
    DevHits hits;
    const float *px, *py, *pz;   // new control points for the update stage (device), or null
    const uint8_t *types;
    float4 *rec, *leaf_box, *nodes;
    const int *leaf_parent;
    uint32_t *refit_flags;
};

// kernels (intersect.cu, scene.cu)
cudaError_t launch_repack(const float *x, const float *y, const float *z, const uint8_t *types, uint32_t n, int local,
                          float4 *rec, float4 *leaf_box, cudaStream_t s);
cudaError_t launch_refit(float4 *nodes, const int *leaf_parent, const float4 *leaf_box, uint32_t *flags,
                         uint32_t n_patches, uint32_t n_nodes, uint32_t width, cudaStream_t s);
cudaError_t launch_intersect(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n,
                             const LaunchCfg &cfg, uint32_t *queue, uint32_t *status, int num_sms, cudaStream_t s,
                             const uint32_t *perm = nullptr);
// work order (order.cu): scratch of order_scratch_words(n, image_width) words; the permutation of ray
// indices in the order the work queue hands them out is its first n words
size_t order_scratch_words(uint32_t n, uint32_t image_width);
cudaError_t launch_order(const DevScene &sc, const DevRays &r, uint32_t n, uint32_t image_width, uint32_t *scratch,
                         cudaStream_t s);
cudaError_t launch_intersect_batch(const BatchEntry *entries, const uint32_t *ray_prefix, uint32_t n_scenes,
                                   uint32_t n_total, const LaunchCfg &cfg, uint32_t *queue, uint32_t *status,
                                   int num_sms, cudaStream_t s, uint32_t width);
// pair engine (pairs.cu): whether a launch with these options runs it, its scratch for n rays, and the
// launches (single scene: scratch from the library's stream-ordered pool; batch: the caller's scratch)
bool use_pairs(const LaunchCfg &cfg);
size_t pairs_scratch_bytes(uint32_t n);
// scratch of one launch from the library's stream-ordered memory pool of the current device (pairs.cu):
// allocated and freed in the order of `s`; freed memory stays in the pool for reuse
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
cudaError_t pool_free(void *p, cudaStream_t s);
cudaError_t launch_pairs_single(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n,
                                const LaunchCfg &cfg, uint32_t *status, int num_sms, cudaStream_t s);
cudaError_t launch_pairs_batch(const BatchEntry *entries, const uint32_t *ray_prefix, uint32_t n_scenes,
                               uint32_t n_total, const LaunchCfg &cfg, void *scratch,
                               uint32_t *status, int num_sms, cudaStream_t s, uint32_t width);
cudaError_t launch_batch_repack(const BatchEntry *entries, const uint32_t *patch_prefix, uint32_t n_scenes,
                                uint32_t n_patches, cudaStream_t s);
cudaError_t launch_batch_refit(const BatchEntry *entries, const uint32_t *patch_prefix, uint32_t n_scenes,
                               uint32_t n_patches, uint32_t *flags, uint32_t n_flag_words, cudaStream_t s);
ccs_status fill_launch_cfg(const ccs_trace_opts *o, LaunchCfg &c);
const MlpWeights *proposal_weights(const ccs_proposal *p);

cudaError_t launch_gen_diffuse(const float4 *rec, const float4 *leaf_box, uint32_t n_patches, const DevRays &in,
                               const DevHits &hits, uint32_t n, unsigned long long seed, int L, float offset_abs, float *o, float *d,
                               float *tmin, float *tmax, int kind, const float *light, int local, cudaStream_t s);

void set_error(const std::string &msg);

}  // namespace ccs

struct ccs_scene {
    uint32_t n = 0;
    int device = 0;
    int num_sms = 0;
    std::vector<float> hx, hy, hz;     // host copy of the input points (BVH build)
    std::vector<uint8_t> htypes;
    float4 *d_rec = nullptr;           // patch records
    float4 *d_leaf_box = nullptr;      // 2 float4 per patch: (lo.xyz, 0), (hi.xyz, 0)
    uint8_t *d_types = nullptr;
    uint32_t n_greg = 0;               // Gregory patches
    float4 *d_nodes = nullptr;
    int *d_leaf_parent = nullptr;      // per patch: (node << 1) | slot
    uint32_t *d_refit_flags = nullptr; // per node arrival counters of the refit
    uint32_t n_nodes = 0;
    uint32_t bvh_width = 2;            // node width of the built BVH (the default of launches)
    // a second BVH of the other width, built with CCS_BVH_BOTH (launches pick it by opts->bvh_width)
    float4 *d_nodes_alt = nullptr;
    int *d_leaf_parent_alt = nullptr;
    uint32_t *d_refit_flags_alt = nullptr;
    uint32_t n_nodes_alt = 0;
    uint32_t alt_width = 0;            // 0: none
    bool built = false;
    bool local = false;                // CCS_SCENE_LOCAL_FRAMES
    uint32_t *d_work = nullptr;        // [1] device status word; [kQueueBase + k] ring of work-queue heads
    std::atomic<uint32_t> next_queue{0};   // next ring slot: launches in flight at once use different heads
    // host-buffer path: staging planes and the copy/compute pipeline (created on first use)
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr, pipe_comp = nullptr;
    cudaEvent_t pipe_ev[2] = {};             // start; end of the copies out
    std::vector<cudaEvent_t> pipe_chunk_ev;  // per chunk of a call: input copied, hits written (grown on use)
};

namespace ccs {
// The scene's work words: the status word, then a ring of queue heads.  Every launch takes the next
// head, so launches on different streams (or the host path's two compute streams) do not share one.
constexpr int kQueueBase = 16, kQueueRing = 48, kWorkWords = kQueueBase + kQueueRing;
inline uint32_t *take_queue(ccs_scene *sc)
{
    return sc->d_work + kQueueBase + sc->next_queue.fetch_add(1, std::memory_order_relaxed) % kQueueRing;
}

inline DevScene dev_scene(const ccs_scene *sc)
{
    return DevScene{sc->d_rec,        sc->d_nodes, sc->d_leaf_box, sc->n, sc->n_nodes, sc->local ? 1u : 0u,
                    sc->bvh_width,    sc->d_types, sc->n_greg};
}

// The scene seen through its BVH of the given width (0: the default one); the caller has checked that
// the scene holds it (has_width).
inline bool has_width(const ccs_scene *sc, uint32_t width)
{
    return width == 0 || width == sc->bvh_width || (sc->alt_width != 0 && width == sc->alt_width);
}
inline DevScene dev_scene(const ccs_scene *sc, uint32_t width)
{
    if (width == 0 || width == sc->bvh_width) return dev_scene(sc);
    return DevScene{sc->d_rec,     sc->d_nodes_alt, sc->d_leaf_box, sc->n,       sc->n_nodes_alt,
                    sc->local ? 1u : 0u, sc->alt_width, sc->d_types, sc->n_greg};
}
}  // namespace ccs
