// Closest hit of several scenes in one persistent launch, without any allocation: the scratch that
// ccs_intersect_batched allocates per call (scene table, ray prefix, queue head, status word) lives in
// one file-scope device array of fixed size instead.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "ccs_internal.h"

namespace ccs {

constexpr uint32_t kNoAllocMaxScenes = CCS_NOALLOC_MAX_SCENES;

struct NoAllocScratch {
    uint32_t queue;                                 // work-queue head of the launch
    uint32_t status;                                // latched device status of the launch
    uint32_t pad[62];
    uint32_t ray_prefix[kNoAllocMaxScenes + 64];   // first global ray index of every scene, + total
    BatchEntry entries[kNoAllocMaxScenes];
};

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Device address of the scratch array in the current device's context.  Looked up at every call: a
// lookup is cheap next to the call's own synchronisation, and an address kept from an earlier context
// would be stale after cudaDeviceReset.
static cudaError_t scratch_on_current_device(NoAllocScratch **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<NoAllocScratch *>(p);
    return cudaSuccess;
}

}  // namespace ccs

using namespace ccs;

extern "C" ccs_status ccs_intersect_batched_noalloc(ccs_scene *const *scenes, const ccs_rays *rays_per_scene,
                                                    const uint32_t *n_per_scene, ccs_hits *hits_per_scene,
                                                    uint32_t n_scenes, const ccs_trace_opts *opts, void *stream)
{
    if (!scenes || !rays_per_scene || !n_per_scene || !hits_per_scene || n_scenes == 0) {
        set_error("ccs_intersect_batched_noalloc: scenes, rays, counts and hits must be given, n_scenes > 0");
        return CCS_ERR_INVALID_ARG;
    }
    if (n_scenes > kNoAllocMaxScenes) {
        set_error("ccs_intersect_batched_noalloc: more scenes than CCS_NOALLOC_MAX_SCENES (the size of its static "
                  "scratch array)");
        return CCS_ERR_INVALID_ARG;
    }
    LaunchCfg cfg;
    ccs_status st = fill_launch_cfg(opts, cfg);
    if (st != CCS_OK) return st;
    cfg.flags &= ~CCS_TRACE_PAIRS;   // the pair engine's scratch grows with the rays: not here
    uint64_t total = 0;
    for (uint32_t s = 0; s < n_scenes; ++s) {
        const ccs_scene *sc = scenes[s];
        if (!sc || !sc->built) {
            set_error("ccs_intersect_batched_noalloc: every scene must exist and have a BVH");
            return sc ? CCS_ERR_NOT_BUILT : CCS_ERR_INVALID_ARG;
        }
        if (sc->bvh_width != scenes[0]->bvh_width || sc->alt_width) {
            set_error("ccs_intersect_batched_noalloc: every scene needs one BVH, all of the same width");
            return CCS_ERR_INVALID_ARG;
        }
        const ccs_rays &r = rays_per_scene[s];
        const ccs_hits &h = hits_per_scene[s];
        if (n_per_scene[s] && (!r.ox || !r.oy || !r.oz || !r.dx || !r.dy || !r.dz || !r.tmin || !r.tmax || !h.t ||
                               !h.u || !h.v || !h.patch_id)) {
            set_error("ccs_intersect_batched_noalloc: a ray or hit plane is NULL");
            return CCS_ERR_INVALID_ARG;
        }
        total += n_per_scene[s];
    }
    if (total > 0xFFFFFFFFull) {
        set_error("ccs_intersect_batched_noalloc: more than 2^32 - 1 rays");
        return CCS_ERR_INVALID_ARG;
    }
    NoAllocScratch *scr = nullptr;
    cudaError_t e = scratch_on_current_device(&scr);
    if (e != cudaSuccess) {
        set_error(std::string("ccs_intersect_batched_noalloc: scratch set-up: ") + cudaGetErrorString(e));
        return CCS_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the scene table and prefix go up in chunks from a fixed host buffer (pageable copies return
    // once the source has been read)
    constexpr uint32_t kChunk = 32;
    BatchEntry chunk[kChunk];
    uint32_t prefix[kChunk + 1];
    uint32_t r0 = 0;
    for (uint32_t b = 0; b < n_scenes; b += kChunk) {
        const uint32_t m = (n_scenes - b) < kChunk ? (n_scenes - b) : kChunk;
        for (uint32_t k = 0; k < m; ++k) {
            const ccs_scene *sc = scenes[b + k];
            const ccs_rays &r = rays_per_scene[b + k];
            const ccs_hits &h = hits_per_scene[b + k];
            BatchEntry &t = chunk[k];
            std::memset(&t, 0, sizeof(t));
            t.sc = dev_scene(sc);
            t.rays = DevRays{r.ox, r.oy, r.oz, r.dx, r.dy, r.dz, r.tmin, r.tmax};
            t.hits = DevHits{h.t, h.u, h.v, h.patch_id};
            prefix[k] = r0;
            r0 += n_per_scene[b + k];
        }
        prefix[m] = r0;
        if ((e = cudaMemcpyAsync(scr->entries + b, chunk, sizeof(BatchEntry) * m, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(scr->ray_prefix + b, prefix, sizeof(uint32_t) * (m + 1), cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            set_error(std::string("ccs_intersect_batched_noalloc: table upload: ") + cudaGetErrorString(e));
            return CCS_ERR_CUDA;
        }
    }
    if ((e = cudaMemsetAsync(&scr->status, 0, sizeof(uint32_t), s)) != cudaSuccess ||
        (e = launch_intersect_batch(scr->entries, scr->ray_prefix, n_scenes, (uint32_t)total, cfg, &scr->queue,
                                    &scr->status, scenes[0]->num_sms, s, scenes[0]->bvh_width)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        set_error(std::string("ccs_intersect_batched_noalloc: ") + cudaGetErrorString(e));
        return CCS_ERR_CUDA;
    }
    uint32_t w = 0;
    if ((e = cudaMemcpy(&w, &scr->status, sizeof(uint32_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        set_error(std::string("ccs_intersect_batched_noalloc: status read: ") + cudaGetErrorString(e));
        return CCS_ERR_CUDA;
    }
    if (w) {
        set_error("a ray reached the traversal iteration cap and was written as a miss");
        return CCS_ERR_TRAVERSAL_LIMIT;
    }
    return CCS_OK;
}
