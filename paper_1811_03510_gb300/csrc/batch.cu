// Batched scenes: many scenes with their own rays in one launch per stage.  Per run: one repack
// launch (new control points of every scene), one refit launch (every BVH) and one persistent
// intersect launch whose work queue spans the rays of all scenes.  The run enqueues no allocation
// and no synchronisation, so it can be captured into a CUDA graph (ccs_batch_capture).
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "scene_dev.cuh"

namespace ccs {

__device__ __forceinline__ uint32_t find_scene(const uint32_t *__restrict__ prefix, uint32_t n_scenes, uint32_t i)
{
    uint32_t lo = 0, hi = n_scenes;   // largest s with prefix[s] <= i
    while (hi - lo > 1) {
        const uint32_t m = (lo + hi) >> 1;
        if (__ldg(prefix + m) <= i) lo = m; else hi = m;
    }
    return lo;
}

__global__ void k_batch_repack(const BatchEntry *__restrict__ entries, const uint32_t *__restrict__ patch_prefix,
                               uint32_t n_scenes, uint32_t n_patches)
{
    const uint32_t gp = blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= n_patches) return;
    const uint32_t s = find_scene(patch_prefix, n_scenes, gp);
    const BatchEntry &e = entries[s];
    if (!e.px) return;
    repack_one(e.px, e.py, e.pz, e.types, gp - patch_prefix[s], e.rec, e.leaf_box, (int)e.sc.local);
}

__global__ void k_batch_refit(const BatchEntry *__restrict__ entries, const uint32_t *__restrict__ patch_prefix,
                              uint32_t n_scenes, uint32_t n_patches)
{
    const uint32_t gp = blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= n_patches) return;
    const uint32_t s = find_scene(patch_prefix, n_scenes, gp);
    const BatchEntry &e = entries[s];
    refit_one(e.nodes, e.leaf_parent, e.leaf_box, e.refit_flags, gp - patch_prefix[s], e.sc.width);
}

cudaError_t launch_batch_repack(const BatchEntry *entries, const uint32_t *patch_prefix, uint32_t n_scenes,
                                uint32_t n_patches, cudaStream_t s)
{
    if (n_patches == 0) return cudaSuccess;
    k_batch_repack<<<(n_patches + 127) / 128, 128, 0, s>>>(entries, patch_prefix, n_scenes, n_patches);
    return cudaGetLastError();
}

cudaError_t launch_batch_refit(const BatchEntry *entries, const uint32_t *patch_prefix, uint32_t n_scenes,
                               uint32_t n_patches, uint32_t *flags, uint32_t n_flag_words, cudaStream_t s)
{
    if (n_patches == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * n_flag_words, s);
    if (e != cudaSuccess) return e;
    k_batch_refit<<<(n_patches + 127) / 128, 128, 0, s>>>(entries, patch_prefix, n_scenes, n_patches);
    return cudaGetLastError();
}

}  // namespace ccs

using namespace ccs;

struct ccs_batch {
    uint32_t n = 0;                       // scenes
    uint32_t n_rays = 0, n_patches = 0, n_nodes = 0;
    int num_sms = 0;
    uint32_t width = 2;                   // BVH node width of every scene
    BatchEntry *h_table = nullptr;        // pinned host copy, uploaded at the start of every run
    BatchEntry *d_table = nullptr;
    uint32_t *d_ray_prefix = nullptr, *d_patch_prefix = nullptr;
    uint32_t *d_flags = nullptr;          // refit arrival counters of every scene's nodes
    uint32_t *d_work = nullptr;           // [0] queue head, [1] status word
    void *d_pairs = nullptr;              // the pair engine's scratch (CCS_TRACE_PAIRS), made on first use
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void batch_free(ccs_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFreeHost(b->h_table);
    cudaFree(b->d_table);
    cudaFree(b->d_ray_prefix);
    cudaFree(b->d_patch_prefix);
    cudaFree(b->d_flags);
    cudaFree(b->d_work);
    cudaFree(b->d_pairs);
    delete b;
}

#define BCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                        \
            return e_ == cudaErrorMemoryAllocation ? CCS_ERR_OOM : CCS_ERR_CUDA;                  \
        }                                                                                         \
    } while (0)

extern "C" {

ccs_status ccs_batch_create(ccs_batch **out, ccs_scene *const *scenes, uint32_t n_scenes, const ccs_rays *rays,
                            const uint32_t *n_rays, const ccs_hits *hits)
{
    if (!out || !scenes || n_scenes == 0 || !rays || !n_rays || !hits) {
        set_error("ccs_batch_create: out, scenes, rays, n_rays and hits must be given, n_scenes > 0");
        return CCS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    uint64_t tot_r = 0, tot_p = 0, tot_n = 0;
    for (uint32_t s = 0; s < n_scenes; ++s) {
        const ccs_scene *sc = scenes[s];
        if (!sc || !sc->built) {
            set_error("ccs_batch_create: every scene must exist and have a BVH (ccs_bvh_build)");
            return sc ? CCS_ERR_NOT_BUILT : CCS_ERR_INVALID_ARG;
        }
        if (sc->bvh_width != scenes[0]->bvh_width || sc->alt_width) {
            set_error("ccs_batch_create: every scene needs one BVH, all of the same width");
            return CCS_ERR_INVALID_ARG;
        }
        if (n_rays[s] && (!rays[s].ox || !rays[s].oy || !rays[s].oz || !rays[s].dx || !rays[s].dy || !rays[s].dz ||
                          !rays[s].tmin || !rays[s].tmax || !hits[s].t || !hits[s].u || !hits[s].v ||
                          !hits[s].patch_id)) {
            set_error("ccs_batch_create: a ray or hit plane is NULL");
            return CCS_ERR_INVALID_ARG;
        }
        tot_r += n_rays[s];
        tot_p += sc->n;
        tot_n += sc->n_nodes;
    }
    if (tot_r > 0xFFFFFFFFull || tot_p > (1ull << 30) || tot_n > (1ull << 31)) {
        set_error("ccs_batch_create: batch too large");
        return CCS_ERR_INVALID_ARG;
    }
    ccs_batch *b = new (std::nothrow) ccs_batch();
    if (!b) {
        set_error("host allocation failed");
        return CCS_ERR_OOM;
    }
    b->n = n_scenes;
    b->n_rays = (uint32_t)tot_r;
    b->n_patches = (uint32_t)tot_p;
    b->n_nodes = (uint32_t)tot_n;
    b->num_sms = scenes[0]->num_sms;
    b->width = scenes[0]->bvh_width;
    std::vector<uint32_t> rp(n_scenes + 1), pp(n_scenes + 1);
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMallocHost(&b->h_table, sizeof(BatchEntry) * n_scenes)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->d_table, sizeof(BatchEntry) * n_scenes)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->d_ray_prefix, sizeof(uint32_t) * (n_scenes + 1))) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->d_patch_prefix, sizeof(uint32_t) * (n_scenes + 1))) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->d_flags, sizeof(uint32_t) * (b->n_nodes ? b->n_nodes : 1))) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->d_work, 64)) != cudaSuccess) break;
        if ((e = cudaMemset(b->d_work, 0, 64)) != cudaSuccess) break;
        uint32_t r = 0, p = 0, nn = 0;
        for (uint32_t s = 0; s < n_scenes; ++s) {
            ccs_scene *sc = scenes[s];
            BatchEntry &t = b->h_table[s];
            std::memset(&t, 0, sizeof(t));
            t.sc = dev_scene(sc);
            t.rays = DevRays{rays[s].ox, rays[s].oy, rays[s].oz, rays[s].dx, rays[s].dy, rays[s].dz, rays[s].tmin,
                             rays[s].tmax};
            t.hits = DevHits{hits[s].t, hits[s].u, hits[s].v, hits[s].patch_id};
            t.types = sc->d_types;
            t.rec = sc->d_rec;
            t.leaf_box = sc->d_leaf_box;
            t.nodes = sc->d_nodes;
            t.leaf_parent = sc->d_leaf_parent;
            t.refit_flags = b->d_flags + nn;
            rp[s] = r;
            pp[s] = p;
            r += n_rays[s];
            p += sc->n;
            nn += sc->n_nodes;
        }
        rp[n_scenes] = r;
        pp[n_scenes] = p;
        if ((e = cudaMemcpy(b->d_ray_prefix, rp.data(), sizeof(uint32_t) * (n_scenes + 1), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            break;
        if ((e = cudaMemcpy(b->d_patch_prefix, pp.data(), sizeof(uint32_t) * (n_scenes + 1),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
        if ((e = cudaMemcpy(b->d_table, b->h_table, sizeof(BatchEntry) * n_scenes, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            break;
        if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) break;
        *out = b;
        return CCS_OK;
    } while (0);
    set_error(std::string("ccs_batch_create: ") + cudaGetErrorString(e));
    batch_free(b);
    return e == cudaErrorMemoryAllocation ? CCS_ERR_OOM : CCS_ERR_CUDA;
}

ccs_status ccs_batch_set_points(ccs_batch *b, uint32_t scene_index, const float *x, const float *y, const float *z)
{
    if (!b || scene_index >= b->n || ((x || y || z) && !(x && y && z))) {
        set_error("ccs_batch_set_points: bad batch, index or point planes");
        return CCS_ERR_INVALID_ARG;
    }
    BatchEntry &t = b->h_table[scene_index];
    t.px = x;
    t.py = y;
    t.pz = z;
    return CCS_OK;
}

ccs_status ccs_batch_run(ccs_batch *b, uint32_t stages, const ccs_trace_opts *opts, void *stream)
{
    if (!b) {
        set_error("ccs_batch_run: batch is NULL");
        return CCS_ERR_INVALID_ARG;
    }
    LaunchCfg cfg;
    ccs_status st = fill_launch_cfg(opts, cfg);
    if (st != CCS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    BCK(cudaMemcpyAsync(b->d_table, b->h_table, sizeof(BatchEntry) * b->n, cudaMemcpyHostToDevice, s));
    if (stages & CCS_BATCH_UPDATE) BCK(launch_batch_repack(b->d_table, b->d_patch_prefix, b->n, b->n_patches, s));
    if (stages & CCS_BATCH_REFIT)
        BCK(launch_batch_refit(b->d_table, b->d_patch_prefix, b->n, b->n_patches, b->d_flags, b->n_nodes, s));
    if ((stages & CCS_BATCH_INTERSECT) && use_pairs(cfg)) {
        if (!b->d_pairs) BCK(cudaMalloc(&b->d_pairs, pairs_scratch_bytes(b->n_rays ? b->n_rays : 1)));
        BCK(launch_pairs_batch(b->d_table, b->d_ray_prefix, b->n, b->n_rays, cfg, b->d_pairs, b->d_work + 1,
                               b->num_sms, s, b->width));
    } else if (stages & CCS_BATCH_INTERSECT) {
        BCK(launch_intersect_batch(b->d_table, b->d_ray_prefix, b->n, b->n_rays, cfg, b->d_work, b->d_work + 1,
                                   b->num_sms, s, b->width));
    }
    return CCS_OK;
}

ccs_status ccs_batch_capture(ccs_batch *b, uint32_t stages, const ccs_trace_opts *opts)
{
    if (!b) {
        set_error("ccs_batch_capture: batch is NULL");
        return CCS_ERR_INVALID_ARG;
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    // one eager run first: kernel attributes are set outside the capture
    ccs_status st = ccs_batch_run(b, stages, opts, b->cap_stream);
    if (st != CCS_OK) return st;
    BCK(cudaStreamSynchronize(b->cap_stream));
    BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    st = ccs_batch_run(b, stages, opts, b->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != CCS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        set_error(std::string("ccs_batch_capture: ") + cudaGetErrorString(e));
        return CCS_ERR_CUDA;
    }
    b->graph = g;
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return CCS_OK;
}

ccs_status ccs_batch_launch(ccs_batch *b, void *stream)
{
    if (!b || !b->exec) {
        set_error("ccs_batch_launch: no captured graph (ccs_batch_capture)");
        return b ? CCS_ERR_NOT_BUILT : CCS_ERR_INVALID_ARG;
    }
    BCK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return CCS_OK;
}

ccs_status ccs_batch_sync_status(ccs_batch *b, void *stream)
{
    if (!b) {
        set_error("ccs_batch_sync_status: batch is NULL");
        return CCS_ERR_INVALID_ARG;
    }
    BCK(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t w = 0;
    BCK(cudaMemcpy(&w, b->d_work + 1, 4, cudaMemcpyDeviceToHost));
    if (w) {
        BCK(cudaMemset(b->d_work + 1, 0, 4));
        set_error("a ray reached the traversal iteration cap and was written as a miss");
        return CCS_ERR_TRAVERSAL_LIMIT;
    }
    return CCS_OK;
}

ccs_status ccs_batch_destroy(ccs_batch *b)
{
    if (b) {
        cudaStreamSynchronize(b->cap_stream);
        batch_free(b);
    }
    return CCS_OK;
}

ccs_status ccs_intersect_batched(ccs_scene *const *scenes, const ccs_rays *rays_per_scene, const uint32_t *n_per_scene,
                                 ccs_hits *hits_per_scene, uint32_t n_scenes, const ccs_trace_opts *opts, void *stream)
{
    ccs_batch *b = nullptr;
    ccs_status st = ccs_batch_create(&b, scenes, n_scenes, rays_per_scene, n_per_scene, hits_per_scene);
    if (st != CCS_OK) return st;
    st = ccs_batch_run(b, CCS_BATCH_INTERSECT, opts, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (st == CCS_OK && e != cudaSuccess) {
        set_error(std::string("ccs_intersect_batched: ") + cudaGetErrorString(e));
        st = CCS_ERR_CUDA;
    }
    uint32_t w = 0;
    if (st == CCS_OK && cudaMemcpy(&w, b->d_work + 1, 4, cudaMemcpyDeviceToHost) == cudaSuccess && w) {
        set_error("a ray reached the traversal iteration cap and was written as a miss");
        st = CCS_ERR_TRAVERSAL_LIMIT;
    }
    batch_free(b);
    return st;
}

}  // extern "C"
