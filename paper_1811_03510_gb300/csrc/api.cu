// C ABI of libccs (declared in include/ccs.h): scene store, BVH build/refit, intersect launches.
#include <cuda_runtime.h>

#include <cmath>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "bvh_build.h"
#include "ccs_internal.h"
#include "host_plan.h"

namespace ccs {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

}  // namespace ccs

using namespace ccs;

#define CCS_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
            return e_ == cudaErrorMemoryAllocation ? CCS_ERR_OOM : CCS_ERR_CUDA;       \
        }                                                                              \
    } while (0)

#define CCS_ARG(cond, msg)                  \
    do {                                    \
        if (!(cond)) {                      \
            set_error(msg);                 \
            return CCS_ERR_INVALID_ARG;     \
        }                                   \
    } while (0)

static const uint32_t kMaxPatches = 1u << 26;

namespace {

void free_scene(ccs_scene *s)
{
    if (!s) return;
    cudaFree(s->d_rec);
    cudaFree(s->d_leaf_box);
    cudaFree(s->d_types);
    cudaFree(s->d_nodes);
    cudaFree(s->d_leaf_parent);
    cudaFree(s->d_refit_flags);
    cudaFree(s->d_nodes_alt);
    cudaFree(s->d_leaf_parent_alt);
    cudaFree(s->d_refit_flags_alt);
    cudaFree(s->d_work);
    cudaFree(s->d_stage);
    for (cudaEvent_t e : s->pipe_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : s->pipe_chunk_ev) cudaEventDestroy(e);
    for (cudaStream_t q : {s->pipe_h2d, s->pipe_d2h, s->pipe_comp})
        if (q) cudaStreamDestroy(q);
    delete s;
}

}  // namespace

ccs_status ccs::fill_launch_cfg(const ccs_trace_opts *o, LaunchCfg &c)
{
    c.leaf_depth = o && o->leaf_depth ? o->leaf_depth : 8;
    c.block_threads = o && o->block_threads ? o->block_threads : 128;
    c.blocks_per_sm = o && o->blocks_per_sm ? o->blocks_per_sm : 4;
    c.refill = o && o->refill ? o->refill : 8;
    c.chunk = o && o->chunk ? o->chunk : 32;
    c.bvh_burst = o && o->bvh_burst ? o->bvh_burst : 8;
    c.cache_slots = (!o || o->cache_slots == CCS_CACHE_DEFAULT) ? 2 : o->cache_slots;
    c.min_blocks = o ? o->min_blocks : 0;
    c.vote = o ? o->vote : 0;
    c.lanes_per_ray = o && o->lanes_per_ray ? o->lanes_per_ray : 1;
    c.pixel_spread = o ? o->pixel_spread : 0.0f;
    c.mc.spread = c.pixel_spread;
    c.iter_cap = o && o->iter_cap ? o->iter_cap : (1u << 22);
    c.flags = o ? o->flags : 0;
    c.image_width = o ? o->image_width : 0;
    c.host_chunk = o ? o->host_chunk : 0;
    c.bvh_width = o ? o->bvh_width : 0;
    c.counters = o ? reinterpret_cast<unsigned long long *>(o->counters) : nullptr;
    CCS_ARG(c.leaf_depth >= 1 && c.leaf_depth <= (uint32_t)kMaxLeafDepth, "leaf_depth must be in 1..15");
    CCS_ARG(c.block_threads % 32 == 0 && c.block_threads >= 32 && c.block_threads <= 128,
            "block_threads must be a multiple of 32 in 32..128");
    CCS_ARG(c.blocks_per_sm >= 1 && c.blocks_per_sm <= 64, "blocks_per_sm must be in 1..64");
    CCS_ARG(c.refill >= 1 && c.refill <= 32, "refill must be in 1..32");
    CCS_ARG(c.chunk % 32 == 0 && c.chunk >= 32 && c.chunk <= 4096, "chunk must be a multiple of 32 in 32..4096");
    CCS_ARG(c.bvh_burst >= 1 && c.bvh_burst <= 16, "bvh_burst must be in 1..16");
    CCS_ARG(c.cache_slots <= 2, "cache_slots must be 0, 1 or 2");
    CCS_ARG(c.min_blocks == 0 || c.min_blocks == 4, "min_blocks must be 0 or 4");
    CCS_ARG(c.vote <= 32, "vote must be in 0..32");
    CCS_ARG(c.lanes_per_ray == 1 || c.lanes_per_ray == 3, "lanes_per_ray must be 1 or 3");
    CCS_ARG(c.pixel_spread >= 0.0f && c.pixel_spread < 1.0f, "pixel_spread must be in [0, 1) radians per pixel");
    CCS_ARG(c.bvh_width == 0 || c.bvh_width == 2 || c.bvh_width == 4, "bvh_width must be 0, 2 or 4");
    CCS_ARG(!(c.flags & CCS_TRACE_COUNT) || c.counters, "CCS_TRACE_COUNT needs opts->counters");
    CCS_ARG((c.flags & ~(CCS_TRACE_COUNT | CCS_TRACE_ORDER | CCS_TRACE_HOST_MAPPED | CCS_TRACE_PAIRS)) == 0,
            "unknown trace flags");
    return CCS_OK;
}

namespace {

ccs_status check_rays(const ccs_rays *r, const ccs_hits *h)
{
    CCS_ARG(r && h, "rays and hits must not be NULL");
    CCS_ARG(r->ox && r->oy && r->oz && r->dx && r->dy && r->dz && r->tmin && r->tmax, "a ray plane is NULL");
    CCS_ARG(h->t && h->u && h->v && h->patch_id, "a hit plane is NULL");
    return CCS_OK;
}

// With CCS_TRACE_ORDER: the permutation of the launch's rays in estimated-cost order, computed on
// `stream` into scratch of its own from the library's stream-ordered pool (so that launches on different
// streams never share it); the caller releases it on the same stream after the launch (release_order).
// *perm stays null without the flag.
ccs_status work_order(const ccs_scene *sc, const LaunchCfg &cfg, const DevRays &dr, uint32_t n, cudaStream_t s,
                      const uint32_t **perm)
{
    *perm = nullptr;
    if (!(cfg.flags & CCS_TRACE_ORDER) || n == 0 || use_pairs(cfg)) return CCS_OK;
    const size_t words = order_scratch_words(n, cfg.image_width);
    void *p = nullptr;
    CCS_CUDA(pool_alloc(&p, words * sizeof(uint32_t), s));
    // the estimate counts the patch boxes a ray enters, the same in either tree: it walks the 4-wide one
    // when the scene has it (fewer dependent node loads)
    const uint32_t est_width = (sc->bvh_width == 4 || sc->alt_width == 4) ? 4u : 0u;
    const cudaError_t e = launch_order(dev_scene(sc, est_width), dr, n, cfg.image_width, static_cast<uint32_t *>(p), s);
    if (e != cudaSuccess) {
        pool_free(p, s);
        CCS_CUDA(e);
    }
    *perm = static_cast<const uint32_t *>(p);
    return CCS_OK;
}

ccs_status release_order(const uint32_t *perm, cudaStream_t s)
{
    if (perm) CCS_CUDA(pool_free(const_cast<uint32_t *>(perm), s));
    return CCS_OK;
}

// One batch of host rays for the staged pipeline.
struct HostBatch {
    const ccs_rays *hr;
    uint32_t n;
    ccs_hits *hh;
    LaunchCfg cfg;
};

// The staged copy/trace pipeline of the host-buffer entry points, over the chunks of one or more batches
// in order: chunk k's rays are copied in while chunk k-1 is traced and chunk k-2's hits are copied out.
// Every chunk's copy in is queued first, so that the copy engine never waits for the host to queue a
// launch.  Consecutive chunks alternate between the caller's stream and a second compute stream, each
// launch with its own queue head, so that one chunk's launch fills the SMs that the previous one frees
// while its last rays finish; across batches the same holds, so one batch's copies and launch overlap the
// end of the last.  (A third compute stream measured the same.)
// Chunks stay large: every launch ends on its slowest rays, and many small chunks pay that drain more
// often than they save in exposed copy time.  An image's chunk boundaries fall on rows of 8-pixel tiles
// of the work order, or on the bands of 4 rows of the pair engine's candidate pass, so that each chunk is
// an image too.  Batch j stages its twelve planes (eight of rays, four of hits) at
// 12 * (rays of the batches before it) floats into the scene's staging buffer.
ccs_status host_pipeline(ccs_scene *sc, const HostBatch *bt, uint32_t nb, cudaStream_t s)
{
    size_t total = 0;
    std::vector<size_t> base(nb);
    for (uint32_t j = 0; j < nb; ++j) {
        base[j] = 12 * total;
        total += bt[j].n;
    }
    if (total == 0) return CCS_OK;
    const size_t need = total * 12 * sizeof(float);
    if (need > sc->stage_bytes) {
        CCS_CUDA(cudaStreamSynchronize(s));
        cudaFree(sc->d_stage);
        sc->d_stage = nullptr;
        sc->stage_bytes = 0;
        CCS_CUDA(cudaMalloc(&sc->d_stage, need));
        sc->stage_bytes = need;
    }
    if (!sc->pipe_h2d) {
        for (cudaStream_t *q : {&sc->pipe_h2d, &sc->pipe_d2h, &sc->pipe_comp})
            CCS_CUDA(cudaStreamCreateWithFlags(q, cudaStreamNonBlocking));
        for (cudaEvent_t &e : sc->pipe_ev) CCS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    std::vector<uint32_t> ns(nb), hc(nb);
    std::vector<size_t> align(nb);
    for (uint32_t j = 0; j < nb; ++j) {
        const LaunchCfg &c = bt[j].cfg;
        ns[j] = bt[j].n;
        hc[j] = c.host_chunk;
        // the pair engine pays a launch's drain once per chunk: a batch under 2^19 rays goes in one chunk;
        // chunk boundaries fall on its candidate pass's bands of 4 image rows
        const bool pairs = use_pairs(c);
        if (!hc[j] && pairs && ns[j] < (1u << 19)) hc[j] = ns[j];
        align[j] = (c.flags & CCS_TRACE_ORDER) && c.image_width ? (size_t)c.image_width * 8
                   : pairs && c.image_width && (c.image_width & 7u) == 0 ? (size_t)c.image_width * 4
                                                                        : 1;
    }
    const std::vector<HostChunk> chunks = host_batch_chunks(nb, ns.data(), hc.data(), align.data());
    // events: start, end of the copies out, and a pair per chunk (input copied, hits written)
    while (sc->pipe_chunk_ev.size() < 2 * chunks.size()) {
        cudaEvent_t e;
        CCS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        sc->pipe_chunk_ev.push_back(e);
    }
    const cudaEvent_t ev_start = sc->pipe_ev[0], ev_out = sc->pipe_ev[1];
    CCS_CUDA(cudaEventRecord(ev_start, s));
    for (cudaStream_t q : {sc->pipe_h2d, sc->pipe_d2h, sc->pipe_comp}) CCS_CUDA(cudaStreamWaitEvent(q, ev_start, 0));
    // planes at one constant stride (rows of one host block) move as one 2D copy per chunk
    auto stride_of = [](const void *const *pl, int k, size_t n) -> size_t {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(pl[0]);
        const uintptr_t a1 = reinterpret_cast<uintptr_t>(pl[1]);
        if (a1 <= a0 || (a1 - a0) % 4 != 0 || a1 - a0 < n * 4) return 0;
        for (int c = 2; c < k; ++c)
            if (reinterpret_cast<uintptr_t>(pl[c]) != a0 + (uintptr_t)c * (a1 - a0)) return 0;
        return a1 - a0;
    };
    std::vector<size_t> in_pitch(nb), out_pitch(nb);
    for (uint32_t j = 0; j < nb; ++j) {
        const ccs_rays *r = bt[j].hr;
        const ccs_hits *h = bt[j].hh;
        const void *srcv[8] = {r->ox, r->oy, r->oz, r->dx, r->dy, r->dz, r->tmin, r->tmax};
        const void *dstv[4] = {h->t, h->u, h->v, h->patch_id};
        in_pitch[j] = stride_of(srcv, 8, bt[j].n);
        out_pitch[j] = stride_of(dstv, 4, bt[j].n);
    }
    float *stage = static_cast<float *>(sc->d_stage);
    // (1) every chunk's rays in, in order
    for (size_t k = 0; k < chunks.size(); ++k) {
        const HostChunk &ck = chunks[k];
        const HostBatch &B = bt[ck.j];
        const size_t n = B.n, a = ck.a, m = ck.m;
        float *b = stage + base[ck.j];
        const float *src[8] = {B.hr->ox, B.hr->oy, B.hr->oz, B.hr->dx, B.hr->dy, B.hr->dz, B.hr->tmin, B.hr->tmax};
        // (equally spaced planes of separate allocations are refused by the runtime at the call, with
        // nothing enqueued; the copies then go plane by plane)
        if (in_pitch[ck.j] && cudaMemcpy2DAsync(b + a, n * 4, src[0] + a, in_pitch[ck.j], m * 4, 8,
                                                cudaMemcpyHostToDevice, sc->pipe_h2d) != cudaSuccess) {
            (void)cudaGetLastError();
            in_pitch[ck.j] = 0;
        }
        if (!in_pitch[ck.j]) {
            for (int c = 0; c < 8; ++c)
                CCS_CUDA(cudaMemcpyAsync(b + c * n + a, src[c] + a, m * 4, cudaMemcpyHostToDevice, sc->pipe_h2d));
        }
        CCS_CUDA(cudaEventRecord(sc->pipe_chunk_ev[2 * k], sc->pipe_h2d));
    }
    // (2) the launches, each chunk's hits out after its launch
    for (size_t k = 0; k < chunks.size(); ++k) {
        const HostChunk &ck = chunks[k];
        const HostBatch &B = bt[ck.j];
        const size_t n = B.n, a = ck.a, m = ck.m;
        float *b = stage + base[ck.j];
        void *dst[4] = {B.hh->t, B.hh->u, B.hh->v, B.hh->patch_id};
        const cudaEvent_t ev_hit = sc->pipe_chunk_ev[2 * k + 1];
        cudaStream_t cs = (k & 1) ? sc->pipe_comp : s;
        CCS_CUDA(cudaStreamWaitEvent(cs, sc->pipe_chunk_ev[2 * k], 0));
        const DevRays dr{b + a, b + n + a, b + 2 * n + a, b + 3 * n + a, b + 4 * n + a, b + 5 * n + a,
                         b + 6 * n + a, b + 7 * n + a};
        const DevHits dh{b + 8 * n + a, b + 9 * n + a, b + 10 * n + a, reinterpret_cast<uint32_t *>(b + 11 * n + a)};
        const uint32_t *perm;
        ccs_status st = work_order(sc, B.cfg, dr, (uint32_t)m, cs, &perm);
        if (st != CCS_OK) return st;
        CCS_CUDA(launch_intersect(dev_scene(sc, B.cfg.bvh_width), dr, dh, (uint32_t)m, B.cfg, take_queue(sc),
                                  sc->d_work + 1, sc->num_sms, cs, perm));
        if ((st = release_order(perm, cs)) != CCS_OK) return st;
        CCS_CUDA(cudaEventRecord(ev_hit, cs));
        CCS_CUDA(cudaStreamWaitEvent(sc->pipe_d2h, ev_hit, 0));
        if (out_pitch[ck.j] && cudaMemcpy2DAsync(static_cast<char *>(dst[0]) + a * 4, out_pitch[ck.j], b + 8 * n + a,
                                                 n * 4, m * 4, 4, cudaMemcpyDeviceToHost, sc->pipe_d2h) != cudaSuccess) {
            (void)cudaGetLastError();
            out_pitch[ck.j] = 0;
        }
        if (!out_pitch[ck.j]) {
            for (int c = 0; c < 4; ++c)
                CCS_CUDA(cudaMemcpyAsync(static_cast<char *>(dst[c]) + a * 4, b + (8 + c) * n + a, m * 4,
                                         cudaMemcpyDeviceToHost, sc->pipe_d2h));
        }
    }
    CCS_CUDA(cudaEventRecord(ev_out, sc->pipe_d2h));
    CCS_CUDA(cudaStreamWaitEvent(s, ev_out, 0));
    CCS_CUDA(cudaStreamSynchronize(s));
    return CCS_OK;
}

}  // namespace

extern "C" {

const char *ccs_last_error(void) { return g_err.c_str(); }

ccs_status ccs_scene_create(ccs_scene **out, const float *x, const float *y, const float *z, const uint8_t *types,
                            uint32_t n_patches, int flags, void *stream)
{
    CCS_ARG(out, "out must not be NULL");
    *out = nullptr;
    CCS_ARG((flags & ~(CCS_SCENE_DEVICE_PTRS | CCS_SCENE_LOCAL_FRAMES)) == 0, "unknown scene flags");
    const bool device_ptrs = (flags & CCS_SCENE_DEVICE_PTRS) != 0;
    CCS_ARG(n_patches <= kMaxPatches, "n_patches above 2^26");
    CCS_ARG(n_patches == 0 || (x && y && z && types), "point or type array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    ccs_scene *sc = new (std::nothrow) ccs_scene();
    if (!sc) {
        set_error("host allocation failed");
        return CCS_ERR_OOM;
    }
    sc->n = n_patches;
    sc->local = (flags & CCS_SCENE_LOCAL_FRAMES) != 0;
    ccs_status st = CCS_OK;
    do {
        cudaError_t e;
        if ((e = cudaGetDevice(&sc->device)) != cudaSuccess) break;
        if ((e = cudaDeviceGetAttribute(&sc->num_sms, cudaDevAttrMultiProcessorCount, sc->device)) != cudaSuccess) break;
        const size_t np = (size_t)n_patches * 20;
        sc->hx.resize(np);
        sc->hy.resize(np);
        sc->hz.resize(np);
        sc->htypes.resize(n_patches);
        if ((e = cudaMalloc(&sc->d_work, kWorkWords * sizeof(uint32_t))) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(sc->d_work, 0, kWorkWords * sizeof(uint32_t), s)) != cudaSuccess) break;
        if (n_patches) {
            const cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
            if ((e = cudaMemcpy(sc->hx.data(), x, np * 4, k)) != cudaSuccess) break;
            if ((e = cudaMemcpy(sc->hy.data(), y, np * 4, k)) != cudaSuccess) break;
            if ((e = cudaMemcpy(sc->hz.data(), z, np * 4, k)) != cudaSuccess) break;
            if ((e = cudaMemcpy(sc->htypes.data(), types, n_patches, k)) != cudaSuccess) break;
            for (uint32_t i = 0; i < n_patches; ++i) {
                sc->htypes[i] = sc->htypes[i] ? 1 : 0;
                sc->n_greg += sc->htypes[i];
            }
            if ((e = cudaMalloc(&sc->d_rec, (size_t)n_patches * kRecF4 * sizeof(float4))) != cudaSuccess) break;
            if ((e = cudaMalloc(&sc->d_leaf_box, (size_t)n_patches * 2 * sizeof(float4))) != cudaSuccess) break;
            if ((e = cudaMalloc(&sc->d_types, n_patches)) != cudaSuccess) break;
            float *tmp = nullptr;
            if ((e = cudaMalloc(&tmp, np * 3 * 4)) != cudaSuccess) break;
            cudaMemcpyAsync(tmp, sc->hx.data(), np * 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(tmp + np, sc->hy.data(), np * 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(tmp + 2 * np, sc->hz.data(), np * 4, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(sc->d_types, sc->htypes.data(), n_patches, cudaMemcpyHostToDevice, s);
            e = launch_repack(tmp, tmp + np, tmp + 2 * np, sc->d_types, n_patches, sc->local ? 1 : 0, sc->d_rec,
                              sc->d_leaf_box, s);
            cudaError_t e2 = cudaStreamSynchronize(s);
            cudaFree(tmp);
            if (e == cudaSuccess) e = e2;
            if (e != cudaSuccess) break;
        }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        *out = sc;
        return CCS_OK;
    } while (0);
    cudaError_t e = cudaGetLastError();
    set_error(std::string("scene creation failed: ") + cudaGetErrorString(e));
    st = e == cudaErrorMemoryAllocation ? CCS_ERR_OOM : CCS_ERR_CUDA;
    free_scene(sc);
    return st;
}

ccs_status ccs_scene_destroy(ccs_scene *scene)
{
    if (!scene) return CCS_OK;
    free_scene(scene);
    return CCS_OK;
}

ccs_status ccs_scene_info(const ccs_scene *scene, uint32_t *n_patches, uint32_t *n_nodes)
{
    CCS_ARG(scene, "scene is NULL");
    if (n_patches) *n_patches = scene->n;
    if (n_nodes) *n_nodes = scene->n_nodes;
    return CCS_OK;
}

ccs_status ccs_bvh_build(ccs_scene *sc, const ccs_bvh_params *params)
{
    CCS_ARG(sc, "scene is NULL");
    int bins = params && params->bins ? (int)params->bins : 16;
    CCS_ARG(bins >= 4 && bins <= 64, "bins must be in 4..64");
    const uint32_t width = params && params->width ? params->width : 2;
    CCS_ARG(width == 2 || width == 4 || width == CCS_BVH_BOTH, "width must be 2, 4 or CCS_BVH_BOTH");
    const uint32_t n = sc->n;
    std::vector<float> lo(3 * (size_t)n), hi(3 * (size_t)n);
    for (uint32_t p = 0; p < n; ++p) {
        const int np = sc->htypes[p] ? 20 : 16;
        const float *pl[3] = {&sc->hx[20 * (size_t)p], &sc->hy[20 * (size_t)p], &sc->hz[20 * (size_t)p]};
        for (int c = 0; c < 3; ++c) {
            float a = pl[c][0], b = pl[c][0];
            for (int k = 1; k < np; ++k) {
                a = std::min(a, pl[c][k]);
                b = std::max(b, pl[c][k]);
            }
            lo[3 * (size_t)p + c] = a;
            hi[3 * (size_t)p + c] = b;
        }
    }
    BvhHost bin, wide;
    std::string err;
    if (!build_bvh(lo, hi, n, bins, bin, err)) {
        set_error(err);
        return CCS_ERR_INVALID_ARG;
    }
    if (width != 2 && !collapse_bvh4(bin, n, wide, err)) {
        set_error(err);
        return CCS_ERR_INVALID_ARG;
    }
    for (float4 **p : {&sc->d_nodes, &sc->d_nodes_alt}) {
        cudaFree(*p);
        *p = nullptr;
    }
    for (int **p : {&sc->d_leaf_parent, &sc->d_leaf_parent_alt}) {
        cudaFree(*p);
        *p = nullptr;
    }
    for (uint32_t **p : {&sc->d_refit_flags, &sc->d_refit_flags_alt}) {
        cudaFree(*p);
        *p = nullptr;
    }
    sc->n_nodes = sc->n_nodes_alt = 0;
    sc->alt_width = 0;
    sc->built = false;
    // upload one tree: nodes, leaf back-links and refit arrival counters
    auto upload = [n](const BvhHost &t, uint32_t per_node, float4 **nodes, int **parent, uint32_t **flags,
                      uint32_t *n_nodes) -> cudaError_t {
        *n_nodes = (uint32_t)(t.nodes.size() / per_node);
        if (*n_nodes == 0) return cudaSuccess;
        cudaError_t e;
        if ((e = cudaMalloc(nodes, t.nodes.size() * sizeof(float))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(*nodes, t.nodes.data(), t.nodes.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMalloc(parent, (size_t)n * sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(*parent, t.leaf_parent.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        return cudaMalloc(flags, (size_t)*n_nodes * sizeof(uint32_t));
    };
    if (width == 4) {
        CCS_CUDA(upload(wide, 32, &sc->d_nodes, &sc->d_leaf_parent, &sc->d_refit_flags, &sc->n_nodes));
        sc->bvh_width = 4;
    } else {
        CCS_CUDA(upload(bin, 16, &sc->d_nodes, &sc->d_leaf_parent, &sc->d_refit_flags, &sc->n_nodes));
        sc->bvh_width = 2;
    }
    if (width == CCS_BVH_BOTH) {
        CCS_CUDA(upload(wide, 32, &sc->d_nodes_alt, &sc->d_leaf_parent_alt, &sc->d_refit_flags_alt, &sc->n_nodes_alt));
        sc->alt_width = 4;
    }
    sc->built = true;
    return CCS_OK;
}

ccs_status ccs_scene_update_points(ccs_scene *sc, const float *x, const float *y, const float *z, void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    CCS_ARG(sc->n == 0 || (x && y && z), "point array is NULL");
    CCS_CUDA(launch_repack(x, y, z, sc->d_types, sc->n, sc->local ? 1 : 0, sc->d_rec, sc->d_leaf_box,
                           (cudaStream_t)stream));
    return CCS_OK;
}

ccs_status ccs_bvh_refit(ccs_scene *sc, void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    if (!sc->built) {
        set_error("ccs_bvh_refit before ccs_bvh_build");
        return CCS_ERR_NOT_BUILT;
    }
    CCS_CUDA(launch_refit(sc->d_nodes, sc->d_leaf_parent, sc->d_leaf_box, sc->d_refit_flags, sc->n, sc->n_nodes,
                          sc->bvh_width, (cudaStream_t)stream));
    if (sc->alt_width)
        CCS_CUDA(launch_refit(sc->d_nodes_alt, sc->d_leaf_parent_alt, sc->d_leaf_box, sc->d_refit_flags_alt, sc->n,
                              sc->n_nodes_alt, sc->alt_width, (cudaStream_t)stream));
    return CCS_OK;
}

ccs_status ccs_intersect(const ccs_scene *sc, const ccs_rays *rays, uint32_t n, ccs_hits *hits,
                         const ccs_trace_opts *opts, void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    ccs_status st = check_rays(rays, hits);
    if (st != CCS_OK) return st;
    if (!sc->built) {
        set_error("ccs_intersect before ccs_bvh_build");
        return CCS_ERR_NOT_BUILT;
    }
    LaunchCfg cfg;
    if ((st = fill_launch_cfg(opts, cfg)) != CCS_OK) return st;
    CCS_ARG(has_width(sc, cfg.bvh_width), "the scene has no BVH of the width opts->bvh_width asks for");
    if (cfg.pixel_spread > 0.0f) cfg.mode = 4;   // screen-space termination (one lane per ray)
    DevScene ds = dev_scene(sc, cfg.bvh_width);
    DevRays dr{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax};
    DevHits dh{hits->t, hits->u, hits->v, hits->patch_id};
    const uint32_t *perm;
    if ((st = work_order(sc, cfg, dr, n, (cudaStream_t)stream, &perm)) != CCS_OK) return st;
    CCS_CUDA(launch_intersect(ds, dr, dh, n, cfg, take_queue(const_cast<ccs_scene *>(sc)), sc->d_work + 1, sc->num_sms,
                              (cudaStream_t)stream, perm));
    return release_order(perm, (cudaStream_t)stream);
}

ccs_status ccs_trace_export(const ccs_scene *sc, const ccs_rays *rays, uint32_t n, ccs_hits *hits,
                            const ccs_trace_opts *opts, float *features, uint8_t *labels, uint32_t capacity,
                            uint32_t *count, void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    ccs_status st = check_rays(rays, hits);
    if (st != CCS_OK) return st;
    CCS_ARG(features && labels && count, "features, labels and count must be given");
    if (!sc->built) {
        set_error("ccs_trace_export before ccs_bvh_build");
        return CCS_ERR_NOT_BUILT;
    }
    LaunchCfg cfg;
    if ((st = fill_launch_cfg(opts, cfg)) != CCS_OK) return st;
    CCS_ARG(has_width(sc, cfg.bvh_width), "the scene has no BVH of the width opts->bvh_width asks for");
    CCS_ARG(cfg.leaf_depth >= 3, "trace export needs leaf_depth >= 3 (labels are depth-3 cells)");
    cfg.flags &= ~CCS_TRACE_COUNT;
    cfg.mode = 1;
    cfg.mc = ModeCtx{features, labels, count, capacity, nullptr, 0.0f};
    CCS_CUDA(cudaMemsetAsync(count, 0, sizeof(uint32_t), (cudaStream_t)stream));
    DevScene ds = dev_scene(sc, cfg.bvh_width);
    DevRays dr{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax};
    DevHits dh{hits->t, hits->u, hits->v, hits->patch_id};
    CCS_CUDA(launch_intersect(ds, dr, dh, n, cfg, take_queue(const_cast<ccs_scene *>(sc)), sc->d_work + 1, sc->num_sms,
                              (cudaStream_t)stream));
    return CCS_OK;
}

ccs_status ccs_intersect_learned(const ccs_scene *sc, const ccs_proposal *prop, const ccs_rays *rays, uint32_t n,
                                 ccs_hits *hits, const ccs_trace_opts *opts, float min_confidence, void *stream)
{
    CCS_ARG(sc && prop, "scene and proposal must not be NULL");
    ccs_status st = check_rays(rays, hits);
    if (st != CCS_OK) return st;
    if (!sc->built) {
        set_error("ccs_intersect_learned before ccs_bvh_build");
        return CCS_ERR_NOT_BUILT;
    }
    LaunchCfg cfg;
    if ((st = fill_launch_cfg(opts, cfg)) != CCS_OK) return st;
    CCS_ARG(has_width(sc, cfg.bvh_width), "the scene has no BVH of the width opts->bvh_width asks for");
    CCS_ARG(cfg.leaf_depth >= 3, "the learned proposal needs leaf_depth >= 3 (it proposes depth-3 cells)");
    CCS_ARG(cfg.block_threads == 128, "the learned proposal runs with 128 threads per block");
    cfg.mode = 2;
    cfg.cache_slots = 0;
    cfg.mlp = proposal_weights(prop);
    cfg.min_conf = min_confidence;
    DevScene ds = dev_scene(sc, cfg.bvh_width);
    DevRays dr{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax};
    DevHits dh{hits->t, hits->u, hits->v, hits->patch_id};
    CCS_CUDA(launch_intersect(ds, dr, dh, n, cfg, take_queue(const_cast<ccs_scene *>(sc)), sc->d_work + 1, sc->num_sms,
                              (cudaStream_t)stream));
    return CCS_OK;
}

ccs_status ccs_intersect_host(ccs_scene *sc, const ccs_rays *hr, uint32_t n, ccs_hits *hh, const ccs_trace_opts *opts,
                              void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    ccs_status st = check_rays(hr, hh);
    if (st != CCS_OK) return st;
    if (!sc->built) {
        set_error("ccs_intersect_host before ccs_bvh_build");
        return CCS_ERR_NOT_BUILT;
    }
    LaunchCfg cfg;
    if ((st = fill_launch_cfg(opts, cfg)) != CCS_OK) return st;
    CCS_ARG(has_width(sc, cfg.bvh_width), "the scene has no BVH of the width opts->bvh_width asks for");
    if (cfg.pixel_spread > 0.0f) cfg.mode = 4;
    if (n == 0) return CCS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // CCS_TRACE_HOST_MAPPED with mapped page-locked planes: the launch reads the rays and writes the hits
    // through the host memory's device mapping (NVLink-C2C on Grace systems), as one launch with no
    // staging copies.  Both ends of every plane must lie in one mapped allocation; anything else takes
    // the copies.
    auto mapped = [n](const void *p, void **dev) -> bool {
        const size_t last = (size_t)n * 4 - 1;
        cudaPointerAttributes a, z;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
            cudaPointerGetAttributes(&z, static_cast<const char *>(p) + last) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || z.type != cudaMemoryTypeHost || !a.devicePointer || !z.devicePointer)
            return false;
        if (static_cast<char *>(z.devicePointer) - static_cast<char *>(a.devicePointer) != (ptrdiff_t)last)
            return false;
        *dev = a.devicePointer;
        return true;
    };
    if (cfg.flags & CCS_TRACE_HOST_MAPPED) {
        const void *in[8] = {hr->ox, hr->oy, hr->oz, hr->dx, hr->dy, hr->dz, hr->tmin, hr->tmax};
        const void *out[4] = {hh->t, hh->u, hh->v, hh->patch_id};
        void *din[8], *dout[4];
        bool zc = true;
        for (int c = 0; c < 8 && zc; ++c) zc = mapped(in[c], &din[c]);
        for (int c = 0; c < 4 && zc; ++c) zc = mapped(out[c], &dout[c]);
        if (zc) {
            const DevRays dr{static_cast<const float *>(din[0]), static_cast<const float *>(din[1]),
                             static_cast<const float *>(din[2]), static_cast<const float *>(din[3]),
                             static_cast<const float *>(din[4]), static_cast<const float *>(din[5]),
                             static_cast<const float *>(din[6]), static_cast<const float *>(din[7])};
            const DevHits dh{static_cast<float *>(dout[0]), static_cast<float *>(dout[1]),
                             static_cast<float *>(dout[2]), static_cast<uint32_t *>(dout[3])};
            const uint32_t *perm;
            if ((st = work_order(sc, cfg, dr, n, s, &perm)) != CCS_OK) return st;
            CCS_CUDA(launch_intersect(dev_scene(sc, cfg.bvh_width), dr, dh, n, cfg, take_queue(sc), sc->d_work + 1, sc->num_sms, s,
                                      perm));
            if ((st = release_order(perm, s)) != CCS_OK) return st;
            CCS_CUDA(cudaStreamSynchronize(s));
            return CCS_OK;
        }
    }
    const HostBatch one{hr, n, hh, cfg};
    return host_pipeline(sc, &one, 1, s);
}

ccs_status ccs_intersect_host_batches(ccs_scene *sc, uint32_t n_batches, const ccs_rays *hr, const uint32_t *n,
                                      ccs_hits *hh, const ccs_trace_opts *const *opts, void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    CCS_ARG(n_batches == 0 || (hr && n && hh), "rays, n and hits must be given when n_batches > 0");
    if (!sc->built) {
        set_error("ccs_intersect_host_batches before ccs_bvh_build");
        return CCS_ERR_NOT_BUILT;
    }
    // every batch is checked before any work is queued
    std::vector<HostBatch> bt(n_batches);
    for (uint32_t j = 0; j < n_batches; ++j) {
        ccs_status st = check_rays(&hr[j], &hh[j]);
        if (st != CCS_OK) return st;
        LaunchCfg cfg;
        if ((st = fill_launch_cfg(opts ? opts[j] : nullptr, cfg)) != CCS_OK) return st;
        CCS_ARG(has_width(sc, cfg.bvh_width), "the scene has no BVH of the width opts->bvh_width asks for");
        if (cfg.pixel_spread > 0.0f) cfg.mode = 4;
        bt[j] = HostBatch{&hr[j], n[j], &hh[j], cfg};
    }
    return host_pipeline(sc, bt.data(), n_batches, (cudaStream_t)stream);
}

static ccs_status gen_secondary(const ccs_scene *sc, const ccs_rays *in, const ccs_hits *hits, uint32_t n, uint64_t seed,
                                uint32_t leaf_depth, float offset_abs, ccs_rays *out, int kind, const float *light,
                                void *stream)
{
    CCS_ARG(sc && out, "scene and out_rays must not be NULL");
    ccs_status st = check_rays(in, hits);
    if (st != CCS_OK) return st;
    CCS_ARG(out->ox && out->dx && out->tmin && out->tmax, "an output plane is NULL");
    CCS_ARG(out->oy == out->ox + n && out->oz == out->ox + 2 * (size_t)n && out->dy == out->dx + n &&
                out->dz == out->dx + 2 * (size_t)n,
            "output origin and direction planes must each be one contiguous block of 3n floats");
    CCS_ARG(leaf_depth >= 1 && leaf_depth <= (uint32_t)kMaxLeafDepth, "leaf_depth must be in 1..15");
    if (n == 0) return CCS_OK;
    DevRays dr{in->ox, in->oy, in->oz, in->dx, in->dy, in->dz, in->tmin, in->tmax};
    DevHits dh{hits->t, hits->u, hits->v, hits->patch_id};
    CCS_CUDA(launch_gen_diffuse(sc->d_rec, sc->d_leaf_box, sc->n, dr, dh, n, seed, (int)leaf_depth, offset_abs,
                                const_cast<float *>(out->ox), const_cast<float *>(out->dx),
                                const_cast<float *>(out->tmin), const_cast<float *>(out->tmax), kind, light,
                                sc->local ? 1 : 0, (cudaStream_t)stream));
    return CCS_OK;
}

ccs_status ccs_gen_diffuse(const ccs_scene *sc, const ccs_rays *in, const ccs_hits *hits, uint32_t n, uint64_t seed,
                           uint32_t leaf_depth, float offset_abs, ccs_rays *out, void *stream)
{
    return gen_secondary(sc, in, hits, n, seed, leaf_depth, offset_abs, out, 0, nullptr, stream);
}

ccs_status ccs_gen_mirror(const ccs_scene *sc, const ccs_rays *in, const ccs_hits *hits, uint32_t n,
                          uint32_t leaf_depth, float offset_abs, ccs_rays *out, void *stream)
{
    return gen_secondary(sc, in, hits, n, 0, leaf_depth, offset_abs, out, 1, nullptr, stream);
}

ccs_status ccs_gen_shadow(const ccs_scene *sc, const ccs_rays *in, const ccs_hits *hits, uint32_t n, const float *light,
                          uint32_t leaf_depth, float offset_abs, ccs_rays *out, void *stream)
{
    CCS_ARG(light, "light must not be NULL");
    CCS_ARG(std::isfinite(light[0]) && std::isfinite(light[1]) && std::isfinite(light[2]), "light must be finite");
    return gen_secondary(sc, in, hits, n, 0, leaf_depth, offset_abs, out, 2, light, stream);
}

ccs_status ccs_occluded(const ccs_scene *sc, const ccs_rays *rays, uint32_t n, uint8_t *occluded,
                        const ccs_trace_opts *opts, void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    CCS_ARG(rays && rays->ox && rays->oy && rays->oz && rays->dx && rays->dy && rays->dz && rays->tmin && rays->tmax,
            "a ray plane is NULL");
    CCS_ARG(occluded || n == 0, "occluded must not be NULL");
    if (!sc->built) {
        set_error("ccs_occluded before ccs_bvh_build");
        return CCS_ERR_NOT_BUILT;
    }
    ccs_status st;
    LaunchCfg cfg;
    if ((st = fill_launch_cfg(opts, cfg)) != CCS_OK) return st;
    CCS_ARG(has_width(sc, cfg.bvh_width), "the scene has no BVH of the width opts->bvh_width asks for");
    cfg.mode = 3;
    cfg.mc.occluded = occluded;
    DevScene ds = dev_scene(sc, cfg.bvh_width);
    DevRays dr{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->tmin, rays->tmax};
    DevHits dh{nullptr, nullptr, nullptr, nullptr};
    const uint32_t *perm;
    if ((st = work_order(sc, cfg, dr, n, (cudaStream_t)stream, &perm)) != CCS_OK) return st;
    CCS_CUDA(launch_intersect(ds, dr, dh, n, cfg, take_queue(const_cast<ccs_scene *>(sc)), sc->d_work + 1, sc->num_sms,
                              (cudaStream_t)stream, perm));
    return release_order(perm, (cudaStream_t)stream);
}

ccs_status ccs_scene_sync_status(ccs_scene *sc, void *stream)
{
    CCS_ARG(sc, "scene is NULL");
    CCS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t w = 0;
    CCS_CUDA(cudaMemcpy(&w, sc->d_work + 1, 4, cudaMemcpyDeviceToHost));
    if (w) {
        CCS_CUDA(cudaMemset(sc->d_work + 1, 0, 4));
        set_error("a ray reached the traversal iteration cap and was written as a miss");
        return CCS_ERR_TRAVERSAL_LIMIT;
    }
    return CCS_OK;
}

}  // extern "C"
