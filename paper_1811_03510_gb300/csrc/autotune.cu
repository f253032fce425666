// Autotuner of the closest-hit launch: coordinate descent over options that cannot change the answer
// (BVH width when the scene holds two, the engine: ray-persistent kernel with or without the work order,
// or the pair engine; lanes per ray, phase vote, threads per block, blocks per SM, warp refill threshold,
// queue chunk, BVH burst, sibling cache, register budget),
// each candidate timed with CUDA events over `reps` launches on the caller's rays.
#include <cuda_runtime.h>

#include <cfloat>
#include <string>
#include <vector>

#include "ccs_internal.h"

using namespace ccs;

extern "C" {

ccs_status ccs_autotune(const ccs_scene *scene, const ccs_rays *rays, uint32_t n, ccs_hits *hits,
                        const ccs_trace_opts *base, uint32_t reps, ccs_trace_opts *best, float *best_ms,
                        ccs_autotune_trial *trials, uint32_t max_trials, uint32_t *n_trials, void *stream)
{
    if (!scene || !rays || !hits || !best || n == 0) {
        set_error("ccs_autotune: scene, rays, hits and best must be given and n > 0");
        return CCS_ERR_INVALID_ARG;
    }
    if (reps == 0) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    ccs_trace_opts cur{};
    if (base) cur = *base;
    cur.flags &= CCS_TRACE_ORDER | CCS_TRACE_PAIRS;
    cur.counters = nullptr;
    if (!cur.leaf_depth) cur.leaf_depth = 8;
    if (!cur.block_threads) cur.block_threads = 128;
    if (!cur.blocks_per_sm) cur.blocks_per_sm = 4;
    if (!cur.refill) cur.refill = 8;
    if (!cur.chunk) cur.chunk = 32;
    if (!cur.bvh_burst) cur.bvh_burst = 8;
    if (cur.cache_slots == CCS_CACHE_DEFAULT) cur.cache_slots = 2;
    if (!cur.lanes_per_ray) cur.lanes_per_ray = 1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_error("ccs_autotune: cudaEventCreate failed");
        return CCS_ERR_CUDA;
    }
    uint32_t count = 0;
    auto measure = [&](const ccs_trace_opts &o, float &ms) -> ccs_status {
        ccs_status st = ccs_intersect(scene, rays, n, hits, &o, stream);   // warm-up
        if (st != CCS_OK) return st;
        cudaEventRecord(e0, s);
        for (uint32_t r = 0; r < reps; ++r)
            if ((st = ccs_intersect(scene, rays, n, hits, &o, stream)) != CCS_OK) return st;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("ccs_autotune: launch failed");
            return CCS_ERR_CUDA;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (trials && count < max_trials) {
            trials[count].opts = o;
            trials[count].ms = ms;
        }
        ++count;
        return CCS_OK;
    };
    float cur_ms = FLT_MAX;
    ccs_status st = measure(cur, cur_ms);
    const std::vector<uint32_t> threads_c = {64, 96, 128};
    const std::vector<uint32_t> lanes_c = {1, 3};
    const std::vector<uint32_t> bps_c = {1, 2, 3, 4, 5, 6};
    const std::vector<uint32_t> refill_c = {1, 2, 4, 8, 16, 24};
    const std::vector<uint32_t> chunk_c = {32, 64, 128, 256, 512, 1024};
    const std::vector<uint32_t> burst_c = {1, 2, 4, 8, 16};
    const std::vector<uint32_t> cache_c = {0, 1, 2};
    const std::vector<uint32_t> minb_c = {0, 4};
    const std::vector<uint32_t> vote_c = {0, 4, 8, 12, 16, 20, 24};
    const std::vector<uint32_t> order_c = {0, CCS_TRACE_ORDER, CCS_TRACE_PAIRS};
    std::vector<uint32_t> width_c = {0};   // the scene's default BVH, and its second one if it has one
    if (scene->alt_width) width_c.push_back(scene->alt_width);
    const std::vector<uint32_t> *cands[11] = {&width_c, &order_c, &lanes_c, &vote_c, &threads_c, &bps_c, &refill_c,
                                              &chunk_c, &burst_c, &cache_c, &minb_c};
    for (int pass = 0; pass < 2 && st == CCS_OK; ++pass) {
        for (int knob = 0; knob < 11 && st == CCS_OK; ++knob) {
            for (uint32_t v : *cands[knob]) {
                ccs_trace_opts o = cur;
                uint32_t *fields[11] = {&o.bvh_width, &o.flags, &o.lanes_per_ray, &o.vote, &o.block_threads,
                                        &o.blocks_per_sm, &o.refill, &o.chunk, &o.bvh_burst, &o.cache_slots,
                                        &o.min_blocks};
                uint32_t *field = fields[knob];
                if (*field == v) continue;
                *field = v;
                float ms = FLT_MAX;
                if ((st = measure(o, ms)) != CCS_OK) break;
                if (ms < cur_ms) {
                    cur_ms = ms;
                    cur = o;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CCS_OK) return st;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    if (n_trials) *n_trials = count;
    return CCS_OK;
}

}  // extern "C"
