// Launches of the pair engine's subdivision pass (k_pairs), shared by the translation units that
// instantiate them: pairs_plain.cu (one scene, closest hit), pairs_anyhit.cu (one scene, any hit) and
// pairs_batch.cu (a batch of scenes, closest hit).
#pragma once

#include "pairs.cuh"

namespace ccs {

template <bool STATS, int K, int MODE, class Src>
cudaError_t launch_pair_pass(const Src &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n, uint32_t *status,
                             int num_sms, cudaStream_t s)
{
    auto kern = k_pairs<STATS, K, MODE, Src>;
    constexpr uint32_t threads = 128;
    const size_t smem =
        (size_t)threads * (scratch_floats((int)cfg.leaf_depth, K, 3) + kRaySlotFloats + kHelpFloats) * sizeof(float);
    static size_t configured = 0;   // largest dynamic shared memory size set on this instantiation
    static size_t occ_smem = 0;
    static int occ_active = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    if (occ_smem != smem) {
        int a = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, kern, (int)threads, smem);
        if (e != cudaSuccess) return e;
        occ_smem = smem;
        occ_active = a;
    }
    if (occ_active < 1) return cudaErrorInvalidConfiguration;
    uint32_t blocks = (uint32_t)num_sms * (uint32_t)occ_active;
    const uint32_t needed = (n + threads - 1) / threads;   // tasks of one kind are at most one per ray
    if (blocks > needed) blocks = needed;
    if (blocks == 0) blocks = 1;
    kern<<<blocks, threads, smem, s>>>(src, pb, (int)cfg.leaf_depth, cfg.refill, cfg.iter_cap, status, cfg.counters,
                                       cfg.mc.occluded);
    return cudaGetLastError();
}

// The subdivision pass with the launch's sibling cache.
template <int MODE, class Src>
cudaError_t launch_pair_passes(const Src &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n, uint32_t *status,
                               int num_sms, cudaStream_t s)
{
    const uint32_t K = cfg.cache_slots;
    if (cfg.flags & CCS_TRACE_COUNT)
        return K == 0 ? launch_pair_pass<true, 0, MODE, Src>(src, pb, cfg, n, status, num_sms, s)
             : K == 1 ? launch_pair_pass<true, 1, MODE, Src>(src, pb, cfg, n, status, num_sms, s)
                      : launch_pair_pass<true, 2, MODE, Src>(src, pb, cfg, n, status, num_sms, s);
    return K == 0 ? launch_pair_pass<false, 0, MODE, Src>(src, pb, cfg, n, status, num_sms, s)
         : K == 1 ? launch_pair_pass<false, 1, MODE, Src>(src, pb, cfg, n, status, num_sms, s)
                  : launch_pair_pass<false, 2, MODE, Src>(src, pb, cfg, n, status, num_sms, s);
}

cudaError_t pair_passes_single_plain(const SingleSource &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n,
                                     uint32_t *status, int num_sms, cudaStream_t s);
cudaError_t pair_passes_single_anyhit(const SingleSource &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n,
                                      uint32_t *status, int num_sms, cudaStream_t s);
cudaError_t pair_passes_batch(const BatchSource &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n,
                              uint32_t *status, int num_sms, cudaStream_t s);

}  // namespace ccs
