// Pair engine subdivision pass for one scene, any hit (shadow rays).
#include "pairs_launch.cuh"

namespace ccs {

cudaError_t pair_passes_single_anyhit(const SingleSource &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n,
                                      uint32_t *status, int num_sms, cudaStream_t s)
{
    return launch_pair_passes<kModeAnyHit, SingleSource>(src, pb, cfg, n, status, num_sms, s);
}

}  // namespace ccs
