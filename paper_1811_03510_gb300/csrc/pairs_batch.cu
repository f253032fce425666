// Pair engine subdivision pass for a batch of scenes, closest hit.
#include "pairs_launch.cuh"

namespace ccs {

cudaError_t pair_passes_batch(const BatchSource &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n,
                              uint32_t *status, int num_sms, cudaStream_t s)
{
    return launch_pair_passes<kModePlain, BatchSource>(src, pb, cfg, n, status, num_sms, s);
}

}  // namespace ccs
