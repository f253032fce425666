// Closest-hit launches over 4-wide BVHs (the kernels of intersect_impl.cuh with BW = 4).
#include "intersect_impl.cuh"

namespace ccs {

template cudaError_t launch_single_w<4>(const DevScene &, const DevRays &, const DevHits &, uint32_t,
                                        const LaunchCfg &, uint32_t *, uint32_t *, int, cudaStream_t,
                                        const uint32_t *);
template cudaError_t launch_batch_w<4>(const BatchEntry *, const uint32_t *, uint32_t, uint32_t, const LaunchCfg &,
                                       uint32_t *, uint32_t *, int, cudaStream_t);

}  // namespace ccs
