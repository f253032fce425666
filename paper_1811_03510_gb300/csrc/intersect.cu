// Closest-hit launches over binary BVHs, and the entry points that pick the kernels of the scene's BVH
// width (the 4-wide ones are instantiated in intersect4.cu).
#include "intersect_impl.cuh"

namespace ccs {

template cudaError_t launch_single_w<2>(const DevScene &, const DevRays &, const DevHits &, uint32_t,
                                        const LaunchCfg &, uint32_t *, uint32_t *, int, cudaStream_t,
                                        const uint32_t *);
template cudaError_t launch_batch_w<2>(const BatchEntry *, const uint32_t *, uint32_t, uint32_t, const LaunchCfg &,
                                       uint32_t *, uint32_t *, int, cudaStream_t);
extern template cudaError_t launch_single_w<4>(const DevScene &, const DevRays &, const DevHits &, uint32_t,
                                               const LaunchCfg &, uint32_t *, uint32_t *, int, cudaStream_t,
                                               const uint32_t *);
extern template cudaError_t launch_batch_w<4>(const BatchEntry *, const uint32_t *, uint32_t, uint32_t,
                                              const LaunchCfg &, uint32_t *, uint32_t *, int, cudaStream_t);

cudaError_t launch_intersect(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n, const LaunchCfg &cfg,
                             uint32_t *queue, uint32_t *status, int num_sms, cudaStream_t s, const uint32_t *perm)
{
    if (use_pairs(cfg)) return launch_pairs_single(sc, r, h, n, cfg, status, num_sms, s);
    return sc.width == 4 ? launch_single_w<4>(sc, r, h, n, cfg, queue, status, num_sms, s, perm)
                         : launch_single_w<2>(sc, r, h, n, cfg, queue, status, num_sms, s, perm);
}

cudaError_t launch_intersect_batch(const BatchEntry *entries, const uint32_t *ray_prefix, uint32_t n_scenes,
                                   uint32_t n_total, const LaunchCfg &cfg, uint32_t *queue, uint32_t *status,
                                   int num_sms, cudaStream_t s, uint32_t width)
{
    return width == 4 ? launch_batch_w<4>(entries, ray_prefix, n_scenes, n_total, cfg, queue, status, num_sms, s)
                      : launch_batch_w<2>(entries, ray_prefix, n_scenes, n_total, cfg, queue, status, num_sms, s);
}

}  // namespace ccs
