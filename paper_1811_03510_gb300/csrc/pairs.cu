// The pair engine's launch sequence (CCS_TRACE_PAIRS): counters zeroed, the candidate pass (which also
// lists each task under its cost class), then the subdivision pass.  One scene takes its scratch from the
// library's stream-ordered memory pool on the launch's stream; a batch brings its own, allocated with the
// batch, so that its run stays capturable in a CUDA graph.
#include <mutex>

#include "pairs_launch.cuh"

namespace ccs {

bool use_pairs(const LaunchCfg &cfg)
{
    return (cfg.flags & CCS_TRACE_PAIRS) && (cfg.mode == kModePlain || cfg.mode == kModeAnyHit) &&
           cfg.lanes_per_ray == 1;
}

size_t pairs_scratch_bytes(uint32_t n) { return pair_scratch_bytes(n); }

namespace {

// The library's memory pool of the current device (created on first use; freed memory stays in the pool).
cudaError_t pair_pool(cudaMemPool_t *out)
{
    constexpr int kMaxDevices = 64;
    static cudaMemPool_t pools[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if ((e = cudaMemPoolCreate(&p, &props)) != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        if ((e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        pools[dev] = p;
    }
    *out = pools[dev];
    return cudaSuccess;
}

template <bool STATS, int MODE, class Src, int BW>
cudaError_t launch_cand(const Src &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n, uint32_t *status,
                        cudaStream_t s)
{
    // 8 x 4 pixel tiles per warp when the rays are an image whose width is a multiple of 8
    const uint32_t img_w = (cfg.image_width & 7u) == 0u ? cfg.image_width : 0u;
    const uint32_t t = cand_threads(n, img_w);
    k_cand<STATS, MODE, Src, BW><<<(t + kCandBlock - 1) / kCandBlock, kCandBlock, 0, s>>>(
        src, pb, img_w, cfg.iter_cap, status, cfg.counters, cfg.mc.occluded);
    return cudaGetLastError();
}

template <int MODE, class Src>
cudaError_t cand_pass(const Src &src, const PairBufs &pb, const LaunchCfg &cfg, uint32_t n, uint32_t width,
                      uint32_t *status, cudaStream_t s)
{
    const bool stats = (cfg.flags & CCS_TRACE_COUNT) != 0;
    if (width == 4)
        return stats ? launch_cand<true, MODE, Src, 4>(src, pb, cfg, n, status, s)
                     : launch_cand<false, MODE, Src, 4>(src, pb, cfg, n, status, s);
    return stats ? launch_cand<true, MODE, Src, 2>(src, pb, cfg, n, status, s)
                 : launch_cand<false, MODE, Src, 2>(src, pb, cfg, n, status, s);
}

}  // namespace

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s)
{
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = pair_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t pool_free(void *p, cudaStream_t s) { return cudaFreeAsync(p, s); }

cudaError_t launch_pairs_single(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n,
                                const LaunchCfg &cfg, uint32_t *status, int num_sms, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    void *base = nullptr;
    cudaError_t e = pool_alloc(&base, pair_scratch_bytes(n), s);
    if (e != cudaSuccess) return e;
    const PairBufs pb = pair_bufs_at(base, n);
    const SingleSource src{sc, r, h, n, nullptr};
    e = cudaMemsetAsync(pb.ctr, 0, kPairCtrWords * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        if (cfg.mode == kModeAnyHit) {
            e = cand_pass<kModeAnyHit>(src, pb, cfg, n, sc.width, status, s);
            if (e == cudaSuccess) e = pair_passes_single_anyhit(src, pb, cfg, n, status, num_sms, s);
        } else {
            e = cand_pass<kModePlain>(src, pb, cfg, n, sc.width, status, s);
            if (e == cudaSuccess) e = pair_passes_single_plain(src, pb, cfg, n, status, num_sms, s);
        }
    }
    const cudaError_t e2 = pool_free(base, s);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_pairs_batch(const BatchEntry *entries, const uint32_t *ray_prefix, uint32_t n_scenes,
                               uint32_t n_total, const LaunchCfg &cfg, void *scratch,
                               uint32_t *status, int num_sms, cudaStream_t s, uint32_t width)
{
    if (n_total == 0) return cudaSuccess;
    const PairBufs pb = pair_bufs_at(scratch, n_total);
    const BatchSource src{entries, ray_prefix, n_scenes, n_total};
    cudaError_t e = cudaMemsetAsync(pb.ctr, 0, kPairCtrWords * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if ((e = cand_pass<kModePlain>(src, pb, cfg, n_total, width, status, s)) != cudaSuccess) return e;
    return pair_passes_batch(src, pb, cfg, n_total, status, num_sms, s);
}

}  // namespace ccs
