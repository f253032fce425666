// Plain closest-hit kernel.  Persistent blocks; each warp keeps 32 rays in flight and takes new rays
// from a global work queue whenever enough of its lanes are idle (warp-aggregated atomic).  Each
// iteration of the warp loop advances every lane by one unit of work (lane_step), so lanes in
// different phases (BVH, subdivision, re-descent) cost one step each instead of serialising whole
// patch traversals.
#include "traverse.cuh"

namespace ccs {

template <bool STATS, int K, int MINB>
__global__ void __launch_bounds__(128, MINB) k_intersect(DevScene sc, DevRays rays, DevHits hits, uint32_t n, int L,
                                                   uint32_t refill, uint32_t chunk, int burst, uint32_t iter_cap,
                                                   uint32_t *queue, uint32_t *status, unsigned long long *counters)
{
    extern __shared__ float smem[];
    const int stride = blockDim.x;
    Scratch scr;
    scr.stride = stride;
    scr.sib = reinterpret_cast<float2 *>(smem) + threadIdx.x;
    scr.cache = smem + 2 * 2 * L * stride + threadIdx.x;
    scr.tag = reinterpret_cast<int *>(smem + (2 * 2 * L + 48 * K) * stride) + threadIdx.x;
    Counters cnt;
#pragma unroll
    for (int k = 0; k < kNumCounters; ++k) cnt.v[k] = 0;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float cellw = __int_as_float((127 - L) << 23);
    Lane s;
    BvhStack stk;
    float g[48];
    bool has = false, exhausted = false;
    uint32_t ray_i = 0;
    uint32_t wnext = 0, wend = 0;   // warp-uniform range of rays taken from the queue, not yet handed out
    for (;;) {
        const unsigned idle = __ballot_sync(FULL, !has);
        if (idle != 0u && ((uint32_t)__popc(idle) >= refill || idle == FULL)) {
            if (wnext == wend && !exhausted) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(queue, chunk);
                base = __shfl_sync(FULL, base, 0);
                if (base >= n) {
                    exhausted = true;
                } else {
                    wnext = base;
                    wend = min(base + chunk, n);
                }
            }
            const uint32_t avail = wend - wnext;
            const uint32_t rank = (uint32_t)__popc(idle & lt_mask);
            if (!has && rank < avail) {
                const uint32_t i = wnext + rank;
                has = true;
                ray_i = i;
                begin_ray(s, sc, __ldg(rays.ox + i), __ldg(rays.oy + i), __ldg(rays.oz + i), __ldg(rays.dx + i),
                          __ldg(rays.dy + i), __ldg(rays.dz + i), __ldg(rays.tmin + i), __ldg(rays.tmax + i), iter_cap);
            }
            const uint32_t taken = avail < (uint32_t)__popc(idle) ? avail : (uint32_t)__popc(idle);
            wnext += taken;
        }
        if (__ballot_sync(FULL, has) == 0u) {
            if (exhausted && wnext == wend) break;
            continue;
        }
        if (has) {
            const bool ok = lane_step<STATS, K>(s, g, stk, sc, L, scr, cnt, burst);
            if (!ok || lane_done(s)) {
                if (!ok) {
                    atomicOr(status, 1u);
                    s.best.pid = kMissId;
                }
                const uint32_t i = ray_i;
                if (s.best.pid != kMissId) {
                    const uint32_t cu = s.best.cell & ((1u << L) - 1u), cv = s.best.cell >> L;
                    hits.t[i] = s.best.t;
                    hits.u[i] = ((float)cu + 0.5f) * cellw;
                    hits.v[i] = ((float)cv + 0.5f) * cellw;
                    hits.pid[i] = s.best.pid;
                } else {
                    hits.t[i] = __int_as_float(0x7f800000);
                    hits.u[i] = 0.0f;
                    hits.v[i] = 0.0f;
                    hits.pid[i] = kMissId;
                }
                has = false;
            }
        }
    }
    if (STATS) {
#pragma unroll
        for (int k = 0; k < kNumCounters; ++k) {
            unsigned long long v = cnt.v[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            if (lane == 0 && v) atomicAdd(counters + k, v);
        }
    }
}

size_t intersect_smem_bytes(uint32_t threads, uint32_t L, uint32_t K)
{
    return (size_t)threads * (2 * 2 * L + 48 * K + K) * sizeof(float);
}

template <bool STATS, int K, int MINB>
static cudaError_t launch_one(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n, const LaunchCfg &cfg,
                              uint32_t *queue, uint32_t *status, int num_sms, cudaStream_t s)
{
    auto kern = k_intersect<STATS, K, MINB>;
    const uint32_t threads = cfg.block_threads;
    const size_t smem = intersect_smem_bytes(threads, cfg.leaf_depth, K);
    static size_t configured = 0;   // largest dynamic shared memory size set on this instantiation
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int max_active = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_active, kern, (int)threads, smem);
    if (e != cudaSuccess) return e;
    if (max_active < 1) return cudaErrorInvalidConfiguration;
    uint32_t per_sm = cfg.blocks_per_sm < (uint32_t)max_active ? cfg.blocks_per_sm : (uint32_t)max_active;
    uint32_t blocks = (uint32_t)num_sms * per_sm;
    const uint32_t needed = (n + threads - 1) / threads;
    if (blocks > needed) blocks = needed;
    if (blocks == 0) blocks = 1;
    kern<<<blocks, threads, smem, s>>>(sc, r, h, n, (int)cfg.leaf_depth, cfg.refill, cfg.chunk, (int)cfg.bvh_burst,
                                       cfg.iter_cap, queue, status, cfg.counters);
    return cudaGetLastError();
}

cudaError_t launch_intersect(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n, const LaunchCfg &cfg,
                             uint32_t *queue, uint32_t *status, int num_sms, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const bool stats = (cfg.flags & CCS_TRACE_COUNT) != 0;
    if (stats)   // counting runs are not timed: one register budget is enough
        return cfg.cache_slots == 0 ? launch_one<true, 0, 1>(sc, r, h, n, cfg, queue, status, num_sms, s)
                                    : launch_one<true, 2, 1>(sc, r, h, n, cfg, queue, status, num_sms, s);
    if (cfg.min_blocks >= 4)
        return cfg.cache_slots == 0 ? launch_one<false, 0, 4>(sc, r, h, n, cfg, queue, status, num_sms, s)
                                    : launch_one<false, 2, 4>(sc, r, h, n, cfg, queue, status, num_sms, s);
    return cfg.cache_slots == 0 ? launch_one<false, 0, 1>(sc, r, h, n, cfg, queue, status, num_sms, s)
                                : launch_one<false, 2, 1>(sc, r, h, n, cfg, queue, status, num_sms, s);
}

}  // namespace ccs
