// Plain closest-hit kernel: persistent blocks, warps take chunks of rays from a global work queue,
// each lane traverses the BVH and runs the bit-trail patch subdivision (Algorithm 3) at its leaves.
#include "traverse.cuh"

namespace ccs {

template <bool STATS>
__global__ void __launch_bounds__(128) k_intersect(DevScene sc, DevRays rays, DevHits hits, uint32_t n, int L,
                                                   uint32_t chunk, uint32_t iter_cap, uint32_t *queue,
                                                   uint32_t *status, unsigned long long *counters)
{
    extern __shared__ float2 sib_smem[];
    float2 *sib = sib_smem + threadIdx.x;
    const int stride = blockDim.x;
    Counters cnt;
#pragma unroll
    for (int k = 0; k < kNumCounters; ++k) cnt.v[k] = 0;
    const int lane = threadIdx.x & 31;
    const float cellw = __int_as_float((127 - L) << 23);
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(queue, chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const uint32_t end = min(base + chunk, n);
        for (uint32_t i = base + lane; i < end; i += 32) {
            Best b;
            const bool ok = trace_ray<STATS>(sc, __ldg(rays.ox + i), __ldg(rays.oy + i), __ldg(rays.oz + i),
                                             __ldg(rays.dx + i), __ldg(rays.dy + i), __ldg(rays.dz + i),
                                             __ldg(rays.tmin + i), __ldg(rays.tmax + i), L, b, sib, stride, iter_cap,
                                             cnt);
            if (!ok) {
                atomicOr(status, 1u);
                b.pid = kMissId;
            }
            if (b.pid != kMissId) {
                const uint32_t cu = b.cell & ((1u << L) - 1u), cv = b.cell >> L;
                hits.t[i] = b.t;
                hits.u[i] = ((float)cu + 0.5f) * cellw;
                hits.v[i] = ((float)cv + 0.5f) * cellw;
                hits.pid[i] = b.pid;
            } else {
                hits.t[i] = __int_as_float(0x7f800000);
                hits.u[i] = 0.0f;
                hits.v[i] = 0.0f;
                hits.pid[i] = kMissId;
            }
        }
    }
    if (STATS) {
#pragma unroll
        for (int k = 0; k < kNumCounters; ++k) {
            unsigned long long v = cnt.v[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicAdd(counters + k, v);
        }
    }
}

cudaError_t launch_intersect(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n, const LaunchCfg &cfg,
                             uint32_t *queue, uint32_t *status, int num_sms, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const uint32_t threads = cfg.block_threads;
    const size_t smem = (size_t)threads * 2 * cfg.leaf_depth * sizeof(float2);
    const uint32_t warps_needed = (n + cfg.chunk - 1) / cfg.chunk;
    uint32_t blocks = (uint32_t)num_sms * cfg.blocks_per_sm;
    const uint32_t blocks_needed = (warps_needed * 32 + threads - 1) / threads;
    if (blocks > blocks_needed) blocks = blocks_needed;
    if (blocks == 0) blocks = 1;
    if (cfg.flags & CCS_TRACE_COUNT) {
        k_intersect<true><<<blocks, threads, smem, s>>>(sc, r, h, n, (int)cfg.leaf_depth,
                                                        cfg.chunk, cfg.iter_cap, queue, status, cfg.counters);
    } else {
        k_intersect<false><<<blocks, threads, smem, s>>>(sc, r, h, n, (int)cfg.leaf_depth, cfg.chunk, cfg.iter_cap,
                                                         queue, status, cfg.counters);
    }
    return cudaGetLastError();
}

}  // namespace ccs
