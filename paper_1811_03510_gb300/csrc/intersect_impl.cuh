// Closest-hit kernels.  Persistent blocks; each warp keeps 32 rays in flight, takes ranges of rays from
// a global work queue and hands them to its idle lanes.  Each iteration of the warp loop advances every
// lane by one unit of work (lane_step), so lanes in different phases (BVH, subdivision, re-descent)
// cost one step each instead of serialising whole patch traversals.  The same loop serves one scene
// (SingleSource) or a table of scenes whose rays share one queue (BatchSource, batched launches).
//
// Shared by the translation units that instantiate the kernels for binary (intersect.cu) and 4-wide
// (intersect4.cu) BVHs.
#pragma once
#include <type_traits>

#include "traverse.cuh"

namespace ccs {

// Device clock in nanoseconds (the timeline counters of a counting launch).
CCS_DEV unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Rays of one scene (the scene descriptor stays in kernel-parameter space, uniform over lanes).
struct SingleSource {
    DevScene sc;
    DevRays rays;
    DevHits hits;
    uint32_t n;
    const uint32_t *perm;   // queue position -> ray index (work order), or null for the identity
    struct LaneScene {};
    CCS_DEV uint32_t total() const { return n; }
    CCS_DEV const DevScene &scene(const LaneScene &) const { return sc; }
    CCS_DEV void locate(uint32_t i, LaneScene &, uint32_t &scene, uint32_t &local) const
    {
        scene = 0;
        local = perm ? __ldg(perm + i) : i;
    }
    CCS_DEV const DevRays &rays_of(uint32_t) const { return rays; }
    CCS_DEV const DevHits &hits_of(uint32_t) const { return hits; }
};

// Rays of many scenes, concatenated in scene order (ray_prefix[s] = first global index of scene s).
struct BatchSource {
    const BatchEntry *entries;
    const uint32_t *ray_prefix;   // n_scenes + 1
    uint32_t n_scenes, n;
    struct LaneScene {
        uint32_t s = 0;   // the scene of the lane's ray: its descriptor is read from the table where used, so
                          // that a lane does not hold a copy of it in registers
    };
    CCS_DEV uint32_t total() const { return n; }
    CCS_DEV const DevScene &scene(const LaneScene &l) const { return entries[l.s].sc; }
    CCS_DEV void locate(uint32_t i, LaneScene &lsc, uint32_t &scene, uint32_t &local) const
    {
        uint32_t lo = 0, hi = n_scenes;   // largest s with ray_prefix[s] <= i
        while (hi - lo > 1) {
            const uint32_t m = (lo + hi) >> 1;
            if (__ldg(ray_prefix + m) <= i) lo = m; else hi = m;
        }
        scene = lo;
        local = i - __ldg(ray_prefix + lo);
        lsc.s = lo;
    }
    CCS_DEV const DevRays &rays_of(uint32_t s) const { return entries[s].rays; }
    CCS_DEV const DevHits &hits_of(uint32_t s) const { return entries[s].hits; }
};

// Shared memory per thread, in floats: sibling intervals (2L float2), the sibling grid cache (K slots of
// 16 * NC floats), the K cache tags, padded to 16 bytes; then the float4s of the BVH prefetch slot.
__host__ __device__ constexpr int scratch_floats(int L, int K, int NC) { return cache_floats(K, NC) + 4 * L; }
__host__ __device__ constexpr int scratch_total_floats(int L, int K, int NC, int BW)
{
    return scratch_floats(L, K, NC) + 4 * (BW == 2 ? NC + 1 : 2 * NC + 1);   // node_f4<BW, NC>()
}

// NC = 3: one lane per ray, 32 rays per warp.  NC = 1: groups of three lanes per ray (lanes 3q .. 3q+2,
// component = lane - 3q), 10 rays per warp; lanes 30 and 31 take no ray.  Queue, refill and vote work on
// the group leaders (component 0); every lane of a group loads the ray and runs the same control.
template <bool STATS, int K, int MINB, class Src, int MODE, int NC, int BW>
__global__ void __launch_bounds__(128, MINB) k_intersect(Src src, int L, uint32_t refill, uint32_t chunk, int burst,
                                                         uint32_t iter_cap, uint32_t *queue, uint32_t *status,
                                                         unsigned long long *counters, ModeCtx mc,
                                                         const MlpWeights *__restrict__ mlp, float min_conf,
                                                         uint32_t vote)
{
    static_assert(NC == 3 || MODE == kModePlain, "groups of three lanes run the plain traversal only");
    extern __shared__ __align__(16) float smem[];
    const int stride = blockDim.x;
    const int sf = scratch_floats(L, K, NC);
    MlpWeights *mw = nullptr;
    MlpWarpTiles *mt = nullptr;
    if (MODE == kModeLearned) {   // network weights and per-warp tiles after the traversal scratch
        unsigned char *base = reinterpret_cast<unsigned char *>(smem + scratch_total_floats(L, K, NC, BW) * stride);
        mw = reinterpret_cast<MlpWeights *>(base);
        mt = reinterpret_cast<MlpWarpTiles *>(base + sizeof(MlpWeights)) + (threadIdx.x >> 5);
        load_weights(*mw, mlp);
        __syncthreads();
    }
    Scratch scr;
    scr.stride = stride;
    scr.cstride = cache_floats(K, NC);
    scr.cache = smem + threadIdx.x * scr.cstride;
    scr.tag = reinterpret_cast<int *>(scr.cache + 16 * NC * K);
    scr.sib = reinterpret_cast<float2 *>(smem + cache_floats(K, NC) * stride) + threadIdx.x;
    scr.node = reinterpret_cast<float4 *>(smem + sf * stride) + threadIdx.x;
    Counters cnt;
#pragma unroll
    for (int k = 0; k < kNumSumCounters; ++k) cnt.v[k] = 0;
    if (STATS && (threadIdx.x & 31) == 0) atomicMax(counters + 20, ~global_ns());   // first warp start
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    constexpr int kRaysPerWarp = NC == 3 ? 32 : 10;
    const int grp = NC == 3 ? lane : lane / 3;
    Grp G;
    G.c = NC == 3 ? 0 : lane - 3 * grp;
    G.mask = NC == 3 ? FULL : (7u << (3 * grp)) & FULL;
    G.l1 = 3 * grp + (G.c + 1) % 3;
    G.l2 = 3 * grp + (G.c + 2) % 3;
    G.l0 = 3 * grp;
    const bool valid = grp < kRaysPerWarp;
    const bool lead = valid && G.c == 0;
    const unsigned lead_mask = NC == 3 ? FULL : 0x09249249u;                 // lanes 0, 3, ..., 27
    const unsigned before_me = NC == 3 ? (1u << lane) - 1u : (1u << (3 * grp)) - 1u;   // leaders of earlier rays
    const float cellw = __int_as_float((127 - L) << 23);
    const uint32_t n = src.total();
    Lane<NC> s;
    BvhStack stk;
    float g[16 * NC];
    typename Src::LaneScene lsc;
    bool has = false, exhausted = false;
    uint32_t ray_scene = 0, ray_local = 0;
    uint32_t wnext = 0, wend = 0;   // warp-uniform range of rays taken from the queue, not yet handed out
    for (;;) {
        const unsigned idle = __ballot_sync(FULL, lead && !has);
        if (idle != 0u && ((uint32_t)__popc(idle) >= refill || idle == lead_mask)) {
            if (wnext == wend && !exhausted) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(queue, chunk);
                base = __shfl_sync(FULL, base, 0);
                if (base >= n) {
                    exhausted = true;
                    if (STATS && lane == 0) atomicMax(counters + 21, ~global_ns());   // queue found empty
                } else {
                    wnext = base;
                    wend = min(base + chunk, n);
                }
            }
            if (STATS && lane == 0 && wnext != wend) cnt.v[19] += 1;
            const uint32_t avail = wend - wnext;
            const uint32_t rank = (uint32_t)__popc(idle & before_me);
            if (valid && !has && rank < avail) {
                const uint32_t i = wnext + rank;
                has = true;
                src.locate(i, lsc, ray_scene, ray_local);
                const DevRays &rr = src.rays_of(ray_scene);
                const uint32_t j = ray_local;
                begin_ray<NC>(s, src.scene(lsc), __ldg(rr.ox + j), __ldg(rr.oy + j), __ldg(rr.oz + j),
                              __ldg(rr.dx + j), __ldg(rr.dy + j), __ldg(rr.dz + j), __ldg(rr.tmin + j),
                              __ldg(rr.tmax + j), iter_cap, G);
            }
            const uint32_t taken = avail < (uint32_t)__popc(idle) ? avail : (uint32_t)__popc(idle);
            wnext += taken;
        }
        const unsigned resident = __ballot_sync(FULL, lead && has);
        if (resident == 0u) {
            if (exhausted && wnext == wend) break;
            continue;
        }
        // phase vote: with vote > 0 the warp runs only subdivision steps while at least `vote` rays are in
        // a patch, else only BVH steps, so each iteration pays for one code path (while-while schedule)
        bool step_me = has;
        if (vote) {
            const unsigned in_patch = __ballot_sync(FULL, lead && has && s.in_pair);
            const unsigned in_bvh = __ballot_sync(FULL, lead && has && !s.in_pair);
            const bool patch_turn = (uint32_t)__popc(in_patch) >= vote || in_bvh == 0u;
            step_me = has && (s.in_pair == patch_turn);
        }
        int kind = kStepNone, bsteps = 0;
        if (step_me) {
            kind = lane_step<STATS, K, MODE, NC, BW>(s, g, stk, src.scene(lsc), L, scr, cnt, burst, mc, G, bsteps);
            const bool ok = kind != kStepCap;
            if (!ok || lane_done(s)) {
                if (!ok) {
                    if (lead) atomicOr(status, 1u);
                    s.best.pid = kMissId;
                }
                if (MODE == kModeAnyHit && lead) {
                    mc.occluded[ray_local] = s.best.pid != kMissId ? 1 : 0;
                } else if (lead) {
                    const DevHits &hh = src.hits_of(ray_scene);
                    const uint32_t i = ray_local;
                    if (s.best.pid != kMissId) {
                        const uint32_t cu = s.best.cell & ((1u << L) - 1u), cv = s.best.cell >> L;
                        hh.t[i] = s.best.t;
                        if (MODE == kModeScreen) {   // centre of the leaf node's domain (exact powers of two)
                            const int su = (s.best.lvl + 1) >> 1, sv = s.best.lvl >> 1;
                            hh.u[i] = (float)cu * cellw + __int_as_float((126 - su) << 23);
                            hh.v[i] = (float)cv * cellw + __int_as_float((126 - sv) << 23);
                        } else {
                            hh.u[i] = ((float)cu + 0.5f) * cellw;
                            hh.v[i] = ((float)cv + 0.5f) * cellw;
                        }
                        hh.pid[i] = s.best.pid;
                    } else {
                        hh.t[i] = __int_as_float(0x7f800000);
                        hh.u[i] = 0.0f;
                        hh.v[i] = 0.0f;
                        hh.pid[i] = kMissId;
                    }
                }
                has = false;
            }
        }
        if constexpr (STATS) {   // schedule of this warp iteration, counted in rays (group leaders)
            const unsigned ks = __ballot_sync(FULL, lead && kind == kStepSplit);
            const unsigned kg = __ballot_sync(FULL, lead && kind == kStepGregory);
            const unsigned kl = __ballot_sync(FULL, lead && kind == kStepLeaf);
            const unsigned kb = __ballot_sync(FULL, lead && kind == kStepBvh);
            const int longest = __reduce_max_sync(FULL, bsteps);
            if (lane == 0) {
                cnt.v[8] += 1;
                cnt.v[9] += __popc(resident);
                cnt.v[10] += __popc(ks);
                cnt.v[11] += ks != 0u;
                cnt.v[12] += __popc(kg);
                cnt.v[13] += kg != 0u;
                cnt.v[14] += __popc(kl);
                cnt.v[15] += kl != 0u;
                cnt.v[16] += __popc(kb);
                cnt.v[17] += kb != 0u;
                cnt.v[18] += (unsigned)longest;
            }
        }
        if constexpr (MODE == kModeLearned) {   // network round for every lane that has just started a pair
            const bool mine = has && s.in_pair && s.phase == kPhasePropose;
            const unsigned need = __ballot_sync(FULL, mine);
            // rounds are batched: run once a quarter of the warp waits, or when every active lane does
            const unsigned active = __ballot_sync(FULL, has);
            if (need && (__popc(need) >= 8 || need == active)) {
                if (mine) {
                    float f[kFeat];
                    pair_features(rec_of(src.scene(lsc), s.pid), s.pr.org[0], s.pr.org[1], s.pr.org[2], s.pr.inv[0],
                                  s.pr.inv[1], s.pr.inv[2], s.rc0, s.rc1, f);
#pragma unroll
                    for (int k = 0; k < 32; k += 2)
                        st_bf16x2(mt->x + lane * kXStride + k, k < kFeat ? f[k] : 0.0f,
                                  k + 1 < kFeat ? f[k + 1] : 0.0f);
                }
                __syncwarp();
                if (need & 0x0000ffffu) mlp_round(*mw, *mt, 0, lane, nullptr, 0u);
                if (need & 0xffff0000u) mlp_round(*mw, *mt, 1, lane, nullptr, 0u);
                if (mine) {
                    if (mt->pmax[lane] >= min_conf) {
                        s.phase = kPhaseDirected;
                        s.prop = cell3_path(mt->cell[lane]);
                    } else {
                        s.phase = kPhaseNormal;
                    }
                }
                __syncwarp();
            }
        }
    }
    cp_async_wait_all();
    if (STATS) {   // every lane of a group holds the same counts: the leader reports them
#pragma unroll
        for (int k = 0; k < kNumSumCounters; ++k) {
            unsigned long long v = lead ? cnt.v[k] : 0ull;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            if (lane == 0 && v) atomicAdd(counters + k, v);
        }
        if (lane == 0) atomicMax(counters + 22, global_ns());   // last warp exit
    }
}

template <int BW>
static size_t smem_bytes(uint32_t threads, uint32_t L, uint32_t K, uint32_t NC)
{
    return (size_t)threads * (NC == 3 ? scratch_total_floats((int)L, (int)K, 3, BW)
                                      : scratch_total_floats((int)L, (int)K, 1, BW)) * sizeof(float);
}

template <bool STATS, int K, int MINB, class Src, int MODE, int NC, int BW>
static cudaError_t launch_one(const Src &src, const LaunchCfg &cfg, uint32_t *queue, uint32_t *status, int num_sms,
                              cudaStream_t s)
{
    auto kern = k_intersect<STATS, K, MINB, Src, MODE, NC, BW>;
    const uint32_t threads = cfg.block_threads;
    size_t smem = smem_bytes<BW>(threads, cfg.leaf_depth, K, NC);
    if (MODE == kModeLearned) smem += sizeof(MlpWeights) + (threads / 32) * sizeof(MlpWarpTiles);
    static size_t configured = 0;   // largest dynamic shared memory size set on this instantiation
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    // resident blocks per SM for this instantiation, block size and shared memory (queried once per shape)
    static uint32_t occ_threads = 0;
    static size_t occ_smem = 0;
    static int occ_active = 0;
    if (occ_threads != threads || occ_smem != smem) {
        int max_active = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_active, kern, (int)threads, smem);
        if (e != cudaSuccess) return e;
        occ_threads = threads;
        occ_smem = smem;
        occ_active = max_active;
    }
    const int max_active = occ_active;
    if (max_active < 1) return cudaErrorInvalidConfiguration;
    uint32_t per_sm = cfg.blocks_per_sm < (uint32_t)max_active ? cfg.blocks_per_sm : (uint32_t)max_active;
    uint32_t blocks = (uint32_t)num_sms * per_sm;
    const uint32_t n = src.n;
    const uint32_t rays_per_block = NC == 3 ? threads : threads / 32 * 10;
    const uint32_t needed = (n + rays_per_block - 1) / rays_per_block;
    if (blocks > needed) blocks = needed;
    if (blocks == 0) blocks = 1;
    kern<<<blocks, threads, smem, s>>>(src, (int)cfg.leaf_depth, cfg.refill, cfg.chunk, (int)cfg.bvh_burst,
                                       cfg.iter_cap, queue, status, cfg.counters, cfg.mc, cfg.mlp, cfg.min_conf,
                                       cfg.vote);
    return cudaGetLastError();
}

constexpr int kMinbG3 = 6;   // blocks of 128 threads per SM the grouped kernel is compiled for

template <int BW, class Src>
static cudaError_t dispatch(const Src &src, const LaunchCfg &cfg, uint32_t *queue, uint32_t *status, int num_sms,
                            cudaStream_t s)
{
    if (src.n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const bool stats = (cfg.flags & CCS_TRACE_COUNT) != 0;
    if constexpr (std::is_same<Src, SingleSource>::value) {
        if (cfg.mode == kModeExport)
            return cfg.cache_slots == 0 ? launch_one<false, 0, 3, Src, kModeExport, 3, BW>(src, cfg, queue, status, num_sms, s)
                                        : launch_one<false, 2, 3, Src, kModeExport, 3, BW>(src, cfg, queue, status, num_sms, s);
        if (cfg.mode == kModeScreen) {
            if (stats)
                return cfg.cache_slots == 0 ? launch_one<true, 0, 3, Src, kModeScreen, 3, BW>(src, cfg, queue, status, num_sms, s)
                                            : launch_one<true, 2, 3, Src, kModeScreen, 3, BW>(src, cfg, queue, status, num_sms, s);
            return cfg.cache_slots == 0 ? launch_one<false, 0, 3, Src, kModeScreen, 3, BW>(src, cfg, queue, status, num_sms, s)
                                        : launch_one<false, 2, 3, Src, kModeScreen, 3, BW>(src, cfg, queue, status, num_sms, s);
        }
        if (cfg.mode == kModeAnyHit) {
            if (stats)
                return cfg.cache_slots == 0 ? launch_one<true, 0, 3, Src, kModeAnyHit, 3, BW>(src, cfg, queue, status, num_sms, s)
                                            : launch_one<true, 2, 3, Src, kModeAnyHit, 3, BW>(src, cfg, queue, status, num_sms, s);
            return cfg.cache_slots == 0 ? launch_one<false, 0, 3, Src, kModeAnyHit, 3, BW>(src, cfg, queue, status, num_sms, s)
                                        : launch_one<false, 2, 3, Src, kModeAnyHit, 3, BW>(src, cfg, queue, status, num_sms, s);
        }
        if (cfg.mode == kModeLearned)   // the network's shared memory leaves no room for the sibling cache
            return stats ? launch_one<true, 0, 3, Src, kModeLearned, 3, BW>(src, cfg, queue, status, num_sms, s)
                         : launch_one<false, 0, 3, Src, kModeLearned, 3, BW>(src, cfg, queue, status, num_sms, s);
    }
    if (cfg.lanes_per_ray == 3) {   // groups of three lanes per ray (plain traversal)
        if (stats)
            return cfg.cache_slots == 0 ? launch_one<true, 0, kMinbG3, Src, kModePlain, 1, BW>(src, cfg, queue, status, num_sms, s)
                                        : launch_one<true, 2, kMinbG3, Src, kModePlain, 1, BW>(src, cfg, queue, status, num_sms, s);
        return cfg.cache_slots == 0 ? launch_one<false, 0, kMinbG3, Src, kModePlain, 1, BW>(src, cfg, queue, status, num_sms, s)
                                    : launch_one<false, 2, kMinbG3, Src, kModePlain, 1, BW>(src, cfg, queue, status, num_sms, s);
    }
    if (stats)   // counting runs are not timed: one register budget is enough
        return cfg.cache_slots == 0 ? launch_one<true, 0, 3, Src, kModePlain, 3, BW>(src, cfg, queue, status, num_sms, s)
                                    : launch_one<true, 2, 3, Src, kModePlain, 3, BW>(src, cfg, queue, status, num_sms, s);
    if (cfg.min_blocks >= 4)
        return cfg.cache_slots == 0 ? launch_one<false, 0, 4, Src, kModePlain, 3, BW>(src, cfg, queue, status, num_sms, s)
                                    : launch_one<false, 2, 4, Src, kModePlain, 3, BW>(src, cfg, queue, status, num_sms, s);
    return cfg.cache_slots == 0 ? launch_one<false, 0, 3, Src, kModePlain, 3, BW>(src, cfg, queue, status, num_sms, s)
                                : launch_one<false, 2, 3, Src, kModePlain, 3, BW>(src, cfg, queue, status, num_sms, s);
}

template <int BW>
cudaError_t launch_single_w(const DevScene &sc, const DevRays &r, const DevHits &h, uint32_t n, const LaunchCfg &cfg,
                            uint32_t *queue, uint32_t *status, int num_sms, cudaStream_t s, const uint32_t *perm)
{
    SingleSource src{sc, r, h, n, perm};
    return dispatch<BW>(src, cfg, queue, status, num_sms, s);
}

template <int BW>
cudaError_t launch_batch_w(const BatchEntry *entries, const uint32_t *ray_prefix, uint32_t n_scenes, uint32_t n_total,
                           const LaunchCfg &cfg, uint32_t *queue, uint32_t *status, int num_sms, cudaStream_t s)
{
    BatchSource src{entries, ray_prefix, n_scenes, n_total};
    LaunchCfg c = cfg;
    c.mode = kModePlain;
    return dispatch<BW>(src, c, queue, status, num_sms, s);
}

}  // namespace ccs
