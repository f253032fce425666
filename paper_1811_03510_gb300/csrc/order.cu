// Work order of a closest-hit launch (CCS_TRACE_ORDER).  A persistent launch ends when its slowest
// ray ends, so rays that need many subdivision steps should start first.  A cheap estimate ranks tiles
// of rays: the most candidate patches (leaf boxes of the BVH entered by the ray within [tmin, tmax])
// over a sample of each tile's rays.  Tiles are then ordered by that estimate, costliest first and
// stable within a class, and the permutation of ray indices in that order is what the work queue
// hands out.  Only the order in which rays are processed changes, never a ray's answer.
//
// Tiles: TW x TH rays of an image of width w (ray index y * w + x; a ragged last row is allowed), or,
// for batches that are not an image, runs of 32 consecutive rays (w = n, one row).  Every 4th ray in x
// and y is sampled (4 of an 8 x 8 tile, 8 of a run).
#include <cuda_runtime.h>

#include "ccs_internal.h"
#include "order_plan.h"

namespace ccs {

constexpr int kOrderStack = 64;

// Candidate patches of one ray: the BVH leaves it enters within [t0, t1] (every one, with no pruning by
// a closest hit; counting whole subtrees instead of their leaves ranks the tiles clearly worse).  Binary
// or 4-wide nodes (the stack bound of either tree holds: 62 levels, or three siblings on each of at
// most 21 levels).
__device__ uint32_t count_candidates(const float4 *__restrict__ nodes, uint32_t n_nodes, uint32_t width, float ox,
                                     float oy, float oz, float dx, float dy, float dz, float t0, float t1)
{
    if (n_nodes == 0 || !(t0 <= t1)) return 0;
    const float ix = 1.0f / dx, iy = 1.0f / dy, iz = 1.0f / dz;
    int stack[kOrderStack];
    int sp = 0, node = 0;
    uint32_t cnt = 0;
    // fminf/fmaxf drop the NaN of 0 * inf, as in the traversal's slab test
    auto enters = [&](float lx, float hx, float ly, float hy, float lz, float hz) {
        const float ax = (lx - ox) * ix, bx = (hx - ox) * ix;
        const float ay = (ly - oy) * iy, by = (hy - oy) * iy;
        const float az = (lz - oz) * iz, bz = (hz - oz) * iz;
        const float tn = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), t0));
        const float tf = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), t1));
        return tn <= tf;
    };
    for (;;) {
        int next = -1;
        auto take = [&](bool hit, int child) {
            if (!hit || child == kEmptyChild) return;
            if (child < 0) {
                ++cnt;
            } else if (next < 0) {
                next = child;
            } else if (sp < kOrderStack) {
                stack[sp++] = child;
            }
        };
        if (width == 4) {
            const float4 *nd = nodes + (size_t)node * kNode4F4;
            const float4 lx = __ldg(nd), hx = __ldg(nd + 1), ly = __ldg(nd + 2), hy = __ldg(nd + 3);
            const float4 lz = __ldg(nd + 4), hz = __ldg(nd + 5);
            const int4 ch = __ldg(reinterpret_cast<const int4 *>(nd + 6));
            take(enters(lx.x, hx.x, ly.x, hy.x, lz.x, hz.x), ch.x);
            take(enters(lx.y, hx.y, ly.y, hy.y, lz.y, hz.y), ch.y);
            take(enters(lx.z, hx.z, ly.z, hy.z, lz.z, hz.z), ch.z);
            take(enters(lx.w, hx.w, ly.w, hy.w, lz.w, hz.w), ch.w);
        } else {
            const float4 *nd = nodes + (size_t)node * kNodeF4;
            const float4 qx = __ldg(nd), qy = __ldg(nd + 1), qz = __ldg(nd + 2);
            const int4 ch = __ldg(reinterpret_cast<const int4 *>(nd + 3));
            take(enters(qx.x, qx.y, qy.x, qy.y, qz.x, qz.y), ch.x);
            take(enters(qx.z, qx.w, qy.z, qy.w, qz.z, qz.w), ch.y);
        }
        if (next >= 0) {
            node = next;
        } else if (sp > 0) {
            node = stack[--sp];
        } else {
            break;
        }
    }
    return cnt;
}

// One thread per sampled ray, the samples of a tile in consecutive lanes: the tile's key is the largest
// candidate count of its samples, and each block of S::TPB tiles adds up how many rays it has of each
// key in hist[key * n_blocks + block] (zeroed before the launch).
template <class S>
__global__ void __launch_bounds__(kOrderThreads) k_order_estimate(OrderGeom g, const float4 *__restrict__ nodes,
                                                                    uint32_t n_nodes, uint32_t width, DevRays r,
                                                                    uint32_t *__restrict__ tile_key,
                                                                    uint32_t *__restrict__ hist)
{
    const uint32_t tile = blockIdx.x * S::TPB + threadIdx.x / S::SPT, smp = threadIdx.x % S::SPT;
    const uint32_t tx = tile % g.tiles_x, ty = tile / g.tiles_x;
    uint32_t c = 0, j;
    if (tile < g.n_tiles) {
        if (tile_sample<S>(g, tile, smp, &j)) {
            c = count_candidates(nodes, n_nodes, width, __ldg(r.ox + j), __ldg(r.oy + j), __ldg(r.oz + j),
                                 __ldg(r.dx + j), __ldg(r.dy + j), __ldg(r.dz + j), __ldg(r.tmin + j),
                                 __ldg(r.tmax + j));
        }
    }
#pragma unroll
    for (uint32_t o = S::SPT >> 1; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
    if (smp == 0 && tile < g.n_tiles) {
        const uint32_t key = c < kOrderKeys - 1 ? c : kOrderKeys - 1;
        tile_key[tile] = key;
        atomicAdd(hist + key * gridDim.x + blockIdx.x, tile_size<S>(g, tx * S::TW, ty * S::TH));
    }
}

// One block of kOrderScan threads, thread b of a round for estimate block b: base[k * n_blocks + b] = the
// rays of class k in blocks before b (a scan over blocks for every class at once), and after the last
// round base[kOrderKeys * n_blocks + k] = the rays of the costlier classes, so that block b's tiles of
// class k start at the sum of the two.
constexpr int kOrderScan = 512;
__global__ void __launch_bounds__(kOrderScan) k_order_scan(const uint32_t *__restrict__ hist, uint32_t n_blocks,
                                                            uint32_t *__restrict__ base)
{
    __shared__ uint32_t wtot[kOrderScan / 32][kOrderKeys];
    __shared__ uint32_t carry[kOrderKeys];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < kOrderKeys) carry[t] = 0;
    for (uint32_t r0 = 0; r0 < n_blocks; r0 += kOrderScan) {
        const uint32_t b = r0 + t;
        uint32_t v[kOrderKeys], incl[kOrderKeys];
#pragma unroll
        for (int k = 0; k < kOrderKeys; ++k) v[k] = b < n_blocks ? __ldg(hist + (size_t)k * n_blocks + b) : 0u;
#pragma unroll
        for (int k = 0; k < kOrderKeys; ++k) {
            incl[k] = v[k];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl[k], o);
                if ((int)lane >= o) incl[k] += u;
            }
            if (lane == 31) wtot[warp][k] = incl[k];
        }
        __syncthreads();
        if (t < kOrderKeys) {   // exclusive prefix over the warps of the round, after the carry
            uint32_t run = carry[t];
            for (uint32_t w = 0; w < kOrderScan / 32; ++w) {
                const uint32_t u = wtot[w][t];
                wtot[w][t] = run;
                run += u;
            }
            carry[t] = run;
        }
        __syncthreads();
        if (b < n_blocks) {
#pragma unroll
            for (int k = 0; k < kOrderKeys; ++k) base[(size_t)k * n_blocks + b] = wtot[warp][k] + incl[k] - v[k];
        }
        __syncthreads();
    }
    if (t < kOrderKeys) {
        uint32_t above = 0;
        for (int k = t + 1; k < kOrderKeys; ++k) above += carry[k];
        base[(size_t)kOrderKeys * n_blocks + t] = above;
    }
}

// Block b places the tiles of estimate block b: each tile's first queue position (its class's base for
// the block, then the block's tiles in index order), then the indices of the tiles' rays at those
// positions, row-major within a tile.  Only the image's last row can be partial and it is the last row
// of its tiles, so every earlier row of a tile holds min(TW, w - x0) rays.
template <class S>
__global__ void __launch_bounds__(kOrderThreads) k_order_place(OrderGeom g, const uint32_t *__restrict__ tile_key,
                                                                 const uint32_t *__restrict__ base,
                                                                 uint32_t *__restrict__ perm)
{
    constexpr uint32_t kWarps = (S::TPB + 31) / 32;
    __shared__ uint32_t wsum[kWarps][kOrderKeys];
    __shared__ uint32_t tpos[S::TPB], tx0[S::TPB], ty0[S::TPB];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t tile = blockIdx.x * S::TPB + t;
    const bool valid = t < S::TPB && tile < g.n_tiles;
    const uint32_t key = valid ? tile_key[tile] : (uint32_t)kOrderKeys;
    if (warp < kWarps) {   // whole warps: the class-wise prefix of tile sizes within each warp
        const uint32_t x0 = (tile % g.tiles_x) * S::TW, y0 = (tile / g.tiles_x) * S::TH;
        const uint32_t size = valid ? tile_size<S>(g, x0, y0) : 0u;
        uint32_t pre = 0;   // rays of earlier tiles of this warp in the same class
#pragma unroll 1
        for (uint32_t k = 0; k < (uint32_t)kOrderKeys; ++k) {
            const uint32_t v = key == k ? size : 0u;
            uint32_t incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += u;
            }
            if (key == k) pre = incl - v;
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            if (lane == 0) wsum[warp][k] = tot;
        }
        if (t < S::TPB) {
            tx0[t] = x0;
            ty0[t] = y0;
            tpos[t] = pre;
        }
    }
    __syncthreads();
    if (valid) {
        uint32_t w_before = 0;
        for (uint32_t w = 0; w < warp; ++w) w_before += wsum[w][key];
        tpos[t] += base[(size_t)key * gridDim.x + blockIdx.x] + base[(size_t)kOrderKeys * gridDim.x + key] + w_before;
    }
    __syncthreads();
    constexpr uint32_t kPerTile = S::TW * S::TH;
    const uint32_t first = blockIdx.x * S::TPB;
    const uint32_t tiles = g.n_tiles - first < S::TPB ? g.n_tiles - first : S::TPB;
    for (uint32_t e = t; e < tiles * kPerTile; e += kOrderThreads) {
        const uint32_t lt = e / kPerTile;
        uint32_t j, off;
        if (tile_entry<S>(g, tx0[lt], ty0[lt], e % kPerTile, &j, &off)) perm[tpos[lt] + off] = j;
    }
}

size_t order_scratch_words(uint32_t n, uint32_t image_width)
{
    if (n == 0) return 0;
    const bool img = image_width > 0;
    const OrderGeom g = img ? order_geom<ImageShape>(n, image_width) : order_geom<RunShape>(n, n);
    const uint32_t nb = img ? order_blocks<ImageShape>(g) : order_blocks<RunShape>(g);
    return (size_t)n + g.n_tiles + 2 * (size_t)nb * kOrderKeys + kOrderKeys;
}

template <class S>
static cudaError_t order_with(const DevScene &sc, const DevRays &r, uint32_t n, uint32_t w, uint32_t *scratch,
                              cudaStream_t s)
{
    const OrderGeom g = order_geom<S>(n, w);
    const uint32_t nb = order_blocks<S>(g);
    uint32_t *perm = scratch, *key = scratch + n, *hist = key + g.n_tiles, *base = hist + (size_t)nb * kOrderKeys;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nb * kOrderKeys * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_order_estimate<S><<<nb, kOrderThreads, 0, s>>>(g, sc.nodes, sc.n_nodes, sc.width, r, key, hist);
    k_order_scan<<<1, kOrderScan, 0, s>>>(hist, nb, base);
    k_order_place<S><<<nb, kOrderThreads, 0, s>>>(g, key, base, perm);
    return cudaGetLastError();
}

cudaError_t launch_order(const DevScene &sc, const DevRays &r, uint32_t n, uint32_t image_width, uint32_t *scratch,
                         cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    return image_width > 0 ? order_with<ImageShape>(sc, r, n, image_width, scratch, s)
                           : order_with<RunShape>(sc, r, n, n, scratch, s);
}

}  // namespace ccs
