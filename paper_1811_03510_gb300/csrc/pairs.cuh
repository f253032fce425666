// Closest hit in passes that each keep a warp on one kind of work (the pair engine, CCS_TRACE_PAIRS).
//
//  1. k_cand: one thread per ray walks the BVH (Sec. 4) and keeps the ray's kPairCands nearest candidate
//     patches, ordered by (entry distance of the patch box, patch id).  Before the list is full nothing
//     is pruned but [tmin, tmax]; once it is full, subtrees that enter beyond its last entry are skipped
//     and the smallest entry distance dropped that way is kept (t_evict).  With local frames a Bezier patch
//     whose root box in its own frame the ray does not come near is no candidate (root_box_near: its pair
//     would end at the first split).  A ray with candidates becomes a task with a cost class (the highest when a candidate is a Gregory patch, else its number of
//     candidates); rays with no candidate are written as misses here.
//  2. Each task's index goes to the list of its cost class (the candidate pass counts the classes' places),
//     and the subdivision pass's queue takes the classes costliest first, so that the long rays start
//     early and the launch does not end on a few of them.
//  3. k_pairs: persistent warps take tasks in that order.  A lane runs Algorithm 3 on one (ray, patch) pair
//     at a time, taking the ray's candidates in entry order and stopping at the first one that enters
//     beyond the ray's best hit.  Every warp iteration is one or two subdivision steps (Algorithm 3's loop
//     body) of up to 32 pairs: the BVH walk, whose step count differs from ray to ray, is not in the loop.
//  4. A ray whose dropped candidates could still hold the answer (best hit not before t_evict) has its lane
//     collect the next ones, those after the last listed, by a BVH walk of its own (collect_more), and goes
//     on with them.
//
// The answer is the smallest leaf key over all nested intervals (readings A14/A15), which does not depend
// on the order in which pairs are searched, so every pass reuses the arithmetic of traverse.cuh and the
// hits are bit-identical to k_intersect's.
#pragma once

#include "intersect_impl.cuh"

namespace ccs {

constexpr int kPairCands = 8;            // candidates kept per ray (nearest entries)
constexpr int kCandBlock = 128;          // threads of a candidate-pass block (its warps work independently)
constexpr int kStepsPerIter = 2;         // subdivision steps per warp iteration of the subdivision pass
constexpr int kCostClasses = 16;
// counter words of a launch: the queue head, the tasks of each cost class
constexpr int kCtrQueue = 3, kCtrHist = 16, kPairCtrWords = 64;
// Ray i's task and candidates have fixed places (task i, candidates from i kPairCands), so the candidate
// pass needs no atomic counter for them.  A task is 4 uint4 (64 bytes), everything a lane needs to start
// the ray:
//   (ray, first candidate, z, t_evict bits), (first candidate's patch id, its entry distance, tmin, tmax),
//   (ox, oy, oz, dx), (dy, dz, 0, 0) as float bits;
// z = candidates (bits 0..7) | cost class (bits 8..11) | candidates were dropped (bit 30).
constexpr uint32_t kTaskEvicted = 0x40000000u;

struct PairBufs {
    uint32_t *ctr;            // kPairCtrWords words, zeroed before the candidate pass
    uint4 *task;              // task of ray i at 4 i (rays with candidates only)
    uint32_t *cls;            // per cost class c, from c * n: the rays of its tasks
    uint2 *cand;              // (patch id, entry distance bits), ray i's from i kPairCands
    uint32_t n;               // rays of the launch (the stride of cls)
};

// Bytes of the pair engine's scratch for n rays, and its layout (every part 256-byte aligned).
__host__ __device__ inline size_t pair_align(size_t b) { return (b + 255) & ~(size_t)255; }
inline size_t pair_scratch_bytes(uint32_t n)
{
    return pair_align(kPairCtrWords * 4) + pair_align((size_t)n * 64) + pair_align((size_t)n * 4 * kCostClasses) +
           pair_align((size_t)n * kPairCands * 8);
}
inline PairBufs pair_bufs_at(void *base, uint32_t n)
{
    char *p = static_cast<char *>(base);
    PairBufs b;
    b.ctr = reinterpret_cast<uint32_t *>(p);
    p += pair_align(kPairCtrWords * 4);
    b.task = reinterpret_cast<uint4 *>(p);
    p += pair_align((size_t)n * 64);
    b.cls = reinterpret_cast<uint32_t *>(p);
    p += pair_align((size_t)n * 4 * kCostClasses);
    b.cand = reinterpret_cast<uint2 *>(p);
    b.n = n;
    return b;
}

// Shared memory of a k_pairs thread after its traversal scratch: the world ray of its task (origin,
// 1 / direction, tmin, tmax), t_evict and the direction, read when a pair starts and when the ray ends, and
// the first and end places of the task's candidates (kept here, not in registers, so that the 1-slot sibling
// cache variant does not spill); then the thread's mailbox for the subtrees it handed to other lanes (the smallest (t, cell) key they found,
// 64 bits), the number of them still running, and a flag for one that reached the iteration cap.
constexpr int kRaySlotFloats = 14, kHelpFloats = 4;
// the per-thread helper area must hold the mailbox and the two counters k_pairs places there
static_assert(kHelpFloats * sizeof(float) >= sizeof(unsigned long long) + 2 * sizeof(int),
              "the helper area of a k_pairs thread is smaller than its mailbox and counters");
// A subtree is handed to an idle lane when it has at least this many levels below its root.
constexpr int kMinDonateLevels = 4;

// Order-preserving map of a float's bits to an unsigned integer, and back (the mailbox key).
CCS_DEV uint32_t ord_bits(float t)
{
    const uint32_t u = __float_as_uint(t);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
CCS_DEV float unord_bits(uint32_t k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k); }

// The scene of a lane's pair, handed from lane `from` to the lanes that take one of its subtrees (a batch
// lane carries its scene's index; one scene is the launch's).
template <class Src>
CCS_DEV void share_scene(typename Src::LaneScene &l, int from)
{
    if constexpr (std::is_same<Src, BatchSource>::value) l.s = __shfl_sync(0xffffffffu, l.s, from);
}

CCS_DEV bool cand_less(float ta, uint32_t pa, float tb, uint32_t pb) { return ta < tb || (ta == tb && pa < pb); }

// The ray as k_intersect's begin_ray reads it (false: a ray that is a miss by definition).
CCS_DEV bool load_world_ray(const DevRays &rr, uint32_t j, float (&o)[3], float (&d)[3], float (&inv)[3], float &tmin,
                            float &tmax)
{
    o[0] = __ldg(rr.ox + j);
    o[1] = __ldg(rr.oy + j);
    o[2] = __ldg(rr.oz + j);
    d[0] = __ldg(rr.dx + j);
    d[1] = __ldg(rr.dy + j);
    d[2] = __ldg(rr.dz + j);
    tmin = __ldg(rr.tmin + j);
    tmax = __ldg(rr.tmax + j);
#pragma unroll
    for (int k = 0; k < 3; ++k) inv[k] = safe_inv(d[k]);
    return !(!(tmin <= tmax) || isnan(o[0]) || isnan(o[1]) || isnan(o[2]) || isnan(d[0]) || isnan(d[1]) ||
             isnan(d[2]));
}

template <int MODE, class Src>
CCS_DEV void write_miss(const Src &src, uint32_t scene, uint32_t j, uint8_t *occluded)
{
    if (MODE == kModeAnyHit) {
        occluded[j] = 0;
    } else {
        const DevHits &hh = src.hits_of(scene);
        hh.t[j] = __int_as_float(0x7f800000);
        hh.u[j] = 0.0f;
        hh.v[j] = 0.0f;
        hh.pid[j] = kMissId;
    }
}

// Cull test of a candidate with local frames (Sec. 3.4): does the ray pass near the patch's root box in
// the patch frame?  Every box of a Bezier pair's subdivision lies in that box (de Casteljau midpoints stay
// between their operands), widened by the box extension by at most tau / 2; a pair's FP32 slab tests
// report a hit only within about 1e-6 (|o - anchor| + box diagonal) of a box.  The test pads the box by
// 2^-16 (1 + |o - anchor|_1 + |hi - lo|_1), far more than both and far less than a patch, so a culled
// pair holds no leaf that its subdivision would record.  Gregory patches are kept (their boxes come from
// the bounds of Algorithm 2, not from the control points).
CCS_DEV bool root_box_near(const float4 *__restrict__ rec, const float (&o)[3], const float (&d)[3], float tmin,
                           const Grp &G)
{
    const float4 an = __ldg(rec + 15);
    if (an.w != 0.0f) return true;
    const float4 R[3] = {__ldg(rec + 16), __ldg(rec + 17), __ldg(rec + 18)};
    const float4 hb = __ldg(rec + 19);
    const float o3[3] = {__fsub_rn(o[0], an.x), __fsub_rn(o[1], an.y), __fsub_rn(o[2], an.z)};
    const float pad = __fmul_rn(__int_as_float((127 - 16) << 23),
                                __fadd_rn(hb.w, __fadd_rn(__fadd_rn(fabsf(o3[0]), fabsf(o3[1])), fabsf(o3[2]))));
    RayG<3> r;
    float lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.org[k] = fmaf(R[k].x, o3[0], fmaf(R[k].y, o3[1], R[k].z * o3[2]));
        r.inv[k] = safe_inv(fmaf(R[k].x, d[0], fmaf(R[k].y, d[1], R[k].z * d[2])));
        lo[k] = __fsub_rn(R[k].w, pad);
        hi[k] = __fadd_rn(pick(k, hb.x, hb.y, hb.z), pad);
    }
    float t0, t1;
    slab<3>(r, lo, hi, tmin, __int_as_float(0x7f800000), G, t0, t1);
    return t0 <= t1;
}

// ------------------------------------------------------------------------------------------------
// Pass 1: BVH walk with the sorted candidate list.
// ------------------------------------------------------------------------------------------------
// The BVH walk of the candidate pass (Sec. 4): the C candidates of the ray with the smallest keys (entry
// distance of the patch box, patch id), sorted in kt / kp, counting only keys above (lb_t, lb_p) when has_lb
// (the candidates an earlier walk did not list: all its dropped keys are above its last listed one).  Before
// the list is full nothing is pruned but [tmin, tmax]; once it is full, subtrees entered beyond its last
// entry are skipped and the smallest entry distance dropped that way is kept (t_evict).  With local frames,
// Bezier patches whose root box the ray does not come near are no candidates (root_box_near).  Returns false
// when the iteration budget it ran out.
template <bool STATS, int BW>
CCS_DEV bool walk_candidates(const DevScene &sc, const RayG<3> &r, const float (&ro)[3], const float (&rd)[3],
                             float tmin, float tmax, bool has_lb, float lb_t, uint32_t lb_p, uint32_t &it,
                             float (&kt)[kPairCands], uint32_t (&kp)[kPairCands], int &cnt, float &t_evict,
                             bool &evicted, unsigned long long &nodes, unsigned long long &culled, const Grp &G)
{
    constexpr int C = kPairCands;
    const float kInf = __int_as_float(0x7f800000);
    int2 stk[kBvhStack];
    int sp = 0, node = 0;
    float n0 = tmin;
    for (;;) {
        if (node == kDone) break;
        if (it == 0) return false;
        --it;
        if (node < 0) {   // a patch: into the list (the leaf's box is the patch box)
            const uint32_t p = (uint32_t)(~node);
            bool ins = true;
            if (has_lb && !cand_less(lb_t, lb_p, n0, p)) {
                ins = false;   // listed by an earlier walk
            } else if (sc.local && !root_box_near(rec_of(sc, p), ro, rd, tmin, G)) {
                ins = false;
                if (STATS) ++culled;
            } else if (cnt == C) {
                evicted = true;
                if (!cand_less(n0, p, kt[C - 1], kp[C - 1])) {
                    t_evict = fminf(t_evict, n0);
                    ins = false;
                } else {
                    t_evict = fminf(t_evict, kt[C - 1]);
                }
            } else {
                ++cnt;
            }
            if (ins) {
                int m = 0;
#pragma unroll
                for (int j = 0; j < C; ++j) m += cand_less(kt[j], kp[j], n0, p) ? 1 : 0;
#pragma unroll
                for (int j = C - 1; j >= 1; --j) {
                    kt[j] = j > m ? kt[j - 1] : (j == m ? n0 : kt[j]);
                    kp[j] = j > m ? kp[j - 1] : (j == m ? p : kp[j]);
                }
                kt[0] = m == 0 ? n0 : kt[0];
                kp[0] = m == 0 ? p : kp[0];
            }
        } else {
            ++nodes;
            // once the list is full, a subtree entered beyond its last entry only holds dropped patches
            const float bound = cnt == C ? kt[C - 1] : tmax;
            if constexpr (BW == 4) {
                const float4 *nd = sc.nodes + (size_t)node * kNode4F4;
                float4 lo4[3], hi4[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    lo4[k] = __ldg(nd + 2 * k);
                    hi4[k] = __ldg(nd + 2 * k + 1);
                }
                const int4 ch = __ldg(reinterpret_cast<const int4 *>(nd + 6));
                int c[4] = {ch.x, ch.y, ch.z, ch.w};
                float key[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float lo[3], hi[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        lo[k] = j == 0 ? lo4[k].x : j == 1 ? lo4[k].y : j == 2 ? lo4[k].z : lo4[k].w;
                        hi[k] = j == 0 ? hi4[k].x : j == 1 ? hi4[k].y : j == 2 ? hi4[k].z : hi4[k].w;
                    }
                    float t0, t1;
                    slab<3>(r, lo, hi, tmin, tmax, G, t0, t1);
                    bool h = t0 <= t1 && c[j] != kEmptyChild;
                    if (h && t0 > bound) {
                        h = false;
                        evicted = true;
                        t_evict = fminf(t_evict, t0);
                    }
                    key[j] = h ? t0 : kInf;
                }
                cx4(key, c, 0, 1);
                cx4(key, c, 2, 3);
                cx4(key, c, 0, 2);
                cx4(key, c, 1, 3);
                cx4(key, c, 1, 2);
                if (key[0] < kInf) {
#pragma unroll
                    for (int j = 3; j >= 1; --j) {
                        if (key[j] < kInf && sp < kBvhStack) {
                            stk[sp] = make_int2(c[j], __float_as_int(key[j]));
                            ++sp;
                        }
                    }
                    node = c[0];
                    n0 = key[0];
                    continue;
                }
            } else {
                const float4 *nd = sc.nodes + (size_t)node * kNodeF4;
                float4 q[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) q[k] = __ldg(nd + k);
                const int2 ch = __ldg(reinterpret_cast<const int2 *>(nd + 3));
                float a0, a1, b0, b1;
                node_child_boxes<3>(q, r, tmin, tmax, G, a0, a1, b0, b1);
                bool ha = a0 <= a1 && ch.x != kEmptyChild;
                bool hb = b0 <= b1 && ch.y != kEmptyChild;
                if (ha && a0 > bound) {
                    ha = false;
                    evicted = true;
                    t_evict = fminf(t_evict, a0);
                }
                if (hb && b0 > bound) {
                    hb = false;
                    evicted = true;
                    t_evict = fminf(t_evict, b0);
                }
                if (ha && hb) {
                    const bool bfirst = b0 < a0;
                    if (sp < kBvhStack) {
                        stk[sp] = make_int2(bfirst ? ch.x : ch.y, __float_as_int(bfirst ? a0 : b0));
                        ++sp;
                    }
                    node = bfirst ? ch.y : ch.x;
                    n0 = bfirst ? b0 : a0;
                    continue;
                }
                if (ha || hb) {
                    node = ha ? ch.x : ch.y;
                    n0 = ha ? a0 : b0;
                    continue;
                }
            }
        }
        // pop the nearest pending subtree that can still add to the list
        node = kDone;
        while (sp > 0) {
            --sp;
            const int2 e = stk[sp];
            const float t0 = __int_as_float(e.y);
            if (cnt == C && t0 > kt[C - 1]) {
                evicted = true;
                t_evict = fminf(t_evict, t0);
                continue;
            }
            node = e.x;
            n0 = t0;
            break;
        }
    }
    return true;
}

// The ray of candidate-pass thread t.  With img_w > 0 (a multiple of 8) the rays are an image of that width,
// ray y * img_w + x, and each warp takes a tile of 8 x 4 pixels, whose rays walk more of the same BVH nodes
// than a row of 32; the threads then cover whole bands of 4 rows (cand_threads), and those past the last ray
// have none.  A bijection of [0, cand_threads) onto the same range either way.
CCS_DEV uint32_t cand_ray(uint32_t t, uint32_t img_w)
{
    if (img_w == 0u) return t;
    const uint32_t w = t >> 5, l = t & 31u, tiles_x = img_w >> 3;
    const uint32_t ty = w / tiles_x, tx = w - ty * tiles_x;
    return (ty * 4u + (l >> 3)) * img_w + tx * 8u + (l & 7u);
}
inline uint32_t cand_threads(uint32_t n, uint32_t img_w)
{
    if (img_w == 0u) return n;
    const uint64_t band = 4ull * img_w;
    return (uint32_t)((n + band - 1) / band * band);
}

template <bool STATS, int MODE, class Src, int BW>
__global__ void __launch_bounds__(kCandBlock) k_cand(Src src, PairBufs pb, uint32_t img_w, uint32_t iter_cap,
                                              uint32_t *status, unsigned long long *counters, uint8_t *occluded)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t n = src.total();
    const uint32_t i = cand_ray(blockIdx.x * blockDim.x + threadIdx.x, img_w);
    constexpr int C = kPairCands;
    const float kInf = __int_as_float(0x7f800000);
    float kt[C];
    uint32_t kp[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        kt[j] = kInf;
        kp[j] = kMissId;
    }
    int cnt = 0;
    float t_evict = kInf;
    bool evicted = false, live = false, capped = false;
    uint32_t ray_scene = 0, ray_local = 0;
    typename Src::LaneScene lsc;
    unsigned long long nodes = 0, culled = 0;
    Grp G;
    G.c = 0;
    G.mask = FULL;
    G.l0 = G.l1 = G.l2 = lane;
    float ro[3] = {0.0f, 0.0f, 0.0f}, rd[3] = {0.0f, 0.0f, 0.0f}, tmin = 0.0f, tmax = 0.0f;
    if (i < n) {
        live = true;
        src.locate(i, lsc, ray_scene, ray_local);
        const DevScene &sc = src.scene(lsc);
        RayG<3> r;
        const bool ok = load_world_ray(src.rays_of(ray_scene), ray_local, r.org, rd, r.inv, tmin, tmax);
        ro[0] = r.org[0];
        ro[1] = r.org[1];
        ro[2] = r.org[2];
        if (ok && sc.n_nodes != 0) {
            uint32_t it = iter_cap;
            capped = !walk_candidates<STATS, BW>(sc, r, ro, rd, tmin, tmax, false, 0.0f, 0u, it, kt, kp, cnt, t_evict,
                                                 evicted, nodes, culled, G);
        }
    }
    // the task: the candidates in list order in one run of the buffer; its cost class
    const bool has = live && !capped && cnt > 0;
    int key = -1;
    if (has) {
        const DevScene &sc = src.scene(lsc);
        int ng = 0;
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (j < cnt && __ldg(sc.types + kp[j]) != 0) ++ng;
        // rays with a Gregory candidate first: their pairs then share warps, so fewer warp iterations pay
        // for the bound of Algorithm 2 with a single Gregory lane; the others by their number of candidates
        key = ng > 0 ? kCostClasses - 1 : min(kCostClasses - 2, cnt);
    }
    const uint32_t want = has ? (uint32_t)cnt : 0u;
    const unsigned lt = (1u << lane) - 1u;
    if (has) {
        const size_t off = (size_t)i * C;
        uint2 *dst = pb.cand + off;
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (j < cnt) dst[j] = make_uint2(kp[j], __float_as_uint(kt[j]));
        uint4 *tk = pb.task + 4 * (size_t)i;
        tk[0] = make_uint4(i, (uint32_t)off, (uint32_t)cnt | ((uint32_t)key << 8) | (evicted ? kTaskEvicted : 0u),
                           __float_as_uint(t_evict));
        tk[1] = make_uint4(kp[0], __float_as_uint(kt[0]), __float_as_uint(tmin), __float_as_uint(tmax));
        tk[2] = make_uint4(__float_as_uint(ro[0]), __float_as_uint(ro[1]), __float_as_uint(ro[2]), __float_as_uint(rd[0]));
        tk[3] = make_uint4(__float_as_uint(rd[1]), __float_as_uint(rd[2]), 0u, 0u);
    }
    // the task's place in the list of its class
    const int hkey = has ? key : -1;
    const unsigned same = __match_any_sync(FULL, hkey);
    const int leader = __ffs(same) - 1;
    uint32_t cb = 0;
    if (has && lane == leader) cb = atomicAdd(pb.ctr + kCtrHist + key, (uint32_t)__popc(same));
    cb = __shfl_sync(FULL, cb, leader);
    if (has) pb.cls[(size_t)key * pb.n + cb + __popc(same & lt)] = i;
    if (live && !has) {
        if (capped) atomicOr(status, 1u);
        write_miss<MODE>(src, ray_scene, ray_local, occluded);
    }
    if (STATS) {   // BVH nodes; diagnostics in the schedule slots: candidates listed, rays that dropped some,
                   // candidates culled by their root box
        unsigned long long v[4] = {nodes, want, (unsigned long long)(has && evicted), culled};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], o);
        if (lane == 0) {
            if (v[0]) atomicAdd(counters + 0, v[0]);
            if (v[1]) atomicAdd(counters + 8, v[1]);
            if (v[2]) atomicAdd(counters + 9, v[2]);
            if (v[3]) atomicAdd(counters + 17, v[3]);
        }
    }
}

// The next candidates of a ray whose best hit may lie among those the candidate pass dropped: a walk of the
// BVH by one lane for the kPairCands smallest keys above (lb_t, lb_p), the last listed, written to the ray's
// candidate places.  The ray comes from the lane's task slot in shared memory (rs, strided).  Rare: rays
// with more candidates than the list holds, whose best hit is not before the first dropped one.
struct MoreCands {
    int cnt;          // candidates written (0: none left)
    float t_evict;    // smallest entry distance this walk dropped
    bool evicted, capped;
};
template <int BW>
__device__ __forceinline__ MoreCands collect_more(const DevScene sc, const float *rs, int stride, float lb_t,
                                               uint32_t lb_p, uint32_t iter_cap, uint2 *dst)
{
    constexpr int C = kPairCands;
    RayG<3> r;
    float ro[3], rd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ro[k] = r.org[k] = rs[k * stride];
        r.inv[k] = rs[(3 + k) * stride];
        rd[k] = rs[(9 + k) * stride];
    }
    float kt[C];
    uint32_t kp[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        kt[j] = __int_as_float(0x7f800000);
        kp[j] = kMissId;
    }
    MoreCands out;
    out.cnt = 0;
    out.t_evict = __int_as_float(0x7f800000);
    out.evicted = false;
    unsigned long long nodes = 0, culled = 0;
    Grp G;
    G.c = 0;
    G.mask = 0xffffffffu;
    G.l0 = G.l1 = G.l2 = threadIdx.x & 31;
    uint32_t it = iter_cap;
    out.capped = !walk_candidates<false, BW>(sc, r, ro, rd, rs[6 * stride], rs[7 * stride], true, lb_t, lb_p, it, kt, kp,
                                             out.cnt, out.t_evict, out.evicted, nodes, culled, G);
    if (!out.capped)
        for (int j = 0; j < out.cnt; ++j) dst[j] = make_uint2(kp[j], __float_as_uint(kt[j]));
    return out;
}

// ------------------------------------------------------------------------------------------------
// Pass 3: Algorithm 3 over (ray, patch) pairs, one pair per lane.
// ------------------------------------------------------------------------------------------------
template <bool STATS, int K, int MODE, class Src>
__global__ void __launch_bounds__(128, 3) k_pairs(Src src, PairBufs pb, int L, uint32_t refill, uint32_t iter_cap,
                                                  uint32_t *status, unsigned long long *counters, uint8_t *occluded)
{
    extern __shared__ __align__(16) float smem[];
    const int stride = blockDim.x;
    Scratch scr;
    scr.stride = stride;
    scr.cstride = cache_floats(K, 3);
    scr.cache = smem + threadIdx.x * scr.cstride;
    scr.tag = reinterpret_cast<int *>(scr.cache + 48 * K);
    scr.sib = reinterpret_cast<float2 *>(smem + cache_floats(K, 3) * stride) + threadIdx.x;
    scr.node = nullptr;
    float *rs = smem + scratch_floats(L, K, 3) * stride + threadIdx.x;   // [k * stride], k < kRaySlotFloats
    // mailboxes, helper counts and cap flags of the block's threads (indexed by thread)
    unsigned long long *mbox =
        reinterpret_cast<unsigned long long *>(smem + (scratch_floats(L, K, 3) + kRaySlotFloats) * stride);
    int *hcount = reinterpret_cast<int *>(mbox + stride);
    int *hcap = hcount + stride;
    const int wbase = threadIdx.x & ~31;
    mbox[threadIdx.x] = ~0ull;
    hcount[threadIdx.x] = 0;
    hcap[threadIdx.x] = 0;
    // the queue hands out the tasks class by class, costliest first: cstart[c] = first place of class c
    __shared__ uint32_t cstart[kCostClasses + 1];
    if (threadIdx.x < kCostClasses) {
        uint32_t a = 0;
        for (int c = kCostClasses - 1; c > (int)threadIdx.x; --c) a += pb.ctr[kCtrHist + c];
        cstart[threadIdx.x] = a;
        if (threadIdx.x == 0) cstart[kCostClasses] = a + pb.ctr[kCtrHist];   // all tasks
    }
    __syncthreads();
    Counters cnt;
#pragma unroll
    for (int k = 0; k < kNumSumCounters; ++k) cnt.v[k] = 0;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    Grp G;
    G.c = 0;
    G.mask = FULL;
    G.l0 = G.l1 = G.l2 = lane;
    const float kInf = __int_as_float(0x7f800000);
    const float cellw = __int_as_float((127 - L) << 23);
    const uint32_t n_tasks = cstart[kCostClasses];
    uint32_t *queue = pb.ctr + kCtrQueue;
    if (STATS && lane == 0) atomicMax(counters + 20, ~global_ns());   // first warp start

    // the lane's ray (task)
    bool has_task = false, exhausted = false, evicted = false;
    uint32_t ray = 0, cur = 0, ray_scene = 0, ray_local = 0, iters = 0;
    uint2 nxt = make_uint2(0u, 0u);   // the ray's candidate at cur, loaded ahead
    typename Src::LaneScene lsc;
    Best best;
    best.t = 0.0f;
    best.pid = best.cell = kMissId;
    best.lvl = 0;
    // the lane's pair
    bool in_pair = false, want_root = false, start = false, gpend = false, greg = false;
    bool helper = false, waiting = false;   // a subtree of lane `owner`'s pair; waiting for helpers
    int owner = lane;
    uint32_t pid = 0, start_pid = 0, path = 0, trail = 0;
    RayG<3> pr;
    float tau = 0.0f, c0 = 0.0f, c1 = 0.0f, te = 0.0f;   // intervals are distances from the anchored origin
    float d[3] = {0.0f, 0.0f, 0.0f};
    int level = 0, rd_target = -1, ctop = 0, cvalid = 0;
    float g[48];

    for (;;) {
        // (1) a lane whose pair has ended takes its ray's next candidate (collecting more when dropped
        //     candidates may still hold the answer), or writes the ray's answer; idle lanes take new rays
        //     from the queue, then their first candidate
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            if (has_task && !in_pair && !start) {
                if (cur < __float_as_uint(rs[13 * stride]) && __uint_as_float(nxt.y) <= best.t) {
                    start = true;
                    start_pid = nxt.x;
                    ++cur;
                } else {   // entries are sorted: the rest enter later still
                    // the answer may lie among the candidates the walk dropped (entries from t_evict on): this
                    // lane collects the next ones, after the last listed, by a walk of its own
                    bool finish = true;
                    if (evicted && (MODE == kModeAnyHit ? best.pid == kMissId : !(best.t < rs[8 * stride]))) {
                        const uint2 last = pb.cand[__float_as_uint(rs[13 * stride]) - 1];
                        const uint32_t cbase = __float_as_uint(rs[12 * stride]);
                        const DevScene &sc = src.scene(lsc);
                        const MoreCands mc =
                            sc.width == 4
                                ? collect_more<4>(sc, rs, stride, __uint_as_float(last.y), last.x, iter_cap, pb.cand + cbase)
                                : collect_more<2>(sc, rs, stride, __uint_as_float(last.y), last.x, iter_cap, pb.cand + cbase);
                        if (STATS) cnt.v[10]++;
                        evicted = mc.evicted;
                        if (mc.capped) {   // iteration cap of the walk: a miss, status latched
                            finish = false;
                            has_task = false;
                            atomicOr(status, 1u);
                            write_miss<MODE>(src, ray_scene, ray_local, occluded);
                        } else if (mc.cnt > 0) {
                            finish = false;
                            cur = cbase;
                            rs[13 * stride] = __uint_as_float(cbase + (uint32_t)mc.cnt);
                            nxt = pb.cand[cbase];
                            rs[8 * stride] = mc.t_evict;
                        }
                    }
                    if (finish) {   // the ray's answer
                        has_task = false;
                        if (MODE == kModeAnyHit) {
                            occluded[ray_local] = best.pid != kMissId ? 1 : 0;
                        } else {
                            const DevHits &hh = src.hits_of(ray_scene);
                            const uint32_t j = ray_local;
                            if (best.pid != kMissId) {
                                const uint32_t cu = best.cell & ((1u << L) - 1u), cv = best.cell >> L;
                                hh.t[j] = best.t;
                                hh.u[j] = ((float)cu + 0.5f) * cellw;
                                hh.v[j] = ((float)cv + 0.5f) * cellw;
                                hh.pid[j] = best.pid;
                            } else {
                                hh.t[j] = kInf;
                                hh.u[j] = 0.0f;
                                hh.v[j] = 0.0f;
                                hh.pid[j] = kMissId;
                            }
                        }
                    }
                }
            }
            if (pass == 1 || exhausted) break;
            const unsigned idle = __ballot_sync(FULL, !has_task);
            if (idle == 0u || ((uint32_t)__popc(idle) < refill && idle != FULL)) break;
            uint32_t qb = 0;
            if (lane == 0) qb = atomicAdd(queue, (uint32_t)__popc(idle));
            qb = __shfl_sync(FULL, qb, 0);
            if (qb + (uint32_t)__popc(idle) >= n_tasks) {
                exhausted = true;
                if (STATS && lane == 0) atomicMax(counters + 21, ~global_ns());   // queue found empty
            }
            const uint32_t k = qb + (uint32_t)__popc(idle & lt);
            if (!has_task && k < n_tasks) {
                int c = kCostClasses - 1;
                while (c > 0 && k >= cstart[c - 1]) --c;
                const uint4 *tp = pb.task + 4 * (size_t)__ldg(pb.cls + (size_t)c * pb.n + (k - cstart[c]));
                const uint4 w0 = tp[0], w1 = tp[1], w2 = tp[2], w3 = tp[3];
                has_task = true;
                ray = w0.x;
                cur = w0.y;
                rs[12 * stride] = __uint_as_float(w0.y);
                rs[13 * stride] = __uint_as_float(w0.y + (w0.z & 255u));
                evicted = (w0.z & kTaskEvicted) != 0u;
                nxt = make_uint2(w1.x, w1.y);
                rs[0 * stride] = __uint_as_float(w2.x);
                rs[1 * stride] = __uint_as_float(w2.y);
                rs[2 * stride] = __uint_as_float(w2.z);
                rs[3 * stride] = safe_inv(__uint_as_float(w2.w));
                rs[4 * stride] = safe_inv(__uint_as_float(w3.x));
                rs[5 * stride] = safe_inv(__uint_as_float(w3.y));
                rs[6 * stride] = __uint_as_float(w1.z);
                rs[7 * stride] = __uint_as_float(w1.w);
                rs[8 * stride] = __uint_as_float(w0.w);
                rs[9 * stride] = __uint_as_float(w2.w);
                rs[10 * stride] = __uint_as_float(w3.x);
                rs[11 * stride] = __uint_as_float(w3.y);
                src.locate(ray, lsc, ray_scene, ray_local);
                iters = iter_cap;
                best.t = __uint_as_float(w1.w);
                best.pid = best.cell = kMissId;
            }
        }
        // (2) the lanes that start a pair: the next candidate ahead, root interval, the ray in the patch
        //     frame, and (Bezier) the root grid
        if (start) {
            start = false;
            if (cur < __float_as_uint(rs[13 * stride])) nxt = pb.cand[cur];
            const DevScene &sc = src.scene(lsc);
            pid = start_pid;
            const float4 *rec = rec_of(sc, pid);
            const float4 an = __ldg(rec + 15);
            in_pair = true;
            greg = an.w != 0.0f;
            if (STATS) cnt.v[7]++;
            RayG<3> wr;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                wr.org[k] = rs[k * stride];
                wr.inv[k] = rs[(3 + k) * stride];
            }
            const float tmin = rs[6 * stride];
            {   // the root interval: the slab of the patch box from tmin (as k_intersect computes it)
                const float4 blo = __ldg(sc.leaf_box + 2 * (size_t)pid), bhi = __ldg(sc.leaf_box + 2 * (size_t)pid + 1);
                const float lo[3] = {blo.x, blo.y, blo.z}, hi[3] = {bhi.x, bhi.y, bhi.z};
                slab<3>(wr, lo, hi, tmin, kInf, G, c0, c1);
            }
            {
                const float dw[3] = {rs[9 * stride], rs[10 * stride], rs[11 * stride]};
                te = c0;
                anchored_ray<3>(rec, an, sc.local != 0, wr.org, dw, wr.inv, c0, G, pr);
                c1 = __fsub_rn(c1, c0);
                c0 = 0.0f;
            }
            tau = 0.0f;
            if (sc.local) {   // box extension (Sec. 3.4)
                float o3[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) o3[c] = wr.org[c] - pick(c, an.x, an.y, an.z);
                tau = pair_tau(o3);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) d[k] = 0.0f;
            level = 0;
            rd_target = -1;
            path = trail = 0u;
            ctop = cvalid = 0;
            gpend = greg;
            want_root = !greg;
        }
        if (want_root) {   // a Bezier pair's start or a re-descent: the root grid
            want_root = false;
            load_grid<3>(rec_of(src.scene(lsc), pid), G, g);
        }
        if (STATS) {   // schedule of this warp iteration, in lanes (slots 12..16)
            const unsigned ks = __ballot_sync(FULL, in_pair && !waiting), kh = __ballot_sync(FULL, helper);
            const unsigned kw = __ballot_sync(FULL, waiting), ki = __ballot_sync(FULL, !in_pair && !has_task);
            if (lane == 0) {
                cnt.v[12] += 1;
                cnt.v[13] += __popc(ks);
                cnt.v[14] += __popc(kh);
                cnt.v[15] += __popc(kw);
                cnt.v[16] += __popc(ki);
            }
        }
        // (3) subdivision steps of every lane's pair: the iteration cap first
        if (in_pair && !waiting && iters == 0) {
            if (helper) {   // iteration cap in a subtree: the owner's ray becomes a capped miss
                atomicOr(status, 1u);
                hcap[wbase + owner] = 1;
                __threadfence_block();
                atomicSub(hcount + wbase + owner, 1);
                helper = false;
                in_pair = false;
            } else if (hcount[threadIdx.x] > 0) {   // wait for the subtrees, then the cap
                hcap[threadIdx.x] = 1;
                waiting = true;
            } else {   // iteration cap: a miss, status latched
                has_task = false;
                in_pair = false;
                atomicOr(status, 1u);
                if (MODE == kModeAnyHit) {
                    occluded[ray_local] = 0;
                } else {
                    const DevHits &hh = src.hits_of(ray_scene);
                    hh.t[ray_local] = kInf;
                    hh.u[ray_local] = 0.0f;
                    hh.v[ray_local] = 0.0f;
                    hh.pid[ray_local] = kMissId;
                }
            }
        }
        // up to kStepsPerIter steps (Algorithm 3's loop body) per warp iteration: after the first, the lanes
        // whose pair keeps descending (no leaf, no backtrack, no Gregory bound due) step again, so that the
        // divergent rest of the iteration is paid once for more steps
        bool stepping = in_pair && !waiting && iters > 0, back = false;
#pragma unroll 1
        for (int pass = 0; pass < kStepsPerIter; ++pass) {
            if (pass > 0 && !__any_sync(FULL, stepping)) break;
            if (stepping) {
                --iters;
                if (gpend) {   // Algorithm 2 with the crop of Algorithm 1 for the Gregory node (path, level)
                    float u0, u1, v0, v1;
                    node_domain(path, level, L, u0, u1, v0, v1);
                    gregory_node<3>(rec_of(src.scene(lsc), pid), u0, u1, v0, v1, level, G, g, d);
                    gpend = false;
                }
                const bool redesc = rd_target >= 0;
                const bool leafkids = !redesc && level + 1 == 2 * L;
                const int force = redesc ? (int)((path >> level) & 1u) : -1;
                const int slot = (!redesc && !leafkids && K > 0 && !greg) ? (ctop % (K > 0 ? K : 1)) : -1;
                if (STATS && !redesc) cnt.v[greg ? 2 : 1]++;
                const StepOut so = split_step<K, 3>(g, pr, d, c0, c1, te, best.t, redesc || (!greg && !leafkids), scr,
                                                    slot, true, true, force, G, tau);
                if (redesc) {
                    if (++level == rd_target) rd_target = -1;
                } else if (so.hitL || so.hitR) {
                    const uint32_t bit = 1u << level;
                    if (leafkids) {   // both children are leaves: record them here (key order, A14/A15)
                        uint32_t cu, cv;
                        if (so.hitL) {
                            path_cells(path, L, cu, cv);
                            const uint32_t cell = (cv << L) | cu;
                            const float tk = __fadd_rn(te, so.l0);
                            if (key_less(tk, pid, cell, best)) {
                                best.t = tk;
                                best.pid = pid;
                                best.cell = cell;
                            }
                        }
                        if (so.hitR) {
                            path_cells(path | bit, L, cu, cv);
                            const uint32_t cell = (cv << L) | cu;
                            const float tk = __fadd_rn(te, so.r0);
                            if (key_less(tk, pid, cell, best)) {
                                best.t = tk;
                                best.pid = pid;
                                best.cell = cell;
                            }
                        }
                        if (STATS) cnt.v[3] += (so.hitL ? 1 : 0) + (so.hitR ? 1 : 0);
                        back = true;
                    } else {
                        if (so.hitL && so.hitR) {
                            trail |= bit;
                            scr.sib[level * stride] = so.goR ? make_float2(so.l0, so.l1) : make_float2(so.r0, so.r1);
                            if (K > 0 && !greg) {
                                scr.tag[slot] = level;
                                ++ctop;
                                cvalid = cvalid < K ? cvalid + 1 : K;
                            }
                        }
                        path = so.goR ? (path | bit) : path;
                        c0 = so.goR ? so.r0 : so.l0;
                        c1 = so.goR ? so.r1 : so.l1;
                        ++level;
                        gpend = greg;
                    }
                } else {
                    back = true;
                }
                stepping = !back && !gpend && iters > 0;
            }
        }
        if (back) {   // the deepest pending sibling that may still hold a closer leaf, or the pair ends
            bool found = false;
            if (!(MODE == kModeAnyHit && best.pid != kMissId)) {
                while (trail != 0u) {
                    const int l = 31 - __clz(trail);
                    const uint32_t bit = 1u << l;
                    trail ^= bit;
                    bool cached = false;
                    int cslot = 0;
                    if (K > 0 && !greg && cvalid > 0) {
                        cslot = (ctop - 1) % (K > 0 ? K : 1);
                        if (scr.tag[cslot] == l) {
                            cached = true;
                            --ctop;
                            --cvalid;
                        }
                    }
                    const float2 sb = scr.sib[l * stride];
                    if (__fadd_rn(te, sb.x) > best.t) {
                        if (STATS) cnt.v[6]++;
                        continue;
                    }
                    path = (path & (bit - 1u)) | (~path & bit);
                    c0 = sb.x;
                    c1 = sb.y;
                    if (STATS) cnt.v[4]++;
                    if (greg) {
                        level = l + 1;
                        gpend = true;
                    } else if (cached) {
                        level = l + 1;
                        load_cached<3>(scr.cache + cslot * 48, g);
                    } else {
                        if (STATS) cnt.v[5] += l + 1;
                        level = 0;
                        rd_target = l + 1;
                        want_root = true;
                    }
                    found = true;
                    break;
                }
            } else {
                cur = __float_as_uint(rs[13 * stride]);   // any hit: the ray is answered
            }
            if (!found) {
                if (helper) {   // the subtree is searched: its best leaf to the owner's mailbox
                    if (best.pid == pid)
                        atomicMin(mbox + wbase + owner, ((unsigned long long)ord_bits(best.t) << 32) | best.cell);
                    __threadfence_block();
                    atomicSub(hcount + wbase + owner, 1);
                    helper = false;
                    in_pair = false;
                } else {
                    waiting = true;   // merged when every subtree handed out is searched
                }
            }
        }
        // a lane whose search has ended takes the best leaf of the subtrees it handed out, once every one of
        // them is searched (until then it waits)
        __syncwarp();
        if (waiting && hcount[threadIdx.x] == 0) {
            __threadfence_block();
            const unsigned long long mk = mbox[threadIdx.x];
            if (mk != ~0ull) {
                const float mt = unord_bits((uint32_t)(mk >> 32));
                const uint32_t mc = (uint32_t)mk;
                if (key_less(mt, pid, mc, best)) {
                    best.t = mt;
                    best.pid = pid;
                    best.cell = mc;
                }
                mbox[threadIdx.x] = ~0ull;
            }
            waiting = false;
            in_pair = false;
            if (hcap[threadIdx.x]) {   // a subtree reached the iteration cap: answered as a capped ray
                hcap[threadIdx.x] = 0;
                iters = 0;
                in_pair = true;
            }
        }
        // (4) once the queue is empty, idle lanes take a pending subtree of a busy lane of the warp
        //     (closest-hit mode): the deepest one when its grid is in the busy lane's sibling cache or the
        //     patch is a Gregory patch (no re-descent), else the shallowest one of at least
        //     kMinDonateLevels levels (re-descended); the key of a pair's best leaf is the minimum over its
        //     subtrees
        if (MODE == kModePlain && exhausted) {
            const bool idle_l = !has_task && !in_pair;
            const int lmin = trail != 0u ? __ffs(trail) - 1 : 2 * L;
            const int ldeep = trail != 0u ? 31 - __clz(trail) : 2 * L;
            int cslot = -1;
            if (K > 0 && !greg && cvalid > 0 && trail != 0u) {
                const int c = (ctop - 1) % (K > 0 ? K : 1);
                if (scr.tag[c] == ldeep) cslot = c;
            }
            const bool deep = trail != 0u && (greg || cslot >= 0);
            const int lgive = deep ? ldeep : lmin;
            const bool can_give = in_pair && !waiting && (deep || 2 * L - (lmin + 1) >= kMinDonateLevels);
            const unsigned T = __ballot_sync(FULL, idle_l), D = __ballot_sync(FULL, can_give);
            if (T != 0u && D != 0u) {
                const int m = min(__popc(T), __popc(D));
                int from = lane;
                if (idle_l && __popc(T & lt) < m) from = (int)__fns(D, 0, __popc(T & lt) + 1);
                const bool gives = can_give && __popc(D & lt) < m;
                uint32_t sp = 0u;
                float sx = 0.0f, sy = 0.0f;
                int gslot = -1;   // the donor's cache slot holding the subtree root's grid
                if (gives) {   // the sibling's path and interval, as a backtrack to it would set them
                    const uint32_t bit = 1u << lgive;
                    sp = (path & (bit - 1u)) | (~path & bit);
                    const float2 sb = scr.sib[lgive * stride];
                    sx = sb.x;
                    sy = sb.y;
                    trail ^= bit;
                    if (deep && cslot >= 0) {
                        gslot = cslot;
                        --ctop;
                        --cvalid;
                    }
                }
                const int x_gslot = __shfl_sync(FULL, gslot, from);
                const uint32_t x_pid = __shfl_sync(FULL, pid, from);
                const int x_greg = __shfl_sync(FULL, greg ? 1 : 0, from);
                float x_pr[6];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    x_pr[k] = __shfl_sync(FULL, pr.org[k], from);
                    x_pr[3 + k] = __shfl_sync(FULL, pr.inv[k], from);
                }
                const float x_tau = __shfl_sync(FULL, tau, from);
                const float x_te = __shfl_sync(FULL, te, from);
                const float x_bt = __shfl_sync(FULL, best.t, from);
                const uint32_t x_bp = __shfl_sync(FULL, best.pid, from);
                const uint32_t x_bc = __shfl_sync(FULL, best.cell, from);
                const uint32_t x_sp = __shfl_sync(FULL, sp, from);
                const int x_sl = __shfl_sync(FULL, lgive, from);
                const float x_sx = __shfl_sync(FULL, sx, from);
                const float x_sy = __shfl_sync(FULL, sy, from);
                const int x_owner = __shfl_sync(FULL, helper ? owner : lane, from);
                share_scene<Src>(lsc, from);
                if (idle_l && from != lane) {   // a helper on the subtree below the sibling
                    helper = true;
                    in_pair = true;
                    owner = x_owner;
                    pid = x_pid;
                    greg = x_greg != 0;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        pr.org[k] = x_pr[k];
                        pr.inv[k] = x_pr[3 + k];
                        d[k] = 0.0f;
                    }
                    tau = x_tau;
                    te = x_te;
                    best.t = x_bt;
                    best.pid = x_bp;
                    best.cell = x_bc;
                    path = x_sp;
                    trail = 0u;
                    c0 = x_sx;
                    c1 = x_sy;
                    ctop = cvalid = 0;
                    iters = iter_cap;
                    if (greg) {
                        level = x_sl + 1;
                        rd_target = -1;
                        gpend = true;
                    } else if (x_gslot >= 0) {   // the grid from the donor's cache slot
                        level = x_sl + 1;
                        rd_target = -1;
                        gpend = false;
                        load_cached<3>(scr.cache + (from - lane) * scr.cstride + x_gslot * 48, g);
                    } else {
                        level = 0;
                        rd_target = x_sl + 1;
                        gpend = false;
                        want_root = true;
                    }
                    atomicAdd(hcount + wbase + owner, 1);
                    if (STATS) cnt.v[11]++;
                }
            }
            __syncwarp();
        }
        if (exhausted && !__any_sync(FULL, has_task)) break;
    }
    if (STATS) {
#pragma unroll
        for (int k = 0; k < kNumSumCounters; ++k) {
            unsigned long long v = cnt.v[k];
            for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(FULL, v, o2);
            if (lane == 0 && v) atomicAdd(counters + k, v);
        }
        if (lane == 0) atomicMax(counters + 22, global_ns());   // last warp exit
    }
}

}  // namespace ccs
