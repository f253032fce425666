// Device routines of the closest-hit path: ray/box slab test, de Casteljau split with child boxes,
// Gregory lower patch and displacement (Algorithm 2 with the crop of Algorithm 1), the per-patch
// stackless bit-trail traversal (Algorithm 3) and the BVH traversal.  Shared by every kernel that
// intersects, with one lane or a group of three lanes per ray, so plain, grouped, learned and batched
// launches compute bit-identical answers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ccs_internal.h"
#include "learned.cuh"

namespace ccs {

#define CCS_DEV __device__ __forceinline__

constexpr uint32_t kMissId = 0xFFFFFFFFu;

CCS_DEV float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

CCS_DEV float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// de Casteljau midpoint: rounding of a + b, then an exact halving.  The explicit intrinsics keep the
// compiler from contracting or reassociating, so every path that computes a node computes it the same way.
CCS_DEV float mid(float a, float b) { return __fmul_rn(__fadd_rn(a, b), 0.5f); }

// Robustness factor on the far slab distance (Ize 2013, 1 + 2 gamma_3 rounded up to a float).
constexpr float kFarScale = 1.00000048f;

// ------------------------------------------------------------------------------------------------
// Components of one ray per lane.  NC = 3: a lane holds all three components of its ray.  NC = 1: a
// group of three consecutive lanes holds one ray, one component per lane (Sec. 3.5, thread groups of
// three): component-wise arithmetic (de Casteljau, box extents, the per-axis slab, Algorithm 2) runs in
// the lane of its component, and the three per-axis slab results are combined with shuffles inside the
// group.  Control state is computed identically in all three lanes of a group, so they stay converged.
// ------------------------------------------------------------------------------------------------
struct Grp {
    int c;           // first component held by this lane
    unsigned mask;   // the group's lanes (NC = 1)
    int l1, l2;      // the group's other two lanes (NC = 1)
    int l0;          // the group's lane of component 0 (NC = 1)
};

template <int NC>
CCS_DEV int comp(const Grp &G, int k)
{
    return NC == 3 ? k : G.c;
}

CCS_DEV float pick(int c, float x, float y, float z) { return c == 0 ? x : (c == 1 ? y : z); }

template <int NC>
CCS_DEV float grp_max(const Grp &G, float v)
{
    if constexpr (NC == 3) return v;
    else return max3f(v, __shfl_sync(G.mask, v, G.l1), __shfl_sync(G.mask, v, G.l2));
}

template <int NC>
CCS_DEV float grp_min(const Grp &G, float v)
{
    if constexpr (NC == 3) return v;
    else return min3f(v, __shfl_sync(G.mask, v, G.l1), __shfl_sync(G.mask, v, G.l2));
}

template <int NC>
struct RayG {
    float inv[NC];   // 1 / d (tiny components clamped so that the products stay finite)
    float org[NC];   // origin in the frame in use (world for the BVH, patch-anchored inside a patch)
};

CCS_DEV float safe_inv(float d)
{
    const float eps = 1e-20f;
    return 1.0f / (fabsf(d) < eps ? copysignf(eps, d) : d);
}

// Ray interval inside box [lo, hi], intersected with [c0, c1]: t0 = max(c0, near), t1 = min(c1, far).
// Monotone in the box bounds, so a box inside another gives an interval inside the other's.  The
// difference is rounded before the product, so a bound lying exactly on the origin gives exactly 0
// even for a clamped (huge) inverse: rays along a shared boundary plane stay inside both boxes.  The
// minima and maxima are exact, so a group of three lanes gets the same interval as a single lane.
template <int NC>
CCS_DEV void slab(const RayG<NC> &r, const float (&lo)[NC], const float (&hi)[NC], float c0, float c1, const Grp &G,
                  float &t0, float &t1)
{
    float tn, tf;
    if constexpr (NC == 3) {
        float a[3], b[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a[k] = __fmul_rn(__fsub_rn(lo[k], r.org[k]), r.inv[k]);
            b[k] = __fmul_rn(__fsub_rn(hi[k], r.org[k]), r.inv[k]);
        }
        tn = max3f(fminf(a[0], b[0]), fminf(a[1], b[1]), fminf(a[2], b[2]));
        tf = min3f(fmaxf(a[0], b[0]), fmaxf(a[1], b[1]), fmaxf(a[2], b[2]));
    } else {
        const float a = __fmul_rn(__fsub_rn(lo[0], r.org[0]), r.inv[0]);
        const float b = __fmul_rn(__fsub_rn(hi[0], r.org[0]), r.inv[0]);
        tn = grp_max<1>(G, fminf(a, b));
        tf = grp_min<1>(G, fmaxf(a, b));
    }
    t0 = fmaxf(tn, c0);
    t1 = fminf(__fmul_rn(tf, kFarScale), c1);
}

// ------------------------------------------------------------------------------------------------
// Control-point grid in registers: g[k*16 + a*4 + b], k = component held by the lane, split axis a.
// After a split the kept half is written transposed (the next split is along the other parameter), so
// every split runs the same code (Sec. 3.5: transposing the control grid removes the divergence of the
// axis).  At even tree levels a = u index i and b = v index j; at odd levels a = j and b = i.
// ------------------------------------------------------------------------------------------------

// Root grid of a Bezier record at level 0 (a = i along u): g[k][i][j] = slot 4j + i.
template <int NC>
CCS_DEV void load_grid(const float4 *__restrict__ rec, const Grp &G, float (&g)[16 * NC])
{
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float4 *pl = rec + comp<NC>(G, k) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = __ldg(pl + q);   // slots 4q .. 4q+3: j = q, i = 0..3
            g[k * 16 + 0 * 4 + q] = v.x;
            g[k * 16 + 1 * 4 + q] = v.y;
            g[k * 16 + 2 * 4 + q] = v.z;
            g[k * 16 + 3 * 4 + q] = v.w;
        }
    }
}

// Domain of the node (path, level): positions on the 2^L grid of leaf cells.
CCS_DEV uint32_t compact_even_bits(uint32_t x)
{
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// u and v cell coordinates (first split = most significant bit) of a node, on the 2^L grid
CCS_DEV void path_cells(uint32_t path, int L, uint32_t &cu, uint32_t &cv)
{
    cu = __brev(compact_even_bits(path)) >> (32 - L);
    cv = __brev(compact_even_bits(path >> 1)) >> (32 - L);
}

CCS_DEV void node_domain(uint32_t path, int level, int L, float &u0, float &u1, float &v0, float &v1)
{
    uint32_t cu, cv;
    path_cells(path & ((1u << level) - 1u), L, cu, cv);
    const int su = (level + 1) >> 1, sv = level >> 1;
    const float cell = __int_as_float((127 - L) << 23);   // 2^-L, exact
    u0 = (float)cu * cell;
    v0 = (float)cv * cell;
    u1 = u0 + __int_as_float((127 - su) << 23);           // + 2^-su, exact
    v1 = v0 + __int_as_float((127 - sv) << 23);
}

// ------------------------------------------------------------------------------------------------
// Gregory patches (Sec. 3.2): Algorithm 2 with the crop of Algorithm 1, in FP32.
// Weight of p^u (Algorithm 2's convention): h_11 = u/(u+v), h_21 = (1-u)/((1-u)+v),
// h_12 = u/(u+(1-v)), h_22 = (1-u)/((1-u)+(1-v)); each is monotone in u and in v, so its extremes over
// a domain sit at two opposite corners.  0/0 cannot occur on a non-empty domain here.  Every product
// and sum is written out (fmaf where fused), so all kernels round a node's points the same way.
// ------------------------------------------------------------------------------------------------

CCS_DEV float ratio(float a, float b)
{
    const float s = a + b;
    return s == 0.0f ? 0.5f : __fdiv_rn(a, s);
}

CCS_DEV void bern4(float t, float (&B)[4], float (&D)[4])
{
    const float s = 1.0f - t;
    B[0] = s * s * s;
    B[1] = 3.0f * t * s * s;
    B[2] = 3.0f * t * t * s;
    B[3] = t * t * t;
    D[0] = -3.0f * s * s;
    D[1] = 3.0f * s * fmaf(-2.0f, t, s);
    D[2] = 3.0f * t * fmaf(2.0f, s, -t);
    D[3] = 3.0f * t * t;
}

CCS_DEV float wbar1(float t0, float t1)   // max of B_1^3 = 3t(1-t)^2 over [t0, t1]
{
    const float w = (t0 <= (1.0f / 3.0f) && t1 >= (1.0f / 3.0f)) ? (1.0f / 3.0f) : (t1 <= (1.0f / 3.0f) ? t1 : t0);
    return 3.0f * w * (1.0f - w) * (1.0f - w);
}

CCS_DEV float wbar2(float t0, float t1)   // max of B_2^3 = 3t^2(1-t) over [t0, t1]
{
    const float w = (t0 <= (2.0f / 3.0f) && t1 >= (2.0f / 3.0f)) ? (2.0f / 3.0f) : (t1 < (2.0f / 3.0f) ? t1 : t0);
    return 3.0f * w * w * (1.0f - w);
}

// Weights of a Gregory node on [u0,u1]x[v0,v1], the same for every component.
struct GregW {
    float hA[4], hB[4], wk[4];                                    // extreme inner weights, weight bounds
    float Bu0[4], Du0[4], Bu1[4], Du1[4], Bv0[4], Dv0[4], Bv1[4], Dv1[4];   // Bernstein values, derivatives
    float Du, Dv, Duv;                                            // (u1-u0)/3, (v1-v0)/3, product
};

CCS_DEV void gregory_weights(float u0, float u1, float v0, float v1, GregW &W)
{
    // extreme weights of the four inner points: (1,1), (2,1), (1,2), (2,2)
    W.hA[0] = ratio(u0, v1);
    W.hA[1] = ratio(1.0f - u0, v0);
    W.hA[2] = ratio(u1, 1.0f - v1);
    W.hA[3] = ratio(1.0f - u1, 1.0f - v0);
    W.hB[0] = ratio(u1, v0);
    W.hB[1] = ratio(1.0f - u1, v1);
    W.hB[2] = ratio(u0, 1.0f - v0);
    W.hB[3] = ratio(1.0f - u0, 1.0f - v1);
    const float wu1 = wbar1(u0, u1), wu2 = wbar2(u0, u1), wv1 = wbar1(v0, v1), wv2 = wbar2(v0, v1);
    W.wk[0] = wu1 * wv1;
    W.wk[1] = wu2 * wv1;
    W.wk[2] = wu1 * wv2;
    W.wk[3] = wu2 * wv2;
    bern4(u0, W.Bu0, W.Du0);
    bern4(u1, W.Bu1, W.Du1);
    bern4(v0, W.Bv0, W.Dv0);
    bern4(v1, W.Bv1, W.Dv1);
    W.Du = (u1 - u0) * (1.0f / 3.0f);
    W.Dv = (v1 - v0) * (1.0f / 3.0f);
    W.Duv = W.Du * W.Dv;
}

// Component c of the node's lower patch, cropped (Algorithm 1), written into g[k*16 ..] oriented for a
// split at a level of parity `odd`; dd receives component c of the upper bound's displacement.
template <int N>
CCS_DEV void gregory_comp(const float4 *__restrict__ rec, int c, const GregW &W, bool odd, float (&g)[N], int k,
                          float &dd)
{
    const int inner[4] = {5, 6, 9, 10};
    float p[16];
    const float4 *pl = rec + c * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = __ldg(pl + q);
        p[4 * q + 0] = v.x;
        p[4 * q + 1] = v.y;
        p[4 * q + 2] = v.z;
        p[4 * q + 3] = v.w;
    }
    const float4 pv4 = __ldg(rec + 12 + c);
    const float pv[4] = {pv4.x, pv4.y, pv4.z, pv4.w};
    dd = 0.0f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float pu = p[inner[m]];
        const float a = fmaf(W.hA[m], pu - pv[m], pv[m]);
        const float b = fmaf(W.hB[m], pu - pv[m], pv[m]);
        p[inner[m]] = fminf(a, b);
        dd = fmaf(W.wk[m], fabsf(a - b), dd);
    }
    // rows j: A = sum_i B_i(u) p_ij, E = sum_i B_i'(u) p_ij at u0 and u1
    float A0[4], E0[4], A1[4], E1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float a0 = 0, e0 = 0, a1 = 0, e1 = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float pij = p[4 * j + i];
            a0 = fmaf(W.Bu0[i], pij, a0);
            e0 = fmaf(W.Du0[i], pij, e0);
            a1 = fmaf(W.Bu1[i], pij, a1);
            e1 = fmaf(W.Du1[i], pij, e1);
        }
        A0[j] = a0; E0[j] = e0; A1[j] = a1; E1[j] = e1;
    }
    // corner values: f, f_u, f_v, f_uv at (u0,v0), (u1,v0), (u0,v1), (u1,v1)
    float f[4], fu[4], fv[4], fuv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float *A = (m & 1) ? A1 : A0;
        const float *E = (m & 1) ? E1 : E0;
        const float *Bv = (m & 2) ? W.Bv1 : W.Bv0;
        const float *Dv_ = (m & 2) ? W.Dv1 : W.Dv0;
        float a = 0, b = 0, cc = 0, e = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            a = fmaf(Bv[j], A[j], a);
            b = fmaf(Bv[j], E[j], b);
            cc = fmaf(Dv_[j], A[j], cc);
            e = fmaf(Dv_[j], E[j], e);
        }
        f[m] = a; fu[m] = b; fv[m] = cc; fuv[m] = e;
    }
    const float Du = W.Du, Dv = W.Dv, Duv = W.Duv;
    // Algorithm 1: q_{i,j} at slot 4j + i
    float q[16];
    q[0] = f[0];
    q[3] = f[1];
    q[12] = f[2];
    q[15] = f[3];
    q[1] = fmaf(Du, fu[0], q[0]);
    q[2] = fmaf(-Du, fu[1], q[3]);
    q[4] = fmaf(Dv, fv[0], q[0]);
    q[7] = fmaf(Dv, fv[1], q[3]);
    q[8] = fmaf(-Dv, fv[2], q[12]);
    q[11] = fmaf(-Dv, fv[3], q[15]);
    q[13] = fmaf(Du, fu[2], q[12]);
    q[14] = fmaf(-Du, fu[3], q[15]);
    q[5] = fmaf(Duv, fuv[0], fmaf(Dv, fv[0], q[1]));
    q[6] = fmaf(-Duv, fuv[1], fmaf(-Du, fu[1], q[7]));
    q[9] = fmaf(-Duv, fuv[2], fmaf(-Dv, fv[2], q[13]));
    q[10] = fmaf(Duv, fuv[3], fmaf(-Dv, fv[3], q[14]));
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) g[k * 16 + a * 4 + b] = odd ? q[4 * a + b] : q[4 * b + a];
}

// Lower bounding patch of the Gregory record restricted to [u0,u1]x[v0,v1], cropped (Algorithm 1),
// written into g oriented for a split at `level`; d receives the displacement of the upper bound.
template <int NC>
CCS_DEV void gregory_node(const float4 *__restrict__ rec, float u0, float u1, float v0, float v1, int level,
                          const Grp &G, float (&g)[16 * NC], float (&d)[NC])
{
    GregW W;
    gregory_weights(u0, u1, v0, v1, W);
#pragma unroll
    for (int k = 0; k < NC; ++k) gregory_comp(rec, comp<NC>(G, k), W, (level & 1) != 0, g, k, d[k]);
}

// ------------------------------------------------------------------------------------------------
// Closest-hit key (t, patch id, cell index).
// ------------------------------------------------------------------------------------------------
struct Best {
    float t;
    uint32_t pid, cell;
    int lvl;   // tree level of the recorded leaf (screen-space termination)
};

CCS_DEV bool key_less(float t, uint32_t pid, uint32_t cell, const Best &b)
{
    if (t != b.t) return t < b.t;
    if (pid != b.pid) return pid < b.pid;
    return cell < b.cell;
}

struct Counters {
    unsigned long long v[kNumSumCounters];
};

// ------------------------------------------------------------------------------------------------
// Shared-memory scratch of one thread: a K-slot cache of the lane's components of the most recently
// pushed Bezier siblings' grids (the thread's own rows of 16-byte words: a grid moves in 4 NC 16-byte
// accesses), the entry/exit interval of every pending sibling (one per tree level) and the prefetch slot
// of the next BVH node (both strided by the block size, so a warp's accesses hit 32 consecutive words).
// ------------------------------------------------------------------------------------------------
// Floats of a thread's cache: K slots of 16 NC floats, then the K tags in a 4-float pad.  The stride
// 16 NC K + 4 is 4 or 20 modulo 32, so the 16-byte accesses of 8 consecutive threads hit 8 distinct groups
// of 4 banks: no bank conflicts.
__host__ __device__ constexpr int cache_floats(int K, int NC) { return K > 0 ? 16 * NC * K + 4 : 0; }

struct Scratch {
    float2 *sib;     // [level * stride]
    float *cache;    // this thread's cache: slot s at cache + 16 NC s
    int *tag;        // this thread's tags: [slot]
    float4 *node;    // [k * stride], k < node_f4<BW, NC>(): prefetched float4s of a BVH node
    int stride;
    int cstride;     // floats from one thread's cache to the next thread's
};

// Copy of a cached grid (16 NC floats, 16-byte aligned) into registers.
template <int NC>
CCS_DEV void load_cached(const float *src, float (&g)[16 * NC])
{
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int q = 0; q < 4 * NC; ++q) {
        const float4 v = s4[q];
        g[4 * q + 0] = v.x;
        g[4 * q + 1] = v.y;
        g[4 * q + 2] = v.z;
        g[4 * q + 3] = v.w;
    }
}

// Asynchronous 16-byte global -> shared copy (cached in L1 and L2), per thread.
CCS_DEV void cp_async16(void *smem_dst, const void *gsrc)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
CCS_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
CCS_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One subdivision step of a Bezier/Gregory node (Algorithm 3, the body of the while loop): de Casteljau
// split of the node grid along its fixed axis, the two child boxes (Gregory: upper corner + d), both
// slab tests clipped to the node's interval, closer-first choice (ties: lower half).  Intervals are
// distances from the pair's anchored origin; a child is pruned when te + its entry exceeds the best
// distance tb.  On return g holds
// the chosen child (transposed for its own split) unless neither child is hit; if both are hit the
// other child's grid goes to the cache slot when one is given.
struct StepOut {
    bool hitL, hitR, goR;
    float l0, l1, r0, r1;
    float dL, dR;   // L1 diagonals of the child boxes (the lane's components; screen-space termination)
};

// Widen [lo, hi] symmetrically to at least tau (Sec. 3.4's box extension in local frames).
CCS_DEV void extend(float &lo, float &hi, float tau)
{
    const float w = __fsub_rn(hi, lo);
    if (w < tau) {
        const float e = __fmul_rn(__fsub_rn(tau, w), 0.5f);
        lo = __fsub_rn(lo, e);
        hi = __fadd_rn(hi, e);
    }
}

// Minimum and maximum of 16 values in 8 operations (three-input min/max; exact, so the grouping does not
// change the result).
CCS_DEV float min16(float a0, float a1, float a2, float a3, float a4, float a5, float a6, float a7, float a8,
                    float a9, float a10, float a11, float a12, float a13, float a14, float a15)
{
    return fminf(min3f(min3f(a0, a1, a2), min3f(a3, a4, a5), min3f(a6, a7, a8)),
                 min3f(min3f(a9, a10, a11), min3f(a12, a13, a14), a15));
}
CCS_DEV float max16(float a0, float a1, float a2, float a3, float a4, float a5, float a6, float a7, float a8,
                    float a9, float a10, float a11, float a12, float a13, float a14, float a15)
{
    return fmaxf(max3f(max3f(a0, a1, a2), max3f(a3, a4, a5), max3f(a6, a7, a8)),
                 max3f(max3f(a9, a10, a11), max3f(a12, a13, a14), a15));
}

template <int K, int NC>
CCS_DEV StepOut split_step(float (&g)[16 * NC], const RayG<NC> &r, const float (&d)[NC], float c0, float c1, float te,
                           float tb, bool keep_grid, const Scratch &sc, int cache_slot, bool allowL, bool allowR,
                           int force, const Grp &G, float tau)
{
    float e0[4 * NC], e3[4 * NC], m01[4 * NC], m012[4 * NC], mm[4 * NC], m123[4 * NC], m23[4 * NC];
    float lmin[NC], lmax[NC], rmin[NC], rmax[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int q = c * 4 + b;
            const float b0 = g[c * 16 + 0 * 4 + b], b1 = g[c * 16 + 1 * 4 + b];
            const float b2 = g[c * 16 + 2 * 4 + b], b3 = g[c * 16 + 3 * 4 + b];
            e0[q] = b0;
            e3[q] = b3;
            m01[q] = mid(b0, b1);
            const float m12 = mid(b1, b2);
            m23[q] = mid(b2, b3);
            m012[q] = mid(m01[q], m12);
            m123[q] = mid(m12, m23[q]);
            mm[q] = mid(m012[q], m123[q]);
        }
        // the lower half's 16 points (b0, m01, m012, mm of each column) and the upper half's (mm, m123, m23, b3)
        const int q = c * 4;
        lmin[c] = min16(e0[q], m01[q], m012[q], mm[q], e0[q + 1], m01[q + 1], m012[q + 1], mm[q + 1], e0[q + 2],
                        m01[q + 2], m012[q + 2], mm[q + 2], e0[q + 3], m01[q + 3], m012[q + 3], mm[q + 3]);
        lmax[c] = __fadd_rn(max16(e0[q], m01[q], m012[q], mm[q], e0[q + 1], m01[q + 1], m012[q + 1], mm[q + 1],
                                  e0[q + 2], m01[q + 2], m012[q + 2], mm[q + 2], e0[q + 3], m01[q + 3], m012[q + 3],
                                  mm[q + 3]),
                            d[c]);
        rmin[c] = min16(mm[q], m123[q], m23[q], e3[q], mm[q + 1], m123[q + 1], m23[q + 1], e3[q + 1], mm[q + 2],
                        m123[q + 2], m23[q + 2], e3[q + 2], mm[q + 3], m123[q + 3], m23[q + 3], e3[q + 3]);
        rmax[c] = __fadd_rn(max16(mm[q], m123[q], m23[q], e3[q], mm[q + 1], m123[q + 1], m23[q + 1], e3[q + 1],
                                  mm[q + 2], m123[q + 2], m23[q + 2], e3[q + 2], mm[q + 3], m123[q + 3], m23[q + 3],
                                  e3[q + 3]),
                            d[c]);
    }
    if (tau > 0.0f) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            extend(lmin[c], lmax[c], tau);
            extend(rmin[c], rmax[c], tau);
        }
    }
    StepOut o;
    o.dL = 0.0f;
    o.dR = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        o.dL = __fadd_rn(o.dL, __fsub_rn(lmax[c], lmin[c]));
        o.dR = __fadd_rn(o.dR, __fsub_rn(rmax[c], rmin[c]));
    }
    slab<NC>(r, lmin, lmax, c0, c1, G, o.l0, o.l1);
    slab<NC>(r, rmin, rmax, c0, c1, G, o.r0, o.r1);
    o.hitL = allowL && o.l0 <= o.l1 && __fadd_rn(te, o.l0) <= tb;
    o.hitR = allowR && o.r0 <= o.r1 && __fadd_rn(te, o.r0) <= tb;
    o.goR = force >= 0 ? force == 1 : (o.hitR && (!o.hitL || o.r0 < o.l0));
    if ((force >= 0 || o.hitL || o.hitR) && keep_grid) {
        const bool up = o.goR;
        const bool store = K > 0 && force < 0 && cache_slot >= 0 && o.hitL && o.hitR;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int q = c * 4 + b;
                const float b0 = e0[q], b3 = e3[q];   // g is overwritten in place (transposed) below
                const float k0 = up ? mm[q] : b0, k1 = up ? m123[q] : m01[q];
                const float k2 = up ? m23[q] : m012[q], k3 = up ? b3 : mm[q];
                if (K > 0 && store) {
                    // the other child, in the same transposed layout
                    float4 *dst = reinterpret_cast<float4 *>(sc.cache + cache_slot * 16 * NC);
                    dst[c * 4 + b] = make_float4(up ? b0 : mm[q], up ? m01[q] : m123[q], up ? m012[q] : m23[q],
                                                 up ? mm[q] : b3);
                }
                g[c * 16 + b * 4 + 0] = k0;
                g[c * 16 + b * 4 + 1] = k1;
                g[c * 16 + b * 4 + 2] = k2;
                g[c * 16 + b * 4 + 3] = k3;
            }
        }
    }
    return o;
}

// Slab tests against both child boxes of a BVH node; q[k] = the node's float4 of component comp(k).
template <int NC>
CCS_DEV void node_child_boxes(const float4 (&q)[NC], const RayG<NC> &r, float c0, float c1, const Grp &G, float &a0,
                              float &a1, float &b0, float &b1)
{
    float lo0[NC], hi0[NC], lo1[NC], hi1[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        lo0[k] = q[k].x;
        hi0[k] = q[k].y;
        lo1[k] = q[k].z;
        hi1[k] = q[k].w;
    }
    slab<NC>(r, lo0, hi0, c0, c1, G, a0, a1);
    slab<NC>(r, lo1, hi1, c0, c1, G, b0, b1);
}

constexpr int kBvhStack = 64;
constexpr int kDone = (int)0x80000000;    // traversal finished

// BVH node stack of one thread (local memory): node index and entry distance, one 8-byte word per
// entry.  A patch leaf's exit distance is not kept: its pair recomputes the root interval from the
// patch box.
struct BvhStack {
    int2 e[kBvhStack];
};

// Box extension of the local frames (Sec. 3.4; reading B4): tau = 2^-19 (1 + |o - anchor|_1) from the
// FP32 origin relative to the patch anchor.
CCS_DEV float pair_tau(const float (&o3)[3])
{
    return __fmul_rn(__int_as_float((127 - 19) << 23),
                     __fadd_rn(1.0f, __fadd_rn(__fadd_rn(fabsf(o3[0]), fabsf(o3[1])), fabsf(o3[2]))));
}

// Error-free transformations in FP32: a + b = s + err exactly (Knuth's TwoSum, six operations) and
// a b = p + err exactly (TwoProduct with one FMA), s and p the rounded results.
struct F2 {
    float h, l;
};
CCS_DEV F2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
CCS_DEV F2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// One coordinate of the anchored origin (o - a) + t d as an unevaluated sum h + l: both differences and
// the product are split exactly, the large parts (which cancel near the patch) are added exactly, and the
// small parts once rounded.
CCS_DEV F2 anchored_coord(float o, float a, float t, float d)
{
    const F2 s = two_sum(o, -a);
    const F2 p = two_prod(t, d);
    const F2 h = two_sum(s.h, p.h);
    return {h.h, __fadd_rn(h.l, __fadd_rn(s.l, p.l))};
}

// R . e for e = h + l: the compensated dot product (Ogita, Rump and Oishi 2005, Dot2), as accurate as the
// same sum in twice the working precision and then rounded once.
CCS_DEV float rotate_coord(const float4 &R, const F2 (&e)[3])
{
    const F2 p0 = two_prod(R.x, e[0].h), p1 = two_prod(R.y, e[1].h), p2 = two_prod(R.z, e[2].h);
    const F2 s1 = two_sum(p0.h, p1.h);
    const F2 s2 = two_sum(s1.h, p2.h);
    float c = __fadd_rn(__fadd_rn(p0.l, p1.l), __fadd_rn(s1.l, __fadd_rn(s2.l, p2.l)));
    c = __fmaf_rn(R.x, e[0].l, __fmaf_rn(R.y, e[1].l, __fmaf_rn(R.z, e[2].l, c)));
    return __fadd_rn(s2.h, c);
}

// The ray of a pair.  Sec. 3.4 anchors the patches (points relative to their box centre) to keep the
// magnitudes of the subdivision small; the ray is anchored the same way, at its entry into the patch box:
// its origin e = (o - anchor) + te d, with te the entry distance of the pair's root interval, is formed
// from the FP32 inputs without losing the cancellation to rounding (error-free transformations: about
// twice FP32's precision, as FP64 would give, but on the FP32 pipes), rotated into the patch frame (local
// frames) by a compensated dot product and rounded once.  Distances inside the pair are measured from e,
// so the slab tests subtract numbers of the size of the patch instead of the distance to the camera; a
// leaf's key distance is te + its entry.  The direction is R d in FP32 (the world direction without local
// frames), and pr.inv its inverse.  NC = 1: the group exchanges its components.
template <int NC>
CCS_DEV void anchored_ray(const float4 *__restrict__ rec, const float4 &an, bool local, const float (&o)[NC],
                          const float (&dw)[NC], const float (&winv)[NC], float te, const Grp &G, RayG<NC> &pr)
{
    F2 e[3];
    float dd[3];
    if constexpr (NC == 3) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e[c] = anchored_coord(o[c], pick(c, an.x, an.y, an.z), te, dw[c]);
            dd[c] = dw[c];
        }
    } else {
        const F2 ec = anchored_coord(o[0], pick(G.c, an.x, an.y, an.z), te, dw[0]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e[c].h = __shfl_sync(G.mask, ec.h, G.l0 + c);
            e[c].l = __shfl_sync(G.mask, ec.l, G.l0 + c);
            dd[c] = __shfl_sync(G.mask, dw[0], G.l0 + c);
        }
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int c = comp<NC>(G, k);
        if (!local) {
            pr.org[k] = __fadd_rn(e[c].h, e[c].l);
            pr.inv[k] = winv[k];
        } else {
            const float4 Rk = __ldg(rec + 16 + c);
            pr.org[k] = rotate_coord(Rk, e);
            pr.inv[k] = safe_inv(fmaf(Rk.x, dd[0], fmaf(Rk.y, dd[1], Rk.z * dd[2])));
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Per-ray state machine.  A lane (NC = 3) or a group of three lanes (NC = 1) owns one ray; every call
// of lane_step() does one unit of work: one BVH node, the start of a patch, one subdivision step of
// Algorithm 3, one level of a re-descent, or one leaf / backtrack.  All subdivision and re-descent
// steps go through one call of split_step, so lanes of a warp in different phases of Algorithm 3 stay
// converged on the expensive part.
//
// Algorithm 3 with one bit trail over tree levels:
//   path  bit l = the node at level l+1 is the upper half of its parent's split;
//   trail bit l = the sibling of that node is still pending.
// The split axis is fixed by the level (u at even levels), so one trail encodes both of the paper's
// trails.  The entry/exit interval of every pending sibling is kept in shared memory: on backtracking
// a sibling whose entry exceeds the best distance is dropped with no recomputation, and Gregory
// children are clipped to their parent's interval, which keeps the answer independent of the
// visiting order.  A Bezier sibling's grid comes from the K-slot cache when it is still there, else
// from a de Casteljau re-descent from the root along the path bits (same arithmetic as the descent).
// ------------------------------------------------------------------------------------------------
template <int NC>
struct Lane {
    float o[NC], tmin, tmax;        // ray origin (the lane's components, world frame) and interval
    float dw[NC];                   // ray direction (the lane's components, world frame)
    float te;                       // distance of the current pair's anchored origin along the ray
    RayG<NC> r;
    Best best;
    uint32_t iters;
    int node;                       // BVH: >= 0 internal node, kDone, else leaf of patch ~node
    float n0;                       // entry distance of `node`
    int sp;
    bool in_pair, greg;             // Algorithm 3 on patch `pid`
    bool gpend;                     // Gregory node (path, level) still needs its (q, d): next step computes it
    uint32_t pid;
    RayG<NC> pr;                    // ray in the patch's frame, anchored at its entry into the patch box
    float d[NC];                    // Gregory displacement of the current node
    int level, rd_target;           // tree level; re-descent target level (-1: none)
    uint32_t path, trail;
    float c0, c1;                   // interval of the current node (distances from the anchored origin)
    int ctop, cvalid;               // sibling cache: pushes (slot = ctop % K) and valid entries
    uint32_t skip_path;             // subtree (skip_path, skip_level) not to enter again
    int skip_level;
    int pf;                         // BVH node whose data sits in the lane's prefetch slot (-1: none)
    int phase;                      // learned proposal: kPhase*
    uint32_t prop;                  // path bits (levels 0..5) of the proposed depth-3 cell
    float rc0, rc1;                 // root interval of the current pair
    float tau;                      // box extension of the current pair (local frames), else 0
    bool sleaf;                     // screen-space termination: the current node is a leaf
    uint32_t sleaf_trail;           // bit l: the pending sibling at level l+1 is a screen-space leaf
};

// Kernel modes: plain traversal, trace export (features + depth-3 cell of each pair's best leaf),
// traversal with the learned proposal, any hit (the ray ends at the first leaf it records), and plain
// traversal with screen-space termination (Sec. 3.3).
constexpr int kModePlain = 0, kModeExport = 1, kModeLearned = 2, kModeAnyHit = 3, kModeScreen = 4;
// Phases of a pair with the learned proposal: waiting for the network, descending straight to the
// proposed depth-3 cell, searching that cell's subtree, then the full search with the cell skipped.
constexpr int kPhaseNormal = 0, kPhasePropose = 1, kPhaseDirected = 2, kPhaseSubtree = 3;
constexpr int kProposalLevel = 6;   // depth 3 per axis

template <int NC>
CCS_DEV void begin_ray(Lane<NC> &s, const DevScene &sc, float ox, float oy, float oz, float dx, float dy, float dz,
                       float tmin, float tmax, uint32_t iter_cap, const Grp &G)
{
    s.best.t = tmax;
    s.best.pid = kMissId;
    s.best.cell = kMissId;
    s.sp = 0;
    s.iters = iter_cap;
    s.tmin = tmin;
    s.tmax = tmax;
    s.node = 0;
    s.n0 = tmin;
    s.in_pair = false;
    s.gpend = false;
    s.skip_level = -1;
    s.skip_path = 0xFFFFFFFFu;
    s.phase = kPhaseNormal;
    s.pf = -1;
    const bool bad = !(tmin <= tmax) || sc.n_nodes == 0 || isnan(ox) || isnan(oy) || isnan(oz) || isnan(dx) ||
                     isnan(dy) || isnan(dz);
    if (bad) {
        s.node = kDone;
        return;
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int c = comp<NC>(G, k);
        s.o[k] = pick(c, ox, oy, oz);
        s.dw[k] = pick(c, dx, dy, dz);
        s.r.org[k] = s.o[k];
        s.r.inv[k] = safe_inv(pick(c, dx, dy, dz));
    }
}

template <int NC>
CCS_DEV bool lane_done(const Lane<NC> &s)
{
    return !s.in_pair && s.node == kDone;
}

template <int NC>
CCS_DEV void pop_next(Lane<NC> &s, BvhStack &stk)
{
    while (s.sp > 0) {
        --s.sp;
        const int2 e = stk.e[s.sp];
        const float t0 = __int_as_float(e.y);
        if (t0 > s.best.t) continue;
        s.node = e.x;
        s.n0 = t0;
        return;
    }
    s.node = kDone;
}

CCS_DEV const float4 *rec_of(const DevScene &sc, uint32_t pid) { return sc.rec + (size_t)pid * kRecF4; }

// Begin Algorithm 3 on patch pid with root interval [c0, c1] (the patch box's slab from tmin; the ray's
// tmax is the best distance the search starts from).
template <int MODE, int NC>
CCS_DEV void start_pair(Lane<NC> &s, float (&g)[16 * NC], const DevScene &sc, uint32_t pid, float c0, float c1,
                        const Grp &G)
{
    const float4 *rec = rec_of(sc, pid);
    const float4 an = __ldg(rec + 15);
    s.in_pair = true;
    s.greg = an.w != 0.0f;
    s.pid = pid;
    s.te = c0;
    anchored_ray<NC>(rec, an, sc.local != 0, s.o, s.dw, s.r.inv, c0, G, s.pr);
    s.tau = 0.0f;
    if (sc.local) {   // box extension (Sec. 3.4): boxes below the root at least tau wide along every axis
        float o3[3];
        if constexpr (NC == 3) {
#pragma unroll
            for (int c = 0; c < 3; ++c) o3[c] = s.o[c] - pick(c, an.x, an.y, an.z);
        } else {   // gather the three components from the group
            const float oc = s.o[0] - pick(G.c, an.x, an.y, an.z);
#pragma unroll
            for (int c = 0; c < 3; ++c) o3[c] = __shfl_sync(G.mask, oc, G.l0 + c);
        }
        s.tau = pair_tau(o3);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) s.d[k] = 0.0f;
    s.level = 0;
    s.rd_target = -1;
    s.path = s.trail = 0u;
    s.c0 = 0.0f;   // the root interval from the anchored origin (te = c0)
    s.c1 = __fsub_rn(c1, c0);
    s.ctop = s.cvalid = 0;
    if (MODE == kModeScreen) {
        s.sleaf = false;
        s.sleaf_trail = 0u;
    }
    if (MODE != kModePlain && MODE != kModeScreen) {
        s.rc0 = s.c0;
        s.rc1 = s.c1;
    }
    if (MODE == kModeLearned) {
        s.phase = kPhasePropose;
        s.skip_level = -1;
    }
    s.gpend = s.greg;   // the Gregory root's (q, d) is computed by the next step (one code copy)
    if (!s.greg) load_grid<NC>(rec, G, g);
}

// Restart the current pair at its root (learned proposal), optionally skipping the proposed cell.
template <int NC>
CCS_DEV void restart_pair(Lane<NC> &s, float (&g)[16 * NC], const DevScene &sc, bool skip, const Grp &G)
{
    const float4 *rec = rec_of(sc, s.pid);
    s.level = 0;
    s.rd_target = -1;
    s.path = s.trail = 0u;
    s.c0 = s.rc0;
    s.c1 = s.rc1;
    s.ctop = s.cvalid = 0;
    s.phase = kPhaseNormal;
    s.skip_level = skip ? kProposalLevel : -1;
    s.skip_path = s.prop;
    s.gpend = s.greg;
    if (!s.greg) load_grid<NC>(rec, G, g);
}

// Export of a finished pair whose leaf is the ray's best so far: features + depth-3 cell label.
template <int NC>
CCS_DEV void export_pair(const Lane<NC> &s, const DevScene &sc, int L, const ModeCtx &mc)
{
    if constexpr (NC == 3) {
        if (s.best.pid != s.pid || L < 3) return;
        const uint32_t cu = s.best.cell & ((1u << L) - 1u), cv = s.best.cell >> L;
        const uint32_t label = (cv >> (L - 3)) * 8u + (cu >> (L - 3));
        const uint32_t slot = atomicAdd(mc.ex_count, 1u);
        if (slot >= mc.ex_capacity) return;
        float f[kFeat];
        pair_features(rec_of(sc, s.pid), s.pr.org[0], s.pr.org[1], s.pr.org[2], s.pr.inv[0], s.pr.inv[1],
                      s.pr.inv[2], s.rc0, s.rc1, f);
#pragma unroll
        for (int k = 0; k < kFeat; ++k) mc.ex_features[(size_t)slot * kFeat + k] = f[k];
        mc.ex_labels[slot] = (uint8_t)label;
    }
}

// Backtrack to the deepest pending sibling that can still hold a closer leaf, or end the pair.
template <bool STATS, int K, int MODE, int NC>
CCS_DEV void backtrack(Lane<NC> &s, float (&g)[16 * NC], BvhStack &stk, const DevScene &sc, int L,
                       const Scratch &scr, Counters &cnt, const ModeCtx &mc, const Grp &G)
{
    if (MODE == kModeAnyHit && s.best.pid != kMissId) {   // any leaf answers the query: the ray is done
        s.in_pair = false;
        s.node = kDone;
        s.sp = 0;
        return;
    }
    while (s.trail != 0u) {
        const int l = 31 - __clz(s.trail);
        const uint32_t bit = 1u << l;
        s.trail ^= bit;
        bool cached = false;
        int cslot = 0;
        if (K > 0 && !s.greg && s.cvalid > 0) {
            cslot = (s.ctop - 1) % (K > 0 ? K : 1);
            if (scr.tag[cslot] == l) {
                cached = true;
                --s.ctop;
                --s.cvalid;
            }
        }
        const float2 sb = scr.sib[l * scr.stride];
        if (__fadd_rn(s.te, sb.x) > s.best.t) {
            if (STATS) cnt.v[6]++;
            if (MODE == kModeScreen) s.sleaf_trail &= ~bit;
            continue;
        }
        s.path = (s.path & (bit - 1u)) | (~s.path & bit);
        s.c0 = sb.x;
        s.c1 = sb.y;
        if (STATS) cnt.v[4]++;
        if (MODE == kModeScreen) {
            s.sleaf = (s.sleaf_trail & bit) != 0u;
            s.sleaf_trail &= ~bit;
            if (s.sleaf) {   // a screen-space leaf: recorded by the next step, no points needed
                s.level = l + 1;
                s.gpend = false;
                return;
            }
        }
        if (s.greg) {
            s.level = l + 1;
            s.gpend = s.level < 2 * L;   // a leaf needs no bound
        } else if (cached) {
            s.level = l + 1;
            load_cached<NC>(scr.cache + cslot * 16 * NC, g);
        } else {
            if (STATS) cnt.v[5] += l + 1;
            load_grid<NC>(rec_of(sc, s.pid), G, g);
            s.level = 0;
            s.rd_target = l + 1;
        }
        return;
    }
    if (MODE == kModeLearned && s.phase == kPhaseSubtree) {   // proposed cell searched: now the rest
        restart_pair<NC>(s, g, sc, true, G);
        return;
    }
    if (MODE == kModeExport) export_pair<NC>(s, sc, L, mc);
    s.in_pair = false;
    pop_next<NC>(s, stk);
}

// Kinds of a unit of work, for the schedule counters.
constexpr int kStepNone = 0, kStepSplit = 1, kStepGregory = 2, kStepLeaf = 3, kStepBvh = 4, kStepCap = -1;

// One step of Algorithm 3 on the ray's current pair; returns its kind.
template <bool STATS, int K, int MODE, int NC>
CCS_DEV int pair_step(Lane<NC> &s, float (&g)[16 * NC], BvhStack &stk, const DevScene &sc, int L,
                       const Scratch &scr, Counters &cnt, const ModeCtx &mc, const Grp &G)
{
    if (MODE == kModeLearned && s.phase == kPhasePropose) return kStepNone;   // waits for the network round
    if (s.gpend) {   // Algorithm 2 with the crop of Algorithm 1 for the Gregory node (path, level), then
                     // its split in the same step: a Gregory ray advances one level per warp iteration
        float u0, u1, v0, v1;
        node_domain(s.path, s.level, L, u0, u1, v0, v1);
        gregory_node<NC>(rec_of(sc, s.pid), u0, u1, v0, v1, s.level, G, g, s.d);
        s.gpend = false;
    }
    const bool redesc = s.rd_target >= 0;
    const bool directed = MODE == kModeLearned && s.phase == kPhaseDirected;
    if (!redesc && (s.level == 2 * L || (MODE == kModeScreen && s.sleaf))) {
        uint32_t cu, cv;
        path_cells(s.path, L, cu, cv);   // lowest leaf cell of the node (path bits below its level are 0)
        const uint32_t cell = (cv << L) | cu;
        if (STATS) cnt.v[3]++;
        const float tk = __fadd_rn(s.te, s.c0);   // the leaf's key distance along the ray
        if (key_less(tk, s.pid, cell, s.best)) {
            s.best.t = tk;
            s.best.pid = s.pid;
            s.best.cell = cell;
            if (MODE == kModeScreen) s.best.lvl = s.level;
        }
        if (MODE == kModeScreen) s.sleaf = false;
        backtrack<STATS, K, MODE, NC>(s, g, stk, sc, L, scr, cnt, mc, G);
        return kStepLeaf;
    }
    const int force = redesc ? (int)((s.path >> s.level) & 1u) : directed ? (int)((s.prop >> s.level) & 1u) : -1;
    const int slot = (!redesc && !directed && K > 0 && !s.greg) ? (s.ctop % (K > 0 ? K : 1)) : -1;
    bool allowL = true, allowR = true;   // a subtree already searched by a directed descent is not entered
    if (!redesc && s.skip_level == s.level + 1 && ((s.skip_path ^ s.path) & ((1u << s.level) - 1u)) == 0u) {
        if ((s.skip_path >> s.level) & 1u) allowR = false; else allowL = false;
    }
    if (STATS && !redesc) cnt.v[s.greg ? 2 : 1]++;
    const StepOut o = split_step<K, NC>(g, s.pr, s.d, s.c0, s.c1, s.te, s.best.t, redesc || !s.greg, scr, slot,
                                        allowL, allowR, force, G, s.tau);
    if (redesc) {
        if (++s.level == s.rd_target) s.rd_target = -1;
        return kStepSplit;
    }
    if (directed) {   // straight descent to the proposed cell; abandon it if the ray misses a box on the way
        const bool up = force == 1;
        if (up ? o.hitR : o.hitL) {
            s.path |= (uint32_t)force << s.level;
            s.c0 = up ? o.r0 : o.l0;
            s.c1 = up ? o.r1 : o.l1;
            ++s.level;
            s.gpend = s.greg;
            if (s.level == kProposalLevel) s.phase = kPhaseSubtree;
        } else {
            restart_pair<NC>(s, g, sc, false, G);
        }
        return kStepSplit;
    }
    if (o.hitL || o.hitR) {
        const uint32_t bit = 1u << s.level;
        if (MODE == kModeScreen) {   // Sec. 3.3: a box under half a pixel at its entry distance is a leaf
            const float h = 0.5f * mc.spread;
            s.sleaf = (o.goR ? o.dR : o.dL) < h * __fadd_rn(s.te, o.goR ? o.r0 : o.l0);
            if (o.hitL && o.hitR && (o.goR ? o.dL : o.dR) < h * __fadd_rn(s.te, o.goR ? o.l0 : o.r0))
                s.sleaf_trail |= bit;
        }
        if (o.hitL && o.hitR) {
            s.trail |= bit;
            scr.sib[s.level * scr.stride] = o.goR ? make_float2(o.l0, o.l1) : make_float2(o.r0, o.r1);
            if (K > 0 && !s.greg) {
                scr.tag[slot] = s.level;
                ++s.ctop;
                s.cvalid = s.cvalid < K ? s.cvalid + 1 : K;
            }
        }
        s.path = o.goR ? (s.path | bit) : s.path;
        s.c0 = o.goR ? o.r0 : o.l0;
        s.c1 = o.goR ? o.r1 : o.l1;
        ++s.level;
        s.gpend = s.greg && s.level < 2 * L && !(MODE == kModeScreen && s.sleaf);
        return kStepSplit;
    }
    backtrack<STATS, K, MODE, NC>(s, g, stk, sc, L, scr, cnt, mc, G);
    return kStepSplit;
}

// Float4s of a BVH node that one lane reads: binary, the lane's component planes and the child word;
// 4-wide, the lane's lo and hi planes and the child words.
template <int BW, int NC>
__host__ __device__ constexpr int node_f4() { return BW == 2 ? NC + 1 : 2 * NC + 1; }

// Order a 4-wide node's hit children by entry distance (compare-exchange network; misses carry +inf).
CCS_DEV void cx4(float (&k)[4], int (&c)[4], int a, int b)
{
    const bool sw = k[b] < k[a];
    const float ka = k[a];
    const int ca = c[a];
    k[a] = sw ? k[b] : ka;
    c[a] = sw ? c[b] : ca;
    k[b] = sw ? ka : k[b];
    c[b] = sw ? ca : c[b];
}

// One BVH step: expand an internal node (nearest child first, the others pushed), or start the pair of
// a leaf.
template <bool STATS, int MODE, int NC, int BW>
CCS_DEV void bvh_step(Lane<NC> &s, float (&g)[16 * NC], BvhStack &stk, const DevScene &sc, Counters &cnt,
                      const Scratch &scr, const Grp &G)
{
    if (s.node == kDone) return;
    if (s.node < 0) {
        const uint32_t pid = (uint32_t)(~s.node);
        if (s.n0 <= s.best.t) {
            if (STATS) cnt.v[7]++;
            // the root interval: the slab of the patch box from tmin (tmax bounds the leaves' key distances,
            // through the best distance it starts from)
            float lo[NC], hi[NC], c0, c1;
            const float4 blo = __ldg(sc.leaf_box + 2 * (size_t)pid), bhi = __ldg(sc.leaf_box + 2 * (size_t)pid + 1);
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const int c = comp<NC>(G, k);
                lo[k] = pick(c, blo.x, blo.y, blo.z);
                hi[k] = pick(c, bhi.x, bhi.y, bhi.z);
            }
            slab<NC>(s.r, lo, hi, s.tmin, __int_as_float(0x7f800000), G, c0, c1);
            start_pair<MODE, NC>(s, g, sc, pid, c0, c1, G);
        } else {
            pop_next<NC>(s, stk);
        }
        return;
    }
    if (STATS) cnt.v[0]++;
    if constexpr (BW == 4) {
        float4 lo4[NC], hi4[NC];
        int c[4];
        if (s.pf == s.node) {   // fetched during the previous iteration
            cp_async_wait_all();
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                lo4[k] = scr.node[(2 * k) * scr.stride];
                hi4[k] = scr.node[(2 * k + 1) * scr.stride];
            }
            const float4 ch = scr.node[(2 * NC) * scr.stride];
            c[0] = __float_as_int(ch.x);
            c[1] = __float_as_int(ch.y);
            c[2] = __float_as_int(ch.z);
            c[3] = __float_as_int(ch.w);
        } else {
            const float4 *nd = sc.nodes + (size_t)s.node * kNode4F4;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                lo4[k] = __ldg(nd + 2 * comp<NC>(G, k));
                hi4[k] = __ldg(nd + 2 * comp<NC>(G, k) + 1);
            }
            const int4 ch = __ldg(reinterpret_cast<const int4 *>(nd + 6));
            c[0] = ch.x;
            c[1] = ch.y;
            c[2] = ch.z;
            c[3] = ch.w;
        }
        float key[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float lo[NC], hi[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                lo[k] = j == 0 ? lo4[k].x : j == 1 ? lo4[k].y : j == 2 ? lo4[k].z : lo4[k].w;
                hi[k] = j == 0 ? hi4[k].x : j == 1 ? hi4[k].y : j == 2 ? hi4[k].z : hi4[k].w;
            }
            float t0, t1;
            slab<NC>(s.r, lo, hi, s.tmin, s.tmax, G, t0, t1);
            const bool h = t0 <= t1 && t0 <= s.best.t && c[j] != kEmptyChild;
            key[j] = h ? t0 : __int_as_float(0x7f800000);
        }
        cx4(key, c, 0, 1);
        cx4(key, c, 2, 3);
        cx4(key, c, 0, 2);
        cx4(key, c, 1, 3);
        cx4(key, c, 1, 2);
        if (!(key[0] < __int_as_float(0x7f800000))) {
            pop_next<NC>(s, stk);
            return;
        }
#pragma unroll
        for (int j = 3; j >= 1; --j) {   // farthest first, so that the nearer ones are popped first
            if (key[j] < __int_as_float(0x7f800000) && s.sp < kBvhStack) {
                stk.e[s.sp] = make_int2(c[j], __float_as_int(key[j]));
                ++s.sp;
            }
        }
        s.node = c[0];
        s.n0 = key[0];
        return;
    }
    float4 q[NC];
    int c0, c1;
    if (s.pf == s.node) {   // fetched during the previous iteration
        cp_async_wait_all();
#pragma unroll
        for (int k = 0; k < NC; ++k) q[k] = scr.node[k * scr.stride];
        const float4 ch = scr.node[NC * scr.stride];
        c0 = __float_as_int(ch.x);
        c1 = __float_as_int(ch.y);
    } else {
        const float4 *nd = sc.nodes + (size_t)s.node * kNodeF4;
#pragma unroll
        for (int k = 0; k < NC; ++k) q[k] = __ldg(nd + comp<NC>(G, k));
        const int2 ch = __ldg(reinterpret_cast<const int2 *>(nd + 3));
        c0 = ch.x;
        c1 = ch.y;
    }
    float a0, a1, b0, b1;
    node_child_boxes<NC>(q, s.r, s.tmin, s.tmax, G, a0, a1, b0, b1);
    const bool ha = a0 <= a1 && a0 <= s.best.t && c0 != kEmptyChild;
    const bool hb = b0 <= b1 && b0 <= s.best.t && c1 != kEmptyChild;
    if (ha && hb) {
        const bool bfirst = b0 < a0;
        if (s.sp < kBvhStack) {
            stk.e[s.sp] = make_int2(bfirst ? c0 : c1, __float_as_int(bfirst ? a0 : b0));
            ++s.sp;
        }
        s.node = bfirst ? c1 : c0;
        s.n0 = bfirst ? b0 : a0;
    } else if (ha || hb) {
        s.node = ha ? c0 : c1;
        s.n0 = ha ? a0 : b0;
    } else {
        pop_next<NC>(s, stk);
    }
}

// The data of the next BVH node goes to the lane's shared-memory slot asynchronously (the lane's
// components and the child words), so its latency overlaps the other lanes' subdivision step of the
// next warp iteration.
template <int NC, int BW>
CCS_DEV void prefetch_node(Lane<NC> &s, const DevScene &sc, const Scratch &scr, const Grp &G)
{
    if (s.in_pair || s.node < 0 || s.node == s.pf) return;
    if constexpr (BW == 4) {
        const float4 *nd = sc.nodes + (size_t)s.node * kNode4F4;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            cp_async16(scr.node + (2 * k) * scr.stride, nd + 2 * comp<NC>(G, k));
            cp_async16(scr.node + (2 * k + 1) * scr.stride, nd + 2 * comp<NC>(G, k) + 1);
        }
        cp_async16(scr.node + (2 * NC) * scr.stride, nd + 6);
    } else {
        const float4 *nd = sc.nodes + (size_t)s.node * kNodeF4;
#pragma unroll
        for (int k = 0; k < NC; ++k) cp_async16(scr.node + k * scr.stride, nd + comp<NC>(G, k));
        cp_async16(scr.node + NC * scr.stride, nd + 3);
    }
    cp_async_commit();
    s.pf = s.node;
}

// One unit of work: a subdivision step, or up to `burst` BVH steps (cheap next to a subdivision step,
// so rays that traverse catch up while the others subdivide).  Returns the kind of the step (kStepCap
// on the iteration cap); bsteps receives the number of BVH steps taken.
template <bool STATS, int K, int MODE, int NC, int BW>
CCS_DEV int lane_step(Lane<NC> &s, float (&g)[16 * NC], BvhStack &stk, const DevScene &sc, int L,
                      const Scratch &scr, Counters &cnt, int burst, const ModeCtx &mc, const Grp &G, int &bsteps)
{
    int kind;
    bsteps = 0;
    if (s.in_pair) {
        if (s.iters == 0) return kStepCap;
        --s.iters;
        const bool bound = s.gpend;
        kind = pair_step<STATS, K, MODE, NC>(s, g, stk, sc, L, scr, cnt, mc, G);
        if (bound && kind == kStepSplit) kind = kStepGregory;   // a Gregory bound and its split
    } else {
        kind = kStepBvh;
        for (int k = 0; k < burst && !s.in_pair && s.node != kDone; ++k) {
            if (s.iters == 0) return kStepCap;
            --s.iters;
            ++bsteps;
            bvh_step<STATS, MODE, NC, BW>(s, g, stk, sc, cnt, scr, G);
        }
    }
    prefetch_node<NC, BW>(s, sc, scr, G);
    return kind;
}

}  // namespace ccs
