// Device routines of the scene store shared by the single-scene and batched kernels.
#pragma once

#include "ccs_internal.h"

namespace ccs {

// Patch p of SoA points (20 slots per patch) -> 256-byte record anchored at its box centre
// (Sec. 3.4, anchoring), plus its leaf box (AABB of 16 or 20 points: convex hull, Sec. 3.1/3.2).
// Rows of the local frame of a patch (Sec. 3.4): z along the normal of the corner quad (the cross product
// of its diagonals p33 - p00 and p03 - p30), x along its u edge p30 - p00 made orthogonal to z, y = z x x;
// the world axes where that is degenerate.  Computed in FP64 (once per patch) and rounded: the points and
// the rays are both rotated by this rounded matrix, so they stay in one common frame.
__device__ __forceinline__ void local_frame(const float *const pl[3], float (&R)[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = i == j ? 1.0f : 0.0f;
    double a[3], b[3], e[3];
    for (int c = 0; c < 3; ++c) {
        a[c] = (double)pl[c][15] - (double)pl[c][0];
        b[c] = (double)pl[c][12] - (double)pl[c][3];
        e[c] = (double)pl[c][3] - (double)pl[c][0];
    }
    double z[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double nz = sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
    if (!(nz > 0.0)) return;
    for (int c = 0; c < 3; ++c) z[c] /= nz;
    const double ez = e[0] * z[0] + e[1] * z[1] + e[2] * z[2];
    double x[3] = {e[0] - ez * z[0], e[1] - ez * z[1], e[2] - ez * z[2]};
    const double nx = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    if (!(nx > 0.0)) return;
    for (int c = 0; c < 3; ++c) x[c] /= nx;
    const double y[3] = {z[1] * x[2] - z[2] * x[1], z[2] * x[0] - z[0] * x[2], z[0] * x[1] - z[1] * x[0]};
    for (int c = 0; c < 3; ++c) {
        R[0][c] = (float)x[c];
        R[1][c] = (float)y[c];
        R[2][c] = (float)z[c];
    }
}

__device__ __forceinline__ void repack_one(const float *__restrict__ x, const float *__restrict__ y,
                                           const float *__restrict__ z, const uint8_t *__restrict__ types, uint32_t p,
                                           float4 *__restrict__ rec, float4 *__restrict__ leaf_box, int local)
{
    const bool greg = types[p] != 0;
    const float *pl[3] = {x + (size_t)20 * p, y + (size_t)20 * p, z + (size_t)20 * p};
    float lo[3], hi[3], an[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float a = pl[c][0], b = pl[c][0];
        for (int k = 1; k < 16; ++k) { a = fminf(a, pl[c][k]); b = fmaxf(b, pl[c][k]); }
        if (greg)
            for (int k = 16; k < 20; ++k) { a = fminf(a, pl[c][k]); b = fmaxf(b, pl[c][k]); }
        lo[c] = a;
        hi[c] = b;
        an[c] = __fmul_rn(__fadd_rn(a, b), 0.5f);
    }
    float4 *r = rec + (size_t)p * kRecF4;
    float R[3][3];
    local_frame(pl, R);
    // component c of slot k: anchored, and rotated into the patch frame with local frames
    auto comp = [&](int c, int k) -> float {
        if (!local) return pl[c][k] - an[c];
        const float dx = pl[0][k] - an[0], dy = pl[1][k] - an[1], dz = pl[2][k] - an[2];
        return fmaf(R[c][0], dx, fmaf(R[c][1], dy, R[c][2] * dz));
    };
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int q = 0; q < 4; ++q)
            r[c * 4 + q] = make_float4(comp(c, 4 * q), comp(c, 4 * q + 1), comp(c, 4 * q + 2), comp(c, 4 * q + 3));
        if (greg)
            r[12 + c] = make_float4(comp(c, 16), comp(c, 17), comp(c, 18), comp(c, 19));
        else
            r[12 + c] = make_float4(comp(c, 5), comp(c, 6), comp(c, 9), comp(c, 10));
        r[16 + c] = local ? make_float4(R[c][0], R[c][1], R[c][2], 0.0f)
                          : make_float4(c == 0 ? 1.0f : 0.0f, c == 1 ? 1.0f : 0.0f, c == 2 ? 1.0f : 0.0f, 0.0f);
    }
    r[15] = make_float4(an[0], an[1], an[2], greg ? 1.0f : 0.0f);
    // the root box of a Bezier patch in its own frame: the AABB of the 16 stored grid components, which
    // holds every box of its subdivision (de Casteljau midpoints stay between their operands); lo in
    // the w of the frame rows, hi and 1 + |hi - lo|_1 in slot 19 (Gregory patches: unused, zero)
    float blo[3] = {0.0f, 0.0f, 0.0f}, bhi[3] = {0.0f, 0.0f, 0.0f};
    if (!greg) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float a = r[c * 4].x, b = a;
            for (int q = 0; q < 4; ++q) {
                const float4 v = r[c * 4 + q];
                a = fminf(fminf(a, v.x), fminf(fminf(v.y, v.z), v.w));
                b = fmaxf(fmaxf(b, v.x), fmaxf(fmaxf(v.y, v.z), v.w));
            }
            blo[c] = a;
            bhi[c] = b;
            r[16 + c].w = a;
        }
    }
    r[19] = make_float4(bhi[0], bhi[1], bhi[2],
                        greg ? 0.0f : 1.0f + ((bhi[0] - blo[0]) + (bhi[1] - blo[1])) + (bhi[2] - blo[2]));
    leaf_box[2 * (size_t)p] = make_float4(lo[0], lo[1], lo[2], 0.0f);
    leaf_box[2 * (size_t)p + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
}

__device__ __forceinline__ void write_child_box(float4 *nodes, int node, int slot, float4 lo, float4 hi)
{
    float *nd = reinterpret_cast<float *>(nodes + (size_t)node * kNodeF4);
    // float4 a = axis a: (c0.lo, c0.hi, c1.lo, c1.hi)
    nd[0 + 2 * slot] = lo.x;
    nd[1 + 2 * slot] = hi.x;
    nd[4 + 2 * slot] = lo.y;
    nd[5 + 2 * slot] = hi.y;
    nd[8 + 2 * slot] = lo.z;
    nd[9 + 2 * slot] = hi.z;
}

__device__ __forceinline__ void write_child_box4(float4 *nodes, int node, int slot, float4 lo, float4 hi)
{
    float *nd = reinterpret_cast<float *>(nodes + (size_t)node * kNode4F4);
    // float4 2a = lo of the four children along axis a, 2a + 1 = their hi
    nd[0 + slot] = lo.x;
    nd[4 + slot] = hi.x;
    nd[8 + slot] = lo.y;
    nd[12 + slot] = hi.y;
    nd[16 + slot] = lo.z;
    nd[20 + slot] = hi.z;
}

// Refit from leaf p: write its box into its parent's slot; the last thread to arrive at a node (per
// node arrival counter: two children in a binary node, the children present in a 4-wide one) takes the
// union of the children up to the node's parent.  Sibling boxes are read through L2 (.cg) after a
// fence; the climb is bounded by the tree depth.
__device__ __forceinline__ void refit_one(float4 *nodes, const int *__restrict__ leaf_parent,
                                          const float4 *__restrict__ leaf_box, uint32_t *flags, uint32_t p,
                                          uint32_t width)
{
    float4 lo = leaf_box[2 * (size_t)p], hi = leaf_box[2 * (size_t)p + 1];
    int link = leaf_parent[p];
    const int shift = width == 4 ? 2 : 1;
    for (int guard = 0; guard < 128; ++guard) {
        const int node = link >> shift, slot = link & ((1 << shift) - 1);
        int parent;
        if (width == 4) {
            write_child_box4(nodes, node, slot, lo, hi);
            __threadfence();
            const float4 *nd = nodes + (size_t)node * kNode4F4;
            const float4 meta = __ldcg(nd + 7);
            if (atomicAdd(flags + node, 1u) + 1u < (uint32_t)__float_as_int(meta.z)) return;
            __threadfence();
            const float4 lx = __ldcg(nd + 0), hx = __ldcg(nd + 1), ly = __ldcg(nd + 2), hy = __ldcg(nd + 3);
            const float4 lz = __ldcg(nd + 4), hz = __ldcg(nd + 5);
            // empty slots hold lo = +max, hi = -max and drop out of the union
            lo = make_float4(fminf(fminf(lx.x, lx.y), fminf(lx.z, lx.w)), fminf(fminf(ly.x, ly.y), fminf(ly.z, ly.w)),
                             fminf(fminf(lz.x, lz.y), fminf(lz.z, lz.w)), 0.0f);
            hi = make_float4(fmaxf(fmaxf(hx.x, hx.y), fmaxf(hx.z, hx.w)), fmaxf(fmaxf(hy.x, hy.y), fmaxf(hy.z, hy.w)),
                             fmaxf(fmaxf(hz.x, hz.y), fmaxf(hz.z, hz.w)), 0.0f);
            parent = __float_as_int(meta.x);
            link = (parent << 2) | __float_as_int(meta.y);
        } else {
            write_child_box(nodes, node, slot, lo, hi);
            __threadfence();
            if (atomicAdd(flags + node, 1u) == 0u) return;
            __threadfence();
            const float4 *nd = nodes + (size_t)node * kNodeF4;
            const float4 a = __ldcg(nd + 0), b = __ldcg(nd + 1), c = __ldcg(nd + 2), d = __ldcg(nd + 3);
            lo = make_float4(fminf(a.x, a.z), fminf(b.x, b.z), fminf(c.x, c.z), 0.0f);
            hi = make_float4(fmaxf(a.y, a.w), fmaxf(b.y, b.w), fmaxf(c.y, c.w), 0.0f);
            parent = __float_as_int(d.z);
            link = (parent << 1) | __float_as_int(d.w);
        }
        if (parent < 0) return;
    }
}

}  // namespace ccs
