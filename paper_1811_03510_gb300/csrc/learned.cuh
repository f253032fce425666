// Learned sub-domain proposal: pair features and the warp-level BF16 tensor-core MLP
// (24 -> 64 -> 64 -> 64, ReLU, argmax over the 64 depth-3 cells of the (u,v) domain).
// The network only reorders the search: it proposes the cell searched first, which tightens the best
// distance early; the full traversal still runs, so hits equal those of the plain kernel.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "ccs_internal.h"

namespace ccs {

constexpr int kFeat = 24;
constexpr int kHid = 64;
constexpr int kCells = 64;
constexpr int kParams = 9920;        // W1 [64,24], b1, W2 [64,64], b2, W3 [64,64], b3
constexpr int kW1Stride = 40;        // bf16 elements per row of W1 in shared memory (K padded to 32, +8)
constexpr int kW2Stride = 72;        // rows of W2, W3 and of the hidden tiles (64, +8): no bank conflicts
constexpr int kXStride = 40;

// BF16 weights and FP32 biases as kept in shared memory (and as one blob in global memory).
struct MlpWeights {
    __nv_bfloat16 w1[kHid * kW1Stride];
    __nv_bfloat16 w2[kHid * kW2Stride];
    __nv_bfloat16 w3[kHid * kW2Stride];
    float bias[3 * kHid];
};

// Per-warp tiles for one inference round of 16 rows (32 rows in two rounds).
struct MlpWarpTiles {
    __nv_bfloat16 x[32 * kXStride];
    __nv_bfloat16 h1[16 * kW2Stride];
    __nv_bfloat16 h2[16 * kW2Stride];
    uint8_t cell[32];
    float pmax[32];
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void st_bf16x2(__nv_bfloat16 *p, float a, float b)
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}

// A fragment (16 x 16, row major) of rows [0,16) and columns [k0, k0+16) of a tile with `stride`.
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const __nv_bfloat16 *tile, int stride, int k0, int g, int t)
{
    a[0] = ld_u32(tile + g * stride + k0 + 2 * t);
    a[1] = ld_u32(tile + (g + 8) * stride + k0 + 2 * t);
    a[2] = ld_u32(tile + g * stride + k0 + 8 + 2 * t);
    a[3] = ld_u32(tile + (g + 8) * stride + k0 + 8 + 2 * t);
}

// One dense layer over 16 rows: out = relu(in . W^T + b) stored as BF16 (STORE) or kept in acc.
template <int KSTEPS, bool STORE>
__device__ __forceinline__ void mlp_layer(const __nv_bfloat16 *in, int in_stride, const __nv_bfloat16 *W,
                                          int w_stride, const float *bias, __nv_bfloat16 *out, float (&acc)[8][4],
                                          int g, int t)
{
    uint32_t a[KSTEPS][4];
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks) load_a(a[ks], in, in_stride, 16 * ks, g, t);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float bl = bias[8 * j + 2 * t], bh = bias[8 * j + 2 * t + 1];
        acc[j][0] = bl; acc[j][1] = bh; acc[j][2] = bl; acc[j][3] = bh;
        const __nv_bfloat16 *wrow = W + (8 * j + g) * w_stride;
#pragma unroll
        for (int ks = 0; ks < KSTEPS; ++ks)
            mma_bf16_16816(acc[j], a[ks], ld_u32(wrow + 16 * ks + 2 * t), ld_u32(wrow + 16 * ks + 8 + 2 * t));
        if (STORE) {
            st_bf16x2(out + g * kW2Stride + 8 * j + 2 * t, fmaxf(acc[j][0], 0.0f), fmaxf(acc[j][1], 0.0f));
            st_bf16x2(out + (g + 8) * kW2Stride + 8 * j + 2 * t, fmaxf(acc[j][2], 0.0f), fmaxf(acc[j][3], 0.0f));
        }
    }
}

// Forward pass of rows [16*r, 16*r+16) of the warp's x tile; writes argmax cell and max softmax
// probability per row into the tiles (ties: lowest cell), and optionally the logits (row stride 64).
__device__ __forceinline__ void mlp_round(const MlpWeights &W, MlpWarpTiles &T, int r, int lane, float *logits_out,
                                          uint32_t rows_valid)
{
    const int g = lane >> 2, t = lane & 3;
    float acc[8][4];
    mlp_layer<2, true>(T.x + 16 * r * kXStride, kXStride, W.w1, kW1Stride, W.bias, T.h1, acc, g, t);
    __syncwarp();
    mlp_layer<4, true>(T.h1, kW2Stride, W.w2, kW2Stride, W.bias + kHid, T.h2, acc, g, t);
    __syncwarp();
    mlp_layer<4, false>(T.h2, kW2Stride, W.w3, kW2Stride, W.bias + 2 * kHid, nullptr, acc, g, t);
    // argmax and softmax normaliser of rows g and g + 8 over the quad's 64 columns
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float best = -__int_as_float(0x7f800000);
        int bidx = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float v = acc[j][2 * h + e];
                const int c = 8 * j + 2 * t + e;
                if (v > best) { best = v; bidx = c; }
            }
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
        }
        float sum = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) sum += __expf(acc[j][2 * h] - best) + __expf(acc[j][2 * h + 1] - best);
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        const int row = 16 * r + g + 8 * h;
        if (t == 0) {
            T.cell[row] = (uint8_t)bidx;
            T.pmax[row] = 1.0f / sum;
        }
        if (logits_out && ((rows_valid >> row) & 1u)) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                logits_out[row * kCells + 8 * j + 2 * t] = acc[j][2 * h];
                logits_out[row * kCells + 8 * j + 2 * t + 1] = acc[j][2 * h + 1];
            }
        }
    }
    __syncwarp();
}

// Copy the weight blob into shared memory (whole block).
__device__ __forceinline__ void load_weights(MlpWeights &dst, const MlpWeights *__restrict__ src)
{
    const int n4 = (int)(sizeof(MlpWeights) / 16);
    const float4 *s = reinterpret_cast<const float4 *>(src);
    float4 *d = reinterpret_cast<float4 *>(&dst);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) d[i] = __ldg(s + i);
}

// The 24 features of a (ray, patch) pair at the start of Algorithm 3, in the frame of the patch record
// (anchored; rotated with local frames) scaled by the size S of its corner points: entry point of the
// ray into the patch box (3), unit direction (3), the 4 corners (12), unit normal of the corner quad (3),
// length of the ray inside the box (1, <= 4), cosine of direction and normal (1), Gregory flag (1).
// (lx, ly, lz) is the ray origin and (ix, iy, iz) its inverse direction in that frame.
__device__ __forceinline__ void pair_features(const float4 *__restrict__ rec, float lx, float ly, float lz, float ix,
                                              float iy, float iz, float t0, float t1, float (&f)[kFeat])
{
    const float4 X0 = __ldg(rec + 0), X3 = __ldg(rec + 3), Y0 = __ldg(rec + 4), Y3 = __ldg(rec + 7);
    const float4 Z0 = __ldg(rec + 8), Z3 = __ldg(rec + 11), an = __ldg(rec + 15);
    // corners (anchored): slot 0 = (u,v) (0,0), 3 = (1,0), 12 = (0,1), 15 = (1,1)
    const float cx[4] = {X0.x, X0.w, X3.x, X3.w}, cy[4] = {Y0.x, Y0.w, Y3.x, Y3.w}, cz[4] = {Z0.x, Z0.w, Z3.x, Z3.w};
    float S = 1e-12f;
#pragma unroll
    for (int k = 0; k < 4; ++k) S = fmaxf(S, sqrtf(cx[k] * cx[k] + cy[k] * cy[k] + cz[k] * cz[k]));
    const float inv = 1.0f / S;
    float dx = 1.0f / ix, dy = 1.0f / iy, dz = 1.0f / iz;
    const float dn = rsqrtf(fmaxf(dx * dx + dy * dy + dz * dz, 1e-30f));
    dx *= dn; dy *= dn; dz *= dn;
    const float te = t0 / dn;                                      // entry along the unit direction
    f[0] = (lx + te * dx) * inv;
    f[1] = (ly + te * dy) * inv;
    f[2] = (lz + te * dz) * inv;
    f[3] = dx; f[4] = dy; f[5] = dz;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        f[6 + 3 * k] = cx[k] * inv;
        f[7 + 3 * k] = cy[k] * inv;
        f[8 + 3 * k] = cz[k] * inv;
    }
    const float ax = cx[3] - cx[0], ay = cy[3] - cy[0], az = cz[3] - cz[0];
    const float bx = cx[2] - cx[1], by = cy[2] - cy[1], bz = cz[2] - cz[1];
    float nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
    const float nn = rsqrtf(fmaxf(nx * nx + ny * ny + nz * nz, 1e-30f));
    nx *= nn; ny *= nn; nz *= nn;
    f[18] = nx; f[19] = ny; f[20] = nz;
    f[21] = fminf((t1 - t0) / dn * inv, 4.0f);
    f[22] = dx * nx + dy * ny + dz * nz;
    f[23] = an.w != 0.0f ? 1.0f : 0.0f;
}

// Path bits (levels 0..5) of depth-3 cell `cell` = v3 * 8 + u3: u bits at even levels, v bits at odd,
// most significant first.
__device__ __forceinline__ uint32_t cell3_path(uint32_t cell)
{
    const uint32_t u3 = cell & 7u, v3 = cell >> 3;
    uint32_t p = 0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        p |= ((u3 >> (2 - m)) & 1u) << (2 * m);
        p |= ((v3 >> (2 - m)) & 1u) << (2 * m + 1);
    }
    return p;
}

}  // namespace ccs
