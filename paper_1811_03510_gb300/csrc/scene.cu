// Scene-store kernels: repacking of the caller's SoA control points into anchored 256-byte patch
// records with leaf boxes, and bottom-up BVH refit.
#include "ccs_internal.h"

namespace ccs {

__global__ void k_repack(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                         const uint8_t *__restrict__ types, uint32_t n, float4 *__restrict__ rec,
                         float4 *__restrict__ leaf_box)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
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
        an[c] = __fmul_rn(__fadd_rn(a, b), 0.5f);   // anchor at the box centre (Sec. 3.4)
    }
    float4 *r = rec + (size_t)p * kRecF4;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int q = 0; q < 4; ++q)
            r[c * 4 + q] = make_float4(pl[c][4 * q] - an[c], pl[c][4 * q + 1] - an[c], pl[c][4 * q + 2] - an[c],
                                       pl[c][4 * q + 3] - an[c]);
        if (greg)
            r[12 + c] = make_float4(pl[c][16] - an[c], pl[c][17] - an[c], pl[c][18] - an[c], pl[c][19] - an[c]);
        else
            r[12 + c] = make_float4(pl[c][5] - an[c], pl[c][6] - an[c], pl[c][9] - an[c], pl[c][10] - an[c]);
    }
    r[15] = make_float4(an[0], an[1], an[2], greg ? 1.0f : 0.0f);
    leaf_box[2 * (size_t)p] = make_float4(lo[0], lo[1], lo[2], 0.0f);
    leaf_box[2 * (size_t)p + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
}

cudaError_t launch_repack(const float *x, const float *y, const float *z, const uint8_t *types, uint32_t n,
                          float4 *rec, float4 *leaf_box, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_repack<<<(n + 127) / 128, 128, 0, s>>>(x, y, z, types, n, rec, leaf_box);
    return cudaGetLastError();
}

__device__ __forceinline__ void write_child_box(float4 *nodes, int node, int slot, float4 lo, float4 hi)
{
    float4 *nd = nodes + (size_t)node * kNodeF4;
    // slot 0: [0].x=lo.x [0].y=hi.x [0].z=lo.y [0].w=hi.y [2].x=lo.z [2].y=hi.z ; slot 1 uses [1] and [2].zw
    float *xy = reinterpret_cast<float *>(nd + slot);
    xy[0] = lo.x;
    xy[1] = hi.x;
    xy[2] = lo.y;
    xy[3] = hi.y;
    float *zz = reinterpret_cast<float *>(nd + 2) + 2 * slot;
    zz[0] = lo.z;
    zz[1] = hi.z;
}

// One thread per patch: write its box into the parent's slot, then the second thread to reach a node
// takes the union of both children up to the node's parent.  Reads of siblings go through L2 (.cg).
__global__ void k_refit(float4 *nodes, const int *__restrict__ leaf_parent, const float4 *__restrict__ leaf_box,
                        uint32_t *flags, uint32_t n)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float4 lo = leaf_box[2 * (size_t)p], hi = leaf_box[2 * (size_t)p + 1];
    int link = leaf_parent[p];
    for (int guard = 0; guard < 128; ++guard) {
        const int node = link >> 1, slot = link & 1;
        write_child_box(nodes, node, slot, lo, hi);
        __threadfence();
        if (atomicAdd(flags + node, 1u) == 0u) return;
        __threadfence();
        const float4 *nd = nodes + (size_t)node * kNodeF4;
        const float4 a = __ldcg(nd + 0), b = __ldcg(nd + 1), c = __ldcg(nd + 2), d = __ldcg(nd + 3);
        lo = make_float4(fminf(a.x, b.x), fminf(a.z, b.z), fminf(c.x, c.z), 0.0f);
        hi = make_float4(fmaxf(a.y, b.y), fmaxf(a.w, b.w), fmaxf(c.y, c.w), 0.0f);
        const int parent = __float_as_int(d.z);
        if (parent < 0) return;
        link = (parent << 1) | __float_as_int(d.w);
    }
}

cudaError_t launch_refit(float4 *nodes, const int *leaf_parent, const float4 *leaf_box, uint32_t *flags,
                         uint32_t n_patches, uint32_t n_nodes, cudaStream_t s)
{
    if (n_patches == 0 || n_nodes == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * n_nodes, s);
    if (e != cudaSuccess) return e;
    k_refit<<<(n_patches + 127) / 128, 128, 0, s>>>(nodes, leaf_parent, leaf_box, flags, n_patches);
    return cudaGetLastError();
}

}  // namespace ccs
