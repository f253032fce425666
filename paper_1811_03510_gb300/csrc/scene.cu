// Scene-store kernels: repacking of the caller's SoA control points into anchored 320-byte patch
// records (in local frames if the scene has them) with world leaf boxes, and bottom-up BVH refit.
#include "scene_dev.cuh"

namespace ccs {

__global__ void k_repack(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                         const uint8_t *__restrict__ types, uint32_t n, int local, float4 *__restrict__ rec,
                         float4 *__restrict__ leaf_box)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    repack_one(x, y, z, types, p, rec, leaf_box, local);
}

cudaError_t launch_repack(const float *x, const float *y, const float *z, const uint8_t *types, uint32_t n, int local,
                          float4 *rec, float4 *leaf_box, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_repack<<<(n + 127) / 128, 128, 0, s>>>(x, y, z, types, n, local, rec, leaf_box);
    return cudaGetLastError();
}

__global__ void k_refit(float4 *nodes, const int *__restrict__ leaf_parent, const float4 *__restrict__ leaf_box,
                        uint32_t *flags, uint32_t n, uint32_t width)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    refit_one(nodes, leaf_parent, leaf_box, flags, p, width);
}

cudaError_t launch_refit(float4 *nodes, const int *leaf_parent, const float4 *leaf_box, uint32_t *flags,
                         uint32_t n_patches, uint32_t n_nodes, uint32_t width, cudaStream_t s)
{
    if (n_patches == 0 || n_nodes == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t) * n_nodes, s);
    if (e != cudaSuccess) return e;
    k_refit<<<(n_patches + 127) / 128, 128, 0, s>>>(nodes, leaf_parent, leaf_box, flags, n_patches, width);
    return cudaGetLastError();
}

}  // namespace ccs
