// Secondary-ray generation for a wavefront tracer (test input of the diffuse, mirror and shadow
// workloads, not part of the intersection path): rays leaving the surface point of each hit.
#include "ccs_internal.h"

namespace ccs {

// PCG32 (O'Neill 2014, pcg32_srandom_r / pcg32_random_r), one stream per ray.
struct Pcg32 {
    unsigned long long state, inc;
    __device__ uint32_t next()
    {
        const unsigned long long old = state;
        state = old * 6364136223846793005ull + inc;
        const uint32_t xs = (uint32_t)(((old >> 18u) ^ old) >> 27u);
        const uint32_t rot = (uint32_t)(old >> 59u);
        return (xs >> rot) | (xs << ((32u - rot) & 31u));
    }
    __device__ Pcg32(unsigned long long initstate, unsigned long long initseq)
    {
        state = 0ull;
        inc = (initseq << 1u) | 1ull;
        next();
        state += initstate;
        next();
    }
};

__device__ __forceinline__ float unit24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// Surface point and partial derivatives of the (Gregory-reduced) patch record at (u, v), world space
// (records of a scene with local frames are rotated back with the frame rows [16..18]).
__device__ void patch_frame(const float4 *__restrict__ rec, float u, float v, float f[3], float fu[3], float fv[3],
                            bool local)
{
    const float4 an = rec[15];
    const bool greg = an.w != 0.0f;
    const int inner[4] = {5, 6, 9, 10};
    float h[4];
    {
        const float nu[4] = {u, 1.0f - u, u, 1.0f - u};
        const float dv[4] = {v, v, 1.0f - v, 1.0f - v};
        for (int k = 0; k < 4; ++k) {
            const float s = nu[k] + dv[k];
            h[k] = s == 0.0f ? 0.5f : nu[k] / s;
        }
    }
    const float s = 1.0f - u, t = 1.0f - v;
    const float Bu[4] = {s * s * s, 3 * u * s * s, 3 * u * u * s, u * u * u};
    const float Du[4] = {-3 * s * s, 3 * s * (s - 2 * u), 3 * u * (2 * s - u), 3 * u * u};
    const float Bv[4] = {t * t * t, 3 * v * t * t, 3 * v * v * t, v * v * v};
    const float Dv[4] = {-3 * t * t, 3 * t * (t - 2 * v), 3 * v * (2 * t - v), 3 * v * v};
    const float anc[3] = {an.x, an.y, an.z};
    for (int c = 0; c < 3; ++c) {
        float p[16];
        for (int q = 0; q < 4; ++q) {
            const float4 w = rec[c * 4 + q];
            p[4 * q] = w.x; p[4 * q + 1] = w.y; p[4 * q + 2] = w.z; p[4 * q + 3] = w.w;
        }
        if (greg) {
            const float4 w = rec[12 + c];
            const float pv[4] = {w.x, w.y, w.z, w.w};
            for (int k = 0; k < 4; ++k) p[inner[k]] = pv[k] + h[k] * (p[inner[k]] - pv[k]);
        }
        float a = 0, b = 0, e = 0;
        for (int j = 0; j < 4; ++j)
            for (int i = 0; i < 4; ++i) {
                const float pij = p[4 * j + i];
                a += Bu[i] * Bv[j] * pij;
                b += Du[i] * Bv[j] * pij;
                e += Bu[i] * Dv[j] * pij;
            }
        f[c] = local ? a : a + anc[c];
        fu[c] = b;
        fv[c] = e;
    }
    if (local) {   // world = R^T local + anchor
        const float4 R0 = rec[16], R1 = rec[17], R2 = rec[18];
        const float Rm[3][3] = {{R0.x, R0.y, R0.z}, {R1.x, R1.y, R1.z}, {R2.x, R2.y, R2.z}};
        float wf[3], wu[3], wv[3];
        for (int c = 0; c < 3; ++c) {
            wf[c] = Rm[0][c] * f[0] + Rm[1][c] * f[1] + Rm[2][c] * f[2] + anc[c];
            wu[c] = Rm[0][c] * fu[0] + Rm[1][c] * fu[1] + Rm[2][c] * fu[2];
            wv[c] = Rm[0][c] * fv[0] + Rm[1][c] * fv[1] + Rm[2][c] * fv[2];
        }
        for (int c = 0; c < 3; ++c) {
            f[c] = wf[c];
            fu[c] = wu[c];
            fv[c] = wv[c];
        }
    }
}

// kind 0: cosine-weighted diffuse, 1: mirror reflection, 2: shadow ray toward the point light
__global__ void k_gen_diffuse(const float4 *__restrict__ rec, const float4 *__restrict__ leaf_box, uint32_t n_patches,
                              DevRays in, DevHits hits, uint32_t n, unsigned long long seed, int L, float offset_abs,
                              float *out_o, float *out_d, float *out_tmin, float *out_tmax, int kind, float3 light,
                              int local)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t pid = hits.pid[i];
    if (pid >= n_patches) {   // miss (or an id outside the scene): inactive slot, empty interval
        for (int c = 0; c < 3; ++c) { out_o[c * (size_t)n + i] = 0.0f; out_d[c * (size_t)n + i] = 0.0f; }
        out_d[2 * (size_t)n + i] = 1.0f;
        out_tmin[i] = 1.0f;
        out_tmax[i] = 0.0f;
        return;
    }
    const float4 *r = rec + (size_t)pid * kRecF4;
    float f[3], fu[3], fv[3];
    patch_frame(r, hits.u[i], hits.v[i], f, fu, fv, local != 0);
    float nx = fu[1] * fv[2] - fu[2] * fv[1], ny = fu[2] * fv[0] - fu[0] * fv[2], nz = fu[0] * fv[1] - fu[1] * fv[0];
    const float inv = rsqrtf(fmaxf(nx * nx + ny * ny + nz * nz, 1e-30f));
    nx *= inv; ny *= inv; nz *= inv;
    if (nx * in.dx[i] + ny * in.dy[i] + nz * in.dz[i] > 0.0f) { nx = -nx; ny = -ny; nz = -nz; }
    // offset: absolute term plus twice the L1 size of a leaf cell of the patch's box (Sec. 3.3)
    const float4 lo = leaf_box[2 * (size_t)pid], hi = leaf_box[2 * (size_t)pid + 1];
    const float l1 = (hi.x - lo.x) + (hi.y - lo.y) + (hi.z - lo.z);
    const float off = offset_abs + 2.0f * l1 * __int_as_float((127 - L) << 23);
    const float ox = f[0] + off * nx, oy = f[1] + off * ny, oz = f[2] + off * nz;
    out_o[i] = ox;
    out_o[(size_t)n + i] = oy;
    out_o[2 * (size_t)n + i] = oz;
    if (kind == 2) {   // toward the light; none when the light is behind the surface (self-shadowed)
        const float lx = light.x - ox, ly = light.y - oy, lz = light.z - oz;
        const float dist = sqrtf(lx * lx + ly * ly + lz * lz);
        const bool lit = dist > 0.0f && lx * nx + ly * ny + lz * nz > 0.0f;
        const float id = lit ? 1.0f / dist : 0.0f;
        out_d[i] = lit ? lx * id : 0.0f;
        out_d[(size_t)n + i] = lit ? ly * id : 0.0f;
        out_d[2 * (size_t)n + i] = lit ? lz * id : 1.0f;
        out_tmin[i] = lit ? 0.0f : 1.0f;
        out_tmax[i] = lit ? dist : 0.0f;
        return;
    }
    if (kind == 1) {   // reflection of the incoming direction about the normal
        const float ix = in.dx[i], iy = in.dy[i], iz = in.dz[i];
        const float k = 2.0f * (ix * nx + iy * ny + iz * nz);
        out_d[i] = ix - k * nx;
        out_d[(size_t)n + i] = iy - k * ny;
        out_d[2 * (size_t)n + i] = iz - k * nz;
    } else {
        Pcg32 rng(seed, i);
        const float u1 = unit24(rng.next()), u2 = unit24(rng.next());
        const float rr = sqrtf(u1), phi = 6.283185307179586f * u2;
        const float lx = rr * cosf(phi), ly = rr * sinf(phi), lz = sqrtf(fmaxf(0.0f, 1.0f - u1));
        // orthonormal basis around n (Duff et al. 2017)
        const float sg = copysignf(1.0f, nz);
        const float a = -1.0f / (sg + nz);
        const float b = nx * ny * a;
        const float b1x = 1.0f + sg * nx * nx * a, b1y = sg * b, b1z = -sg * nx;
        const float b2x = b, b2y = sg + ny * ny * a, b2z = -ny;
        out_d[i] = lx * b1x + ly * b2x + lz * nx;
        out_d[(size_t)n + i] = lx * b1y + ly * b2y + lz * ny;
        out_d[2 * (size_t)n + i] = lx * b1z + ly * b2z + lz * nz;
    }
    out_tmin[i] = 0.0f;
    out_tmax[i] = __int_as_float(0x7f800000);
}

cudaError_t launch_gen_diffuse(const float4 *rec, const float4 *leaf_box, uint32_t n_patches, const DevRays &in,
                               const DevHits &hits, uint32_t n, unsigned long long seed, int L, float offset_abs, float *o, float *d,
                               float *tmin, float *tmax, int kind, const float *light, int local, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const float3 lp = light ? make_float3(light[0], light[1], light[2]) : make_float3(0.0f, 0.0f, 0.0f);
    k_gen_diffuse<<<(n + 255) / 256, 256, 0, s>>>(rec, leaf_box, n_patches, in, hits, n, seed, L, offset_abs, o, d, tmin, tmax,
                                                   kind, lp, local);
    return cudaGetLastError();
}

}  // namespace ccs
