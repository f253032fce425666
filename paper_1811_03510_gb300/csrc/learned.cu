// Learned sub-domain proposal: parameters (FP32 masters + Adam state + BF16 copy), training kernels
// (per-sample forward and backward, weight-gradient reduction, Adam), and the tensor-core inference
// kernel.  Softmax cross-entropy over the 64 depth-3 cells; mean over the mini-batch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "learned.cuh"

namespace ccs {

// Parameter offsets in the 9920-vector.
constexpr int kOffW1 = 0, kOffB1 = 1536, kOffW2 = 1600, kOffB2 = 5696, kOffW3 = 5760, kOffB3 = 9856;

// One thread per sample: forward, softmax-CE, backward to the pre-activations.  Keeps x, h1, h2 and the
// gradients dz1, dz2, dz3 (already divided by the batch size) for the weight-gradient kernel.
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(const float *__restrict__ params, const float *__restrict__ X,
                                                     const uint8_t *__restrict__ labels, uint32_t B,
                                                     float *__restrict__ h1o, float *__restrict__ h2o,
                                                     float *__restrict__ dz1o, float *__restrict__ dz2o,
                                                     float *__restrict__ dz3o, float *loss)
{
    __shared__ float w[kParams];
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = params[i];
    __syncthreads();
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float x[kFeat], z1[kHid], z2[kHid], z3[kHid];
    for (int i = 0; i < kFeat; ++i) x[i] = X[(size_t)b * kFeat + i];
    for (int j = 0; j < kHid; ++j) {
        float a = w[kOffB1 + j];
        for (int i = 0; i < kFeat; ++i) a = fmaf(w[kOffW1 + j * kFeat + i], x[i], a);
        z1[j] = a;
    }
    for (int j = 0; j < kHid; ++j) {
        float a = w[kOffB2 + j];
        for (int i = 0; i < kHid; ++i) a = fmaf(w[kOffW2 + j * kHid + i], fmaxf(z1[i], 0.0f), a);
        z2[j] = a;
    }
    float mx = -INFINITY;
    for (int j = 0; j < kCells; ++j) {
        float a = w[kOffB3 + j];
        for (int i = 0; i < kHid; ++i) a = fmaf(w[kOffW3 + j * kHid + i], fmaxf(z2[i], 0.0f), a);
        z3[j] = a;
        mx = fmaxf(mx, a);
    }
    float sum = 0.0f;
    for (int j = 0; j < kCells; ++j) sum += expf(z3[j] - mx);
    const int y = labels[b];
    atomicAdd(loss, (logf(sum) + mx - z3[y]) / (float)B);
    const float invB = 1.0f / (float)B;
    for (int j = 0; j < kCells; ++j) {
        z3[j] = (expf(z3[j] - mx) / sum - (j == y ? 1.0f : 0.0f)) * invB;   // dz3
        dz3o[(size_t)b * kHid + j] = z3[j];
    }
    for (int i = 0; i < kHid; ++i) {
        h2o[(size_t)b * kHid + i] = fmaxf(z2[i], 0.0f);
        h1o[(size_t)b * kHid + i] = fmaxf(z1[i], 0.0f);
    }
    for (int i = 0; i < kHid; ++i) {   // dz2 = (W3^T dz3) * [z2 > 0]
        float a = 0.0f;
        for (int j = 0; j < kCells; ++j) a = fmaf(w[kOffW3 + j * kHid + i], z3[j], a);
        z2[i] = z2[i] > 0.0f ? a : 0.0f;
        dz2o[(size_t)b * kHid + i] = z2[i];
    }
    for (int i = 0; i < kHid; ++i) {   // dz1 = (W2^T dz2) * [z1 > 0]
        float a = 0.0f;
        for (int j = 0; j < kHid; ++j) a = fmaf(w[kOffW2 + j * kHid + i], z2[j], a);
        dz1o[(size_t)b * kHid + i] = z1[i] > 0.0f ? a : 0.0f;
    }
}

// One thread per parameter and batch chunk: grad += sum over the chunk of dz[b][j] * input[b][i].
__global__ void k_mlp_wgrad(const float *__restrict__ X, const float *__restrict__ h1, const float *__restrict__ h2,
                            const float *__restrict__ dz1, const float *__restrict__ dz2,
                            const float *__restrict__ dz3, uint32_t B, uint32_t chunk, float *grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const uint32_t b0 = blockIdx.y * chunk, b1 = min(B, b0 + chunk);
    const float *dz, *in;
    int j, i, in_dim;
    bool bias = false;
    if (p < kOffB1) { j = p / kFeat; i = p % kFeat; dz = dz1; in = X; in_dim = kFeat; }
    else if (p < kOffW2) { j = p - kOffB1; i = 0; dz = dz1; in = X; in_dim = kFeat; bias = true; }
    else if (p < kOffB2) { j = (p - kOffW2) / kHid; i = (p - kOffW2) % kHid; dz = dz2; in = h1; in_dim = kHid; }
    else if (p < kOffW3) { j = p - kOffB2; i = 0; dz = dz2; in = h1; in_dim = kHid; bias = true; }
    else if (p < kOffB3) { j = (p - kOffW3) / kHid; i = (p - kOffW3) % kHid; dz = dz3; in = h2; in_dim = kHid; }
    else { j = p - kOffB3; i = 0; dz = dz3; in = h2; in_dim = kHid; bias = true; }
    float a = 0.0f;
    for (uint32_t b = b0; b < b1; ++b) {
        const float d = dz[(size_t)b * kHid + j];
        a = bias ? a + d : fmaf(d, in[(size_t)b * in_dim + i], a);
    }
    atomicAdd(grad + p, a);
}

// Adam on the FP32 masters, then the BF16 copy used by inference.
__global__ void k_adam(float *params, float *m, float *v, const float *grad, float lr, float b1c, float b2c)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float g = grad[p];
    const float mm = 0.9f * m[p] + 0.1f * g;
    const float vv = 0.999f * v[p] + 0.001f * g * g;
    m[p] = mm;
    v[p] = vv;
    params[p] -= lr * (mm / b1c) / (sqrtf(vv / b2c) + 1e-8f);
}

__global__ void k_publish_bf16(const float *__restrict__ params, MlpWeights *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;   // one thread per output row
    if (n >= kHid) return;
    for (int k = 0; k < kW1Stride; ++k)
        out->w1[n * kW1Stride + k] = __float2bfloat16_rn(k < kFeat ? params[kOffW1 + n * kFeat + k] : 0.0f);
    for (int k = 0; k < kW2Stride; ++k) {
        out->w2[n * kW2Stride + k] = __float2bfloat16_rn(k < kHid ? params[kOffW2 + n * kHid + k] : 0.0f);
        out->w3[n * kW2Stride + k] = __float2bfloat16_rn(k < kHid ? params[kOffW3 + n * kHid + k] : 0.0f);
    }
    out->bias[n] = params[kOffB1 + n];
    out->bias[kHid + n] = params[kOffB2 + n];
    out->bias[2 * kHid + n] = params[kOffB3 + n];
}

// Inference of n feature rows: one warp per 32 rows, tensor-core MLP, argmax cell (and logits).
__global__ void __launch_bounds__(128) k_mlp_infer(const MlpWeights *__restrict__ wts, const float *__restrict__ X,
                                                   uint32_t n, float *logits, uint8_t *cells, float *pmax)
{
    extern __shared__ __align__(16) unsigned char sm[];
    MlpWeights &W = *reinterpret_cast<MlpWeights *>(sm);
    MlpWarpTiles *tiles = reinterpret_cast<MlpWarpTiles *>(sm + sizeof(MlpWeights));
    load_weights(W, wts);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    MlpWarpTiles &T = tiles[warp];
    const uint32_t warps_total = gridDim.x * (blockDim.x >> 5);
    for (uint32_t base = (blockIdx.x * (blockDim.x >> 5) + warp) * 32u; base < n; base += warps_total * 32u) {
        const uint32_t row = base + lane;
        const bool valid = row < n;
#pragma unroll
        for (int k = 0; k < 32; k += 2) {
            const float a = valid && k < kFeat ? X[(size_t)row * kFeat + k] : 0.0f;
            const float b = valid && k + 1 < kFeat ? X[(size_t)row * kFeat + k + 1] : 0.0f;
            st_bf16x2(T.x + lane * kXStride + k, a, b);
        }
        __syncwarp();
        const uint32_t rows_valid = n - base >= 32 ? 0xffffffffu : ((1u << (n - base)) - 1u);
        for (int r = 0; r < 2; ++r) mlp_round(W, T, r, lane, logits ? logits + (size_t)base * kCells : nullptr, rows_valid);
        if (valid) {
            if (cells) cells[row] = T.cell[lane];
            if (pmax) pmax[row] = T.pmax[lane];
        }
        __syncwarp();
    }
}

size_t mlp_infer_smem() { return sizeof(MlpWeights) + 4 * sizeof(MlpWarpTiles); }
size_t mlp_weights_bytes() { return sizeof(MlpWeights); }
size_t mlp_warp_tiles_bytes() { return sizeof(MlpWarpTiles); }

}  // namespace ccs

using namespace ccs;

struct ccs_proposal {
    float *d_params = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr, *d_loss = nullptr;
    MlpWeights *d_bf16 = nullptr;
    float *d_scratch = nullptr;   // training activations and gradients: 5 x B x 64 floats
    uint32_t scratch_batch = 0;
    uint64_t step = 0;
};

static void prop_free(ccs_proposal *p)
{
    if (!p) return;
    cudaFree(p->d_params);
    cudaFree(p->d_m);
    cudaFree(p->d_v);
    cudaFree(p->d_grad);
    cudaFree(p->d_loss);
    cudaFree(p->d_bf16);
    cudaFree(p->d_scratch);
    delete p;
}

#define PCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                        \
            return e_ == cudaErrorMemoryAllocation ? CCS_ERR_OOM : CCS_ERR_CUDA;                  \
        }                                                                                         \
    } while (0)

static ccs_status publish(ccs_proposal *p, cudaStream_t s)
{
    k_publish_bf16<<<1, kHid, 0, s>>>(p->d_params, p->d_bf16);
    PCK(cudaGetLastError());
    return CCS_OK;
}

namespace ccs {
const MlpWeights *proposal_weights(const ccs_proposal *p) { return p ? p->d_bf16 : nullptr; }
}

extern "C" {

ccs_status ccs_proposal_set_params(ccs_proposal *p, const float *host_params)
{
    if (!p || !host_params) {
        set_error("ccs_proposal_set_params: NULL argument");
        return CCS_ERR_INVALID_ARG;
    }
    PCK(cudaMemcpy(p->d_params, host_params, sizeof(float) * kParams, cudaMemcpyHostToDevice));
    PCK(cudaMemset(p->d_m, 0, sizeof(float) * kParams));
    PCK(cudaMemset(p->d_v, 0, sizeof(float) * kParams));
    p->step = 0;
    ccs_status st = publish(p, nullptr);
    if (st != CCS_OK) return st;
    PCK(cudaDeviceSynchronize());
    return CCS_OK;
}

ccs_status ccs_proposal_create(ccs_proposal **out, uint64_t seed)
{
    if (!out) {
        set_error("ccs_proposal_create: out is NULL");
        return CCS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    ccs_proposal *p = new (std::nothrow) ccs_proposal();
    if (!p) {
        set_error("host allocation failed");
        return CCS_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&p->d_params, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_m, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_v, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_grad, sizeof(float) * kParams)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_loss, sizeof(float) * 4)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_bf16, sizeof(MlpWeights))) != cudaSuccess ||
        (e = cudaMemset(p->d_bf16, 0, sizeof(MlpWeights))) != cudaSuccess) {
        set_error(std::string("ccs_proposal_create: ") + cudaGetErrorString(e));
        prop_free(p);
        return e == cudaErrorMemoryAllocation ? CCS_ERR_OOM : CCS_ERR_CUDA;
    }
    // He-normal initialisation from a seeded PCG32 stream (Box-Muller), zero biases
    std::vector<float> h(kParams, 0.0f);
    uint64_t state = 0, inc = (seed << 1) | 1u;
    auto next = [&]() {
        const uint64_t old = state;
        state = old * 6364136223846793005ull + inc;
        const uint32_t xs = (uint32_t)(((old >> 18u) ^ old) >> 27u), rot = (uint32_t)(old >> 59u);
        return (xs >> rot) | (xs << ((32u - rot) & 31u));
    };
    next();
    state += seed;
    next();
    auto normal = [&]() {
        const double u1 = ((next() >> 8) + 1.0) / 16777217.0, u2 = (next() >> 8) / 16777216.0;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    const int offs[3] = {kOffW1, kOffW2, kOffW3}, fan_in[3] = {kFeat, kHid, kHid};
    for (int l = 0; l < 3; ++l)
        for (int k = 0; k < kHid * fan_in[l]; ++k)
            h[offs[l] + k] = (float)(normal() * std::sqrt(2.0 / fan_in[l]));
    ccs_status st = ccs_proposal_set_params(p, h.data());
    if (st != CCS_OK) {
        prop_free(p);
        return st;
    }
    *out = p;
    return CCS_OK;
}

ccs_status ccs_proposal_destroy(ccs_proposal *p)
{
    prop_free(p);
    return CCS_OK;
}

ccs_status ccs_proposal_get_params(const ccs_proposal *p, float *host_params)
{
    if (!p || !host_params) {
        set_error("ccs_proposal_get_params: NULL argument");
        return CCS_ERR_INVALID_ARG;
    }
    PCK(cudaMemcpy(host_params, p->d_params, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    return CCS_OK;
}

static const char kMagic[8] = {'C', 'C', 'S', 'P', 'R', 'O', 'P', '1'};

ccs_status ccs_proposal_save(const ccs_proposal *p, const char *path)
{
    if (!p || !path) {
        set_error("ccs_proposal_save: NULL argument");
        return CCS_ERR_INVALID_ARG;
    }
    std::vector<float> h(kParams);
    ccs_status st = ccs_proposal_get_params(p, h.data());
    if (st != CCS_OK) return st;
    FILE *f = std::fopen(path, "wb");
    if (!f) {
        set_error(std::string("ccs_proposal_save: cannot open ") + path);
        return CCS_ERR_INVALID_ARG;
    }
    const uint32_t shape[4] = {kFeat, kHid, kHid, kCells};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(shape, 4, 4, f) == 4 &&
              std::fwrite(h.data(), 4, kParams, f) == (size_t)kParams;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) {
        set_error("ccs_proposal_save: write failed");
        return CCS_ERR_INVALID_ARG;
    }
    return CCS_OK;
}

ccs_status ccs_proposal_load(ccs_proposal **out, const char *path)
{
    if (!out || !path) {
        set_error("ccs_proposal_load: NULL argument");
        return CCS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) {
        set_error(std::string("ccs_proposal_load: cannot open ") + path);
        return CCS_ERR_INVALID_ARG;
    }
    char magic[8];
    uint32_t shape[4];
    std::vector<float> h(kParams);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(shape, 4, 4, f) == 4 && shape[0] == kFeat && shape[1] == kHid && shape[2] == kHid &&
              shape[3] == kCells && std::fread(h.data(), 4, kParams, f) == (size_t)kParams;
    std::fclose(f);
    if (!ok) {
        set_error("ccs_proposal_load: not a proposal file of this network shape");
        return CCS_ERR_INVALID_ARG;
    }
    ccs_status st = ccs_proposal_create(out, 0);
    if (st != CCS_OK) return st;
    return ccs_proposal_set_params(*out, h.data());
}

static ccs_status run_grad(ccs_proposal *p, const float *X, const uint8_t *y, uint32_t B, cudaStream_t s)
{
    if (B > p->scratch_batch) {
        PCK(cudaStreamSynchronize(s));
        cudaFree(p->d_scratch);
        p->d_scratch = nullptr;
        p->scratch_batch = 0;
        PCK(cudaMalloc(&p->d_scratch, sizeof(float) * 5 * kHid * (size_t)B));
        p->scratch_batch = B;
    }
    float *h1 = p->d_scratch, *h2 = h1 + (size_t)B * kHid, *dz1 = h2 + (size_t)B * kHid, *dz2 = dz1 + (size_t)B * kHid,
          *dz3 = dz2 + (size_t)B * kHid;
    PCK(cudaMemsetAsync(p->d_grad, 0, sizeof(float) * kParams, s));
    PCK(cudaMemsetAsync(p->d_loss, 0, sizeof(float), s));
    k_mlp_fwd_bwd<<<(B + 127) / 128, 128, 0, s>>>(p->d_params, X, y, B, h1, h2, dz1, dz2, dz3, p->d_loss);
    PCK(cudaGetLastError());
    const uint32_t chunk = 512;
    dim3 grid((kParams + 127) / 128, (B + chunk - 1) / chunk);
    k_mlp_wgrad<<<grid, 128, 0, s>>>(X, h1, h2, dz1, dz2, dz3, B, chunk, p->d_grad);
    PCK(cudaGetLastError());
    return CCS_OK;
}

ccs_status ccs_proposal_grad(ccs_proposal *p, const float *features, const uint8_t *labels, uint32_t batch,
                             float *grad, float *loss, void *stream)
{
    if (!p || !features || !labels || batch == 0 || !grad) {
        set_error("ccs_proposal_grad: NULL argument or empty batch");
        return CCS_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    ccs_status st = run_grad(p, features, labels, batch, s);
    if (st != CCS_OK) return st;
    PCK(cudaMemcpyAsync(grad, p->d_grad, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, s));
    if (loss) PCK(cudaMemcpyAsync(loss, p->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return CCS_OK;
}

ccs_status ccs_proposal_train_step(ccs_proposal *p, const float *features, const uint8_t *labels, uint32_t batch,
                                   float lr, float *loss, void *stream)
{
    if (!p || !features || !labels || batch == 0 || !(lr > 0.0f)) {
        set_error("ccs_proposal_train_step: NULL argument, empty batch or lr <= 0");
        return CCS_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    ccs_status st = run_grad(p, features, labels, batch, s);
    if (st != CCS_OK) return st;
    p->step += 1;
    const float b1c = 1.0f - std::pow(0.9f, (float)p->step), b2c = 1.0f - std::pow(0.999f, (float)p->step);
    k_adam<<<(kParams + 127) / 128, 128, 0, s>>>(p->d_params, p->d_m, p->d_v, p->d_grad, lr, b1c, b2c);
    PCK(cudaGetLastError());
    if ((st = publish(p, s)) != CCS_OK) return st;
    if (loss) PCK(cudaMemcpyAsync(loss, p->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return CCS_OK;
}

ccs_status ccs_proposal_infer(const ccs_proposal *p, const float *features, uint32_t n, float *logits, uint8_t *cells,
                              float *pmax, void *stream)
{
    if (!p || !features) {
        set_error("ccs_proposal_infer: NULL argument");
        return CCS_ERR_INVALID_ARG;
    }
    if (n == 0) return CCS_OK;
    const size_t smem = mlp_infer_smem();
    static bool configured = false;
    if (!configured) {
        PCK(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = true;
    }
    const uint32_t warps = (n + 31) / 32;
    const uint32_t blocks = (warps + 3) / 4 < 1024 ? (warps + 3) / 4 : 1024;
    k_mlp_infer<<<blocks, 128, smem, (cudaStream_t)stream>>>(p->d_bf16, features, n, logits, cells, pmax);
    PCK(cudaGetLastError());
    return CCS_OK;
}

}  // extern "C"
