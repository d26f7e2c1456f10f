// mlp.cu -- the surrogate gate's per-spin MLP (6 -> 64 -> 64 -> 2), trained and
// evaluated by hand-written kernels.  This learned gate is an addition to
// the method: the paper has none.
//
//   forward : z = W3 relu(W2 relu(W1 x + b1) + b2) + b3, one thread per sample,
//             weights staged in shared memory (broadcast reads)
//   grad    : mean binary cross-entropy of the two sigmoid outputs; a block
//             takes 128 samples per tile, keeps activations and their
//             gradients in shared rows (stride 65: conflict-free), and each
//             thread accumulates ~38 parameters' gradients over all its tiles
//   reduce  : sum of the per-block partials
//   adamw   : Adam with decoupled weight decay on the FP32 master weights
// Precision: FP32, or BF16 (weights, inputs and hidden activations rounded to
// BF16, FP32 accumulation; gradients are taken w.r.t. the rounded forward).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "hqa_internal.cuh"

namespace {

constexpr int IN = 6, H = 64, OUT = 2;
constexpr int oW1 = 0, ob1 = oW1 + H * IN, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H,
              ob3 = oW3 + OUT * H, P = ob3 + OUT;
constexpr int TS = 128;                   // samples per tile = threads per block
constexpr int NPT = (P + TS - 1) / TS;    // parameters per thread
constexpr int RS = H + 1;                 // padded shared row

__device__ __forceinline__ float rnd(float x, bool bf)
{
    return bf ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + __expf(-z)); }

__device__ __forceinline__ float softplus(float z)
{
    return z > 0.f ? z + log1pf(__expf(-z)) : log1pf(__expf(z));
}

constexpr int FT = 64;  // forward threads per block (static shared memory stays under 48 KB)

__global__ void __launch_bounds__(FT) k_mlp_forward(int64_t n, const float* __restrict__ x,
                                                     float* __restrict__ z,
                                                     const float* __restrict__ w, int bf)
{
    __shared__ float sw[P];
    __shared__ float h1s[FT * RS];    // this thread's hidden row, padded: conflict-free
    for (int i = threadIdx.x; i < P; i += blockDim.x) sw[i] = rnd(w[i], bf);
    __syncthreads();
    float* h1 = h1s + threadIdx.x * RS;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        float xi[IN];
#pragma unroll
        for (int i = 0; i < IN; ++i) xi[i] = rnd(x[s * IN + i], bf);
#pragma unroll 4
        for (int k = 0; k < H; ++k) {
            float a = sw[ob1 + k];
#pragma unroll
            for (int i = 0; i < IN; ++i) a = fmaf(sw[oW1 + k * IN + i], xi[i], a);
            h1[k] = rnd(fmaxf(a, 0.f), bf);
        }
        float z0 = sw[ob3], z1 = sw[ob3 + 1];
#pragma unroll 1
        for (int j = 0; j < H; ++j) {
            float a = sw[ob2 + j];
#pragma unroll 8
            for (int k = 0; k < H; ++k) a = fmaf(sw[oW2 + j * H + k], h1[k], a);
            const float h2 = rnd(fmaxf(a, 0.f), bf);
            z0 = fmaf(sw[oW3 + j], h2, z0);
            z1 = fmaf(sw[oW3 + H + j], h2, z1);
        }
        z[s * OUT] = z0;
        z[s * OUT + 1] = z1;
    }
}

// Shared layout (floats): weights P | x [TS][IN] | h1, d1, h2, d2 [TS][RS] | dz [TS][OUT]
__global__ void __launch_bounds__(TS) k_mlp_grad(int64_t n, const float* __restrict__ x,
                                                 const float* __restrict__ y,
                                                 const float* __restrict__ w,
                                                 float* __restrict__ part, int bf, float inv_n)
{
    extern __shared__ float sm[];
    float* sw = sm;
    float* xs = sw + ((P + 3) & ~3);
    float* h1s = xs + TS * IN;
    float* d1s = h1s + TS * RS;
    float* h2s = d1s + TS * RS;
    float* d2s = h2s + TS * RS;
    float* dzs = d2s + TS * RS;
    const int t = threadIdx.x;
    for (int i = t; i < P; i += TS) sw[i] = rnd(w[i], bf);
    float acc[NPT];
#pragma unroll
    for (int q = 0; q < NPT; ++q) acc[q] = 0.f;
    float lsum = 0.f;
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile * TS < n; tile += gridDim.x) {
        const int64_t s = tile * TS + t;
        const bool valid = s < n;
        // ---- forward, one sample per thread ----
        float xi[IN], h1[H];
#pragma unroll
        for (int i = 0; i < IN; ++i) {
            xi[i] = valid ? rnd(x[s * IN + i], bf) : 0.f;
            xs[t * IN + i] = xi[i];
        }
#pragma unroll
        for (int k = 0; k < H; ++k) {
            float a = sw[ob1 + k];
#pragma unroll
            for (int i = 0; i < IN; ++i) a = fmaf(sw[oW1 + k * IN + i], xi[i], a);
            h1[k] = rnd(fmaxf(a, 0.f), bf);
            h1s[t * RS + k] = valid ? h1[k] : 0.f;
        }
        float z0 = sw[ob3], z1 = sw[ob3 + 1];
        for (int j = 0; j < H; ++j) {
            float a = sw[ob2 + j];
#pragma unroll
            for (int k = 0; k < H; ++k) a = fmaf(sw[oW2 + j * H + k], h1[k], a);
            const float h2 = rnd(fmaxf(a, 0.f), bf);
            h2s[t * RS + j] = valid ? h2 : 0.f;
            z0 = fmaf(sw[oW3 + j], h2, z0);
            z1 = fmaf(sw[oW3 + H + j], h2, z1);
        }
        // ---- loss and d loss / d z ----
        float dz0 = 0.f, dz1 = 0.f;
        if (valid) {
            const float y0 = y[s * OUT], y1 = y[s * OUT + 1];
            lsum += softplus(z0) - y0 * z0 + softplus(z1) - y1 * z1;
            dz0 = (sigm(z0) - y0) * inv_n;
            dz1 = (sigm(z1) - y1) * inv_n;
        }
        dzs[t * OUT] = dz0;
        dzs[t * OUT + 1] = dz1;
        // ---- backward through layer 3 and the second ReLU ----
        for (int j = 0; j < H; ++j) {
            const float g = fmaf(sw[oW3 + j], dz0, sw[oW3 + H + j] * dz1);
            d2s[t * RS + j] = h2s[t * RS + j] > 0.f ? g : 0.f;
        }
        // ---- backward through layer 2 and the first ReLU ----
        float dh1[H];
#pragma unroll
        for (int k = 0; k < H; ++k) dh1[k] = 0.f;
        for (int j = 0; j < H; ++j) {
            const float dj = d2s[t * RS + j];
#pragma unroll
            for (int k = 0; k < H; ++k) dh1[k] = fmaf(sw[oW2 + j * H + k], dj, dh1[k]);
        }
#pragma unroll
        for (int k = 0; k < H; ++k) d1s[t * RS + k] = h1[k] > 0.f ? dh1[k] : 0.f;
        __syncthreads();
        // ---- parameter gradients: sums over the tile's samples ----
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int p = t + TS * q;
            if (p >= P) break;
            float g = 0.f;
            if (p < ob1) {
                const int k = p / IN, i = p % IN;
                for (int u = 0; u < TS; ++u) g = fmaf(d1s[u * RS + k], xs[u * IN + i], g);
            } else if (p < oW2) {
                const int k = p - ob1;
                for (int u = 0; u < TS; ++u) g += d1s[u * RS + k];
            } else if (p < ob2) {
                const int j = (p - oW2) / H, k = (p - oW2) % H;
                for (int u = 0; u < TS; ++u) g = fmaf(d2s[u * RS + j], h1s[u * RS + k], g);
            } else if (p < oW3) {
                const int j = p - ob2;
                for (int u = 0; u < TS; ++u) g += d2s[u * RS + j];
            } else if (p < ob3) {
                const int o = (p - oW3) / H, j = (p - oW3) % H;
                for (int u = 0; u < TS; ++u) g = fmaf(dzs[u * OUT + o], h2s[u * RS + j], g);
            } else {
                const int o = p - ob3;
                for (int u = 0; u < TS; ++u) g += dzs[u * OUT + o];
            }
            acc[q] += g;
        }
        __syncthreads();
    }
    float* out = part + (size_t)blockIdx.x * (P + 1);
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        const int p = t + TS * q;
        if (p < P) out[p] = acc[q];
    }
    // loss: block sum
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    __shared__ float sl[TS / 32];
    if ((t & 31) == 0) sl[t >> 5] = lsum;
    __syncthreads();
    if (t == 0) {
        float v = 0.f;
        for (int k = 0; k < TS / 32; ++k) v += sl[k];
        out[P] = v * inv_n;
    }
}

__global__ void k_mlp_reduce(int nparts, const float* __restrict__ part, float* __restrict__ grad,
                             float* __restrict__ loss)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * (P + 1) + p];
        if (p < P) grad[p] = s;
        else if (loss) *loss = s;
    }
}

__global__ void k_mlp_adamw(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float wd, float c1, float c2)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const float gp = g[p];
        const float mp = b1 * m[p] + (1.f - b1) * gp;
        const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
        m[p] = mp;
        v[p] = vp;
        const float mh = mp / c1, vh = vp / c2;
        w[p] -= lr * (mh / (sqrtf(vh) + eps) + wd * w[p]);
    }
}

size_t grad_smem()
{
    return sizeof(float) * (((P + 3) & ~3) + TS * IN + 4 * TS * RS + TS * OUT);
}

}  // namespace

struct hqa_mlp {
    int device = 0;
    int sm_count = 0;
    float* d_w = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    float* d_part = nullptr;
    size_t part_cap = 0;
    int64_t step = 0;
};

extern "C" {

hqa_status hqa_mlp_create(const float* params, hqa_mlp** out)
{
    if (!out || !params) return HQA_ERR_INVALID_ARG;
    *out = nullptr;
    for (int p = 0; p < P; ++p)
        if (!std::isfinite(params[p])) return HQA_ERR_NONFINITE_INPUT;
    hqa_mlp* m = new (std::nothrow) hqa_mlp();
    if (!m) return HQA_ERR_OOM;
    auto fail = [&](hqa_status s) {
        cudaFree(m->d_w);
        cudaFree(m->d_m);
        cudaFree(m->d_v);
        delete m;
        return s;
    };
    if (cudaGetDevice(&m->device) != cudaSuccess) return fail(HQA_ERR_CUDA);
    cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
    if (cudaMalloc(&m->d_w, P * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->d_m, P * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->d_v, P * sizeof(float)) != cudaSuccess)
        return fail(HQA_ERR_OOM);
    if (cudaMemcpy(m->d_w, params, P * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->d_m, 0, P * sizeof(float)) != cudaSuccess ||
        cudaMemset(m->d_v, 0, P * sizeof(float)) != cudaSuccess)
        return fail(HQA_ERR_CUDA);
    *out = m;
    return HQA_OK;
}

hqa_status hqa_mlp_params(const hqa_mlp* m, float* params)
{
    if (!m || !params) return HQA_ERR_INVALID_ARG;
    HQA_CUDA_TRY(cudaDeviceSynchronize());
    HQA_CUDA_TRY(cudaMemcpy(params, m->d_w, P * sizeof(float), cudaMemcpyDeviceToHost));
    return HQA_OK;
}

hqa_status hqa_mlp_forward(hqa_mlp* m, int64_t n, const float* x, float* logits, int32_t precision,
                           void* stream)
{
    if (!m || n < 0 || (n > 0 && (!x || !logits))) return HQA_ERR_INVALID_ARG;
    if (precision != HQA_PREC_FP32 && precision != HQA_PREC_BF16) return HQA_ERR_INVALID_ARG;
    if (n == 0) return HQA_OK;
    const int64_t blocks = std::min<int64_t>((n + FT - 1) / FT, (int64_t)m->sm_count * 24);
    k_mlp_forward<<<(int)blocks, FT, 0, static_cast<cudaStream_t>(stream)>>>(
        n, x, logits, m->d_w, precision == HQA_PREC_BF16);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_mlp_grad(hqa_mlp* m, int64_t n, const float* x, const float* y, float* grad,
                        float* loss, int32_t precision, void* stream)
{
    if (!m || n < 1 || !x || !y || !grad) return HQA_ERR_INVALID_ARG;
    if (precision != HQA_PREC_FP32 && precision != HQA_PREC_BF16) return HQA_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t tiles = (n + TS - 1) / TS;
    const int blocks = (int)std::min<int64_t>(tiles, (int64_t)m->sm_count);
    const size_t need = (size_t)blocks * (P + 1) * sizeof(float);
    if (need > m->part_cap) {
        cudaFree(m->d_part);
        m->d_part = nullptr;
        m->part_cap = 0;
        HQA_CUDA_TRY(cudaMalloc(&m->d_part, need));
        m->part_cap = need;
    }
    const size_t smem = grad_smem();
    HQA_CUDA_TRY(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_grad<<<blocks, TS, smem, st>>>(n, x, y, m->d_w, m->d_part, precision == HQA_PREC_BF16,
                                         1.f / (float)n);
    k_mlp_reduce<<<(P + 1 + 255) / 256, 256, 0, st>>>(blocks, m->d_part, grad, loss);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_mlp_adamw(hqa_mlp* m, const float* grad, float lr, float beta1, float beta2,
                         float eps, float weight_decay, void* stream)
{
    if (!m || !grad || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
        return HQA_ERR_INVALID_ARG;
    ++m->step;
    const float c1 = 1.f - powf(beta1, (float)m->step), c2 = 1.f - powf(beta2, (float)m->step);
    k_mlp_adamw<<<(P + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        m->d_w, grad, m->d_m, m->d_v, lr, beta1, beta2, eps, weight_decay, c1, c2);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

void hqa_mlp_destroy(hqa_mlp* m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->d_w);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_part);
    delete m;
}

}  // extern "C"
