// surrogate.cu -- features for the surrogate gate and its readout (an
// addition to the method: the paper has no learned component).
//
// hqa_run_features runs the first `steps` leapfrog steps of a trajectory as
// `segments` consecutive resumed runs (bitwise the same trajectory) and, at
// every segment end, samples phi and the local field L.  Six features per
// spin and replica, z-scored per replica over the spins:
//   0 phi at the end, 1 p at the end (p^(S-1/2)),
//   2 mean of L over the samples, 3 variance of L over the samples,
//   4 window mean of phi over the last W steps,
//   5 fraction of consecutive samples between which sgn(phi) changed.
// hqa_surrogate_readout turns the network's logits (z_f: frozen, z_s: s=+1)
// into spins s = sgn(z_s), a rank split on the confidence
// c = sigmoid(z_f) |2 sigmoid(z_s) - 1| (the n least confident spins are
// ambivalent), and per replica the expected number of wrong frozen signs
// E = sum_frozen (1 - |2 sigmoid(z_s) - 1|) / 2; a replica is accepted
// (stops early) when E <= max_expected_errors.
#include <cmath>

#include "hqa_internal.cuh"

namespace {

__global__ void k_feat_zero(size_t n, float* acc)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc[i] = 0.f;
}

// acc layout per element: [sumL, sumL2, flips, last sign]
__global__ void k_feat_accum(size_t n, const float* __restrict__ phi, const float* __restrict__ L,
                             float4* __restrict__ acc, int first)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float4 a = acc[i];
        const float l = L[i];
        const float sg = phi[i] >= 0.f ? 1.f : -1.f;
        a.x += l;
        a.y += l * l;
        if (!first && sg != a.w) a.z += 1.f;
        a.w = sg;
        acc[i] = a;
    }
}

// one block per replica: raw features, then z-score each feature over the N spins
__global__ void __launch_bounds__(256) k_feat_final(int N, int samples, const float* __restrict__ phi,
                                                    const float* __restrict__ p,
                                                    const float* __restrict__ phibar,
                                                    const float4* __restrict__ acc,
                                                    float* __restrict__ feat)
{
    const int r = blockIdx.x;
    const size_t o = (size_t)r * N;
    const float inv_s = 1.f / (float)samples;
    const float inv_f = 1.f / (float)(samples > 1 ? samples - 1 : 1);
    __shared__ float s_sum[6][8], s_sq[6][8];
    float sum[6] = {0, 0, 0, 0, 0, 0}, sq[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float4 a = acc[o + i];
        const float mL = a.x * inv_s;
        float f[6] = {phi[o + i], p[o + i], mL, fmaxf(a.y * inv_s - mL * mL, 0.f), phibar[o + i],
                      a.z * inv_f};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            feat[(o + i) * 6 + k] = f[k];
            sum[k] += f[k];
            sq[k] += f[k] * f[k];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        for (int s = 16; s > 0; s >>= 1) {
            sum[k] += __shfl_xor_sync(0xffffffffu, sum[k], s);
            sq[k] += __shfl_xor_sync(0xffffffffu, sq[k], s);
        }
        if (lane == 0) {
            s_sum[k][warp] = sum[k];
            s_sq[k][warp] = sq[k];
        }
    }
    __syncthreads();
    __shared__ float s_mu[6], s_inv[6];
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        float a = 0.f, b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_sum[k][w];
            b += s_sq[k][w];
        }
        const float mu = a / (float)N;
        const float var = fmaxf(b / (float)N - mu * mu, 0.f);
        s_mu[k] = mu;
        s_inv[k] = var > 1e-20f ? rsqrtf(var) : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const size_t q = (o + i) * 6 + k;
            feat[q] = (feat[q] - s_mu[k]) * s_inv[k];
        }
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

__global__ void k_sur_key(size_t n, const float* __restrict__ z, float* __restrict__ key)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float zf = z[2 * i], zs = z[2 * i + 1];
        // clamped to the smallest normal float so that a zero confidence keeps the sign of z_s
        const float c = fmaxf(sigm(zf) * fabsf(2.f * sigm(zs) - 1.f), 1.17549435e-38f);
        key[i] = zs >= 0.f ? c : -c;
    }
}

__global__ void __launch_bounds__(256) k_sur_decide(int N, const float* __restrict__ z,
                                                    const uint8_t* __restrict__ frozen,
                                                    float max_err, uint8_t* accept, float* err)
{
    const int r = blockIdx.x;
    const size_t o = (size_t)r * N;
    float e = 0.f;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        if (frozen[o + i]) e += 0.5f * (1.f - fabsf(2.f * sigm(z[2 * (o + i) + 1]) - 1.f));
    for (int s = 16; s > 0; s >>= 1) e += __shfl_xor_sync(0xffffffffu, e, s);
    __shared__ float sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        if (err) err[r] = t;
        if (accept) accept[r] = t <= max_err ? 1 : 0;
    }
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 8192); }

}  // namespace

extern "C" {

hqa_status hqa_run_features(hqa_ctx* ctx, const hqa_schedule* sched, double dt, int64_t steps,
                            int32_t segments, int32_t replicas, uint64_t seed,
                            const hqa_run_opts* opts, float* features, float* phi, float* p,
                            void* stream)
{
    if (!ctx || ctx->is_batch || !sched || !features || !phi || !p || replicas < 1)
        return HQA_ERR_INVALID_ARG;
    if (segments < 1 || steps < segments) return HQA_ERR_INVALID_ARG;
    hqa_run_opts o;
    if (opts) o = *opts;
    else hqa_run_opts_default(&o);
    if (o.start_step != 0) return HQA_ERR_INVALID_ARG;
    hqa_capture_touch(ctx);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t RN = (size_t)replicas * ctx->N;
    // workspace: accumulators (float4), phibar, L
    const size_t need = RN * (16 + 4 + 4);
    hqa_status s = hqa_reserve(ctx, &ctx->d_feat, &ctx->feat_cap, need);
    if (s != HQA_OK) return s;
    float4* acc = static_cast<float4*>(ctx->d_feat);
    float* phibar = reinterpret_cast<float*>(acc + RN);
    float* L = phibar + RN;
    k_feat_zero<<<grid_for(4 * RN), 256, 0, st>>>(4 * RN, reinterpret_cast<float*>(acc));
    int64_t m0 = 0;
    for (int seg = 0; seg < segments; ++seg) {
        const int64_t len = steps / segments + (seg < steps % segments ? 1 : 0);
        hqa_run_opts so = o;
        if (seg > 0) {
            so.init = HQA_INIT_GIVEN;
            so.phi0 = phi;
            so.p0 = p;
            so.start_step = m0;
        }
        hqa_result res{};
        res.phi = phi;
        res.p = p;
        res.phibar = phibar;
        s = hqa_run(ctx, sched, dt, len, replicas, seed, &so, &res, stream);
        if (s != HQA_OK) return s;
        hqa_run_opts fo = o;
        fo.init = HQA_INIT_PAPER;
        s = hqa_local_field(ctx, replicas, phi, L, &fo, stream);
        if (s != HQA_OK) return s;
        k_feat_accum<<<grid_for(RN), 256, 0, st>>>(RN, phi, L, acc, seg == 0);
        m0 += len;
    }
    k_feat_final<<<replicas, 256, 0, st>>>(ctx->N, segments, phi, p, phibar, acc, features);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_surrogate_readout(hqa_ctx* ctx, int32_t replicas, const float* logits, int32_t n,
                                 float max_expected_errors, int8_t* spins, uint8_t* frozen,
                                 uint8_t* accept, float* expected_errors, void* stream)
{
    if (!ctx || ctx->is_batch || replicas < 1 || !logits || !spins || !frozen) return HQA_ERR_INVALID_ARG;
    hqa_capture_touch(ctx);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t RN = (size_t)replicas * ctx->N;
    hqa_status s = hqa_reserve(ctx, &ctx->d_feat, &ctx->feat_cap, RN * 4);
    if (s != HQA_OK) return s;
    float* key = static_cast<float*>(ctx->d_feat);
    k_sur_key<<<grid_for(RN), 256, 0, st>>>(RN, logits, key);
    s = hqa_launch_readout(ctx, replicas, key, n, spins, frozen, nullptr, st);
    if (s != HQA_OK) return s;
    if (accept || expected_errors)
        k_sur_decide<<<replicas, 256, 0, st>>>(ctx->N, logits, frozen, max_expected_errors, accept,
                                               expected_errors);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

}  // extern "C"
