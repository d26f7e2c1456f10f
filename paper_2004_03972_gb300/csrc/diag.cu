// diag.cu -- the MD Hamiltonian as a diagnostic (Results, Eq. (3); Methods,
// "Leapfrog algorithm"): per replica
//   H_MD = alpha(tau) sum_i (p_i^2 / 2 + phi_i^M)
//        + beta(tau) (1/2 sum_ij J_ij phi_i phi_j + sum_i h_i |phi_i| phi_i)
//        = alpha sum_i (p_i^2 / 2 + phi_i^M) + beta / 2 sum_i phi_i L_i,
// with the kick's local field L_i = sum_j J_ij phi_j + 2 h_i |phi_i| (the
// library's own field kernel).  The leapfrog momentum is staggered; with
// half_kick the kernel first completes it to the integer step,
//   p_i <- p_i - (h/2) (alpha M phi_i^(M-1) + beta L_i),
// which turns hqa_run's p^(S-1/2) into p^(S).  The per-spin terms are formed
// and summed in FP64 (the only FP64 arithmetic on the device): the energy
// drift of a long run is a small difference of large sums.
#include "hqa_internal.cuh"

namespace {

__device__ __forceinline__ double ipow_d(double x, int m)
{
    double r = 1.0;
    for (int k = 0; k < m; ++k) r *= x;
    return r;
}

__global__ void __launch_bounds__(256) k_hmd(int N, const float* __restrict__ phi,
                                             const float* __restrict__ p,
                                             const float* __restrict__ L, double alpha,
                                             double beta, int M, double half_h,
                                             double* __restrict__ out)
{
    const int r = blockIdx.x;
    const size_t o = (size_t)r * N;
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double x = phi[o + i];
        const double l = L[o + i];
        double q = p[o + i];
        if (half_h != 0.0) q -= half_h * (alpha * M * ipow_d(x, M - 1) + beta * l);
        acc += alpha * (0.5 * q * q + ipow_d(x, M)) + 0.5 * beta * x * l;
    }
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[r] = t;
    }
}

}  // namespace

extern "C" hqa_status hqa_hmd(hqa_ctx* ctx, const hqa_schedule* sched, double tau,
                              int32_t replicas, const float* phi, const float* p,
                              int32_t half_kick, double* out, const hqa_run_opts* opts,
                              void* stream)
{
    if (!ctx || !sched || replicas < 1 || !phi || !p || !out || !std::isfinite(tau))
        return HQA_ERR_INVALID_ARG;
    if (((uintptr_t)out % 8) || ((uintptr_t)phi % 4) || ((uintptr_t)p % 4))
        return HQA_ERR_INVALID_ARG;
    if (ctx->is_batch || sched->kind == HQA_SCHED_TABLE) return HQA_ERR_UNSUPPORTED;
    if (sched->kind != HQA_SCHED_PAPER && sched->kind != HQA_SCHED_LINEAR_GAMMA)
        return HQA_ERR_INVALID_ARG;
    if (sched->M < 2 || sched->M > 16 || !std::isfinite(sched->hstep)) return HQA_ERR_INVALID_ARG;
    hqa_capture_touch(ctx);
    const size_t RN = (size_t)replicas * ctx->N;
    hqa_status s = hqa_reserve(ctx, &ctx->d_diag, &ctx->diag_cap, RN * sizeof(float));
    if (s != HQA_OK) return s;
    float* L = static_cast<float*>(ctx->d_diag);
    s = hqa_local_field(ctx, replicas, phi, L, opts, stream);
    if (s != HQA_OK) return s;
    const double alpha = hqa_sched_alpha(sched, tau);
    const double beta = hqa_sched_beta(sched, tau);
    const double half_h = half_kick ? 0.5 * sched->hstep : 0.0;
    k_hmd<<<replicas, 256, 0, static_cast<cudaStream_t>(stream)>>>(ctx->N, phi, p, L, alpha, beta,
                                                                   sched->M, half_h, out);
    return hqa_capture_note(cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA);
}
