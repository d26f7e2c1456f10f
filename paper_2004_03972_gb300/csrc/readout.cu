// readout.cu -- spin readout, frozen/ambivalent split and exact int64 energies.
//
// Readout (Results, "Sorting frozen and ambivalent variables"; HQA section):
//   s_i = sgn(phibar_i) with sgn(0) = +1; spins ordered by (|phibar_i|, i)
//   ascending; the first n are ambivalent.  One CTA per replica finds the
//   n-th smallest 64-bit key (|phibar| bits << 32 | i) by an 8-pass radix
//   select over 8-bit digits; a spin is ambivalent iff its key <= that key.
//   Keys are unique, so no tie handling is needed beyond the index bits.
// Energy (Eq. (1)) and cut (Methods, "MAX-CUT and Ising spin-glass"):
//   ordered = sum_i s_i sum_{j != i} J_ij s_j   (int32 per row, int64 total)
//   H = ordered / 2 + sum_i h_i s_i,  C = (sum_{ij} J_ij - ordered) / 4.
#include "hqa_internal.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned long long rkey(const float* x, int i)
{
    return ((unsigned long long)__float_as_uint(fabsf(x[i])) << 32) | (unsigned)i;
}

// One replica: x = its N window means; spins/frozen point at its row;
// tally at its two counters (any may be null).
__device__ __forceinline__ void readout_block(const float* __restrict__ x, int N, int n,
                                              int8_t* spins, uint8_t* frozen, int32_t* tally,
                                              uint32_t* status)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ unsigned s_target;
    const int nn = n < 0 ? 0 : (n > N ? N : n);
    unsigned long long K = 0;  // ambivalent iff key <= K (nn >= 1)
    if (nn > 0 && nn < N) {
        if (threadIdx.x == 0) {
            s_prefix = 0;
            s_mask = 0;
            s_target = (unsigned)(nn - 1);
        }
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
            __syncthreads();
            const unsigned long long pre = s_prefix, msk = s_mask;
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const unsigned long long k = rkey(x, i);
                if ((k & msk) == pre) atomicAdd(&hist[(k >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned cum = 0, tgt = s_target;
                for (int b = 0; b < 256; ++b) {
                    if (cum + hist[b] > tgt) {
                        s_prefix = pre | ((unsigned long long)b << shift);
                        s_target = tgt - cum;
                        break;
                    }
                    cum += hist[b];
                }
                s_mask = msk | (255ull << shift);
            }
            __syncthreads();
        }
        K = s_prefix;
    }
    bool bad = false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float v = x[i];
        bad |= !isfinite(v);
        if (spins) spins[i] = v >= 0.f ? 1 : -1;
        bool amb;
        if (nn == 0) amb = false;
        else if (nn == N) amb = true;
        else amb = rkey(x, i) <= K;
        if (frozen) frozen[i] = amb ? 0 : 1;
    }
    if (tally && threadIdx.x == 0) {
        tally[0] = N - nn;
        tally[1] = nn;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, HQA_DEV_NONFINITE);
}

__global__ void __launch_bounds__(kThreads) k_readout(const float* __restrict__ phibar, int N,
                                                      int n, int8_t* spins, uint8_t* frozen,
                                                      int32_t* tally, uint32_t* status)
{
    const size_t r = blockIdx.x, o = r * N;
    readout_block(phibar + o, N, n, spins ? spins + o : nullptr, frozen ? frozen + o : nullptr,
                  tally ? tally + 2 * r : nullptr, status);
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long* sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;  // valid in thread 0
}

// One replica: s = its N spins; energy/cut point at its result (may be null).
__device__ __forceinline__ void energy_block(const int32_t* __restrict__ row_ptr,
                                             const int32_t* __restrict__ col,
                                             const int8_t* __restrict__ val,
                                             const int32_t* __restrict__ h, int N, int64_t sumJ,
                                             const int8_t* s, int64_t* energy, int64_t* cut)
{
    __shared__ long long sh[kThreads / 32];
    // one warp per row: lanes stride the row's entries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long ordered = 0, field = 0;
    for (int i = warp; i < N; i += nw) {
        int acc = 0;
        for (int k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) acc += (int)val[k] * (int)s[col[k]];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            ordered += (long long)acc * s[i];
            if (h) field += (long long)h[i] * s[i];
        }
    }
    const long long tord = block_sum_ll(ordered, sh);
    const long long tfld = block_sum_ll(field, sh);
    if (threadIdx.x == 0) {
        if (energy) *energy = tord / 2 + tfld;
        if (cut) *cut = (sumJ - tord) / 4;
    }
}

__global__ void __launch_bounds__(kThreads) k_energy_csr(const int32_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col,
                                                         const int8_t* __restrict__ val,
                                                         const int32_t* __restrict__ h, int N,
                                                         int64_t sumJ, const int8_t* spins,
                                                         int64_t* energy, int64_t* cut)
{
    const int r = blockIdx.x;
    energy_block(row_ptr, col, val, h, N, sumJ, spins + (size_t)r * N, energy ? energy + r : nullptr,
                 cut ? cut + r : nullptr);
}

// Ising energy in FP64 for real-valued couplings and fields (Results Eq. (1)):
// one block per replica, E = sum_i s_i (h_i + 1/2 sum_j J_ij s_j), each row sum
// and each thread's partial in FP64, then a fixed-shape reduction (warp
// shuffles, warps in order), so the result does not depend on timing.
__global__ void __launch_bounds__(kThreads) k_energy_f64(const int32_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col,
                                                         const float* __restrict__ val,
                                                         const float* __restrict__ h, int N,
                                                         const int8_t* __restrict__ spins,
                                                         double* __restrict__ energy)
{
    const int r = blockIdx.x;
    const int8_t* s = spins + (size_t)r * N;
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double g = 0.0;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) g += (double)val[k] * (double)s[col[k]];
        acc += (double)s[i] * (0.5 * g + (h ? (double)h[i] : 0.0));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double sh[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        energy[r] = t;
    }
}

// Batch of instances: block b is replica b % R of instance b / R; each
// instance's arrays start at R * off[k] (spin-indexed) or R * k (per replica).
__global__ void __launch_bounds__(kThreads) k_readout_batch(const BatchInst* __restrict__ inst,
                                                            int R, int n, const float* phibar,
                                                            int8_t* spins, uint8_t* frozen,
                                                            int32_t* tally, uint32_t* status)
{
    const int k = blockIdx.x / R, r = blockIdx.x % R;
    const BatchInst b = inst[k];
    const size_t o = (size_t)R * b.off + (size_t)r * b.N, q = (size_t)k * R + r;
    readout_block(phibar + o, b.N, n, spins ? spins + o : nullptr, frozen ? frozen + o : nullptr,
                  tally ? tally + 2 * q : nullptr, status);
}

__global__ void __launch_bounds__(kThreads) k_energy_batch(const BatchInst* __restrict__ inst, int R,
                                                           const int8_t* spins, int64_t* energy,
                                                           int64_t* cut)
{
    const int k = blockIdx.x / R, r = blockIdx.x % R;
    const BatchInst b = inst[k];
    const size_t o = (size_t)R * b.off + (size_t)r * b.N, q = (size_t)k * R + r;
    energy_block(b.row_ptr, b.col, b.val_i8, b.h_i32, b.N, b.sumJ, spins + o,
                 energy ? energy + q : nullptr, cut ? cut + q : nullptr);
}

}  // namespace

hqa_status hqa_launch_readout_batch(hqa_ctx* batch, int32_t R, const float* phibar, int32_t n,
                                    int8_t* spins, uint8_t* frozen, int32_t* tally, cudaStream_t st)
{
    const int count = (int)batch->members.size();
    if (count == 0 || R <= 0) return HQA_OK;
    k_readout_batch<<<count * R, kThreads, 0, st>>>(batch->d_binst, R, n, phibar, spins, frozen,
                                                    tally, batch->d_status);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_launch_energy_batch(hqa_ctx* batch, int32_t R, const int8_t* spins, int64_t* energy,
                                   int64_t* cut, cudaStream_t st)
{
    const int count = (int)batch->members.size();
    if (!batch->integer) return HQA_ERR_UNSUPPORTED;
    if (count == 0 || R <= 0) return HQA_OK;
    k_energy_batch<<<count * R, kThreads, 0, st>>>(batch->d_binst, R, spins, energy, cut);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_launch_readout(hqa_ctx* ctx, int32_t R, const float* phibar, int32_t n,
                              int8_t* spins, uint8_t* frozen, int32_t* tally, cudaStream_t st)
{
    if (R <= 0) return HQA_OK;
    k_readout<<<R, kThreads, 0, st>>>(phibar, ctx->N, n, spins, frozen, tally, ctx->d_status);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

extern "C" hqa_status hqa_energy_f64(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                                     double* energy, void* stream)
{
    if (!ctx || replicas < 1 || !spins || !energy || ((uintptr_t)energy % 8))
        return HQA_ERR_INVALID_ARG;
    if (ctx->is_batch) return HQA_ERR_UNSUPPORTED;
    hqa_capture_touch(ctx);
    k_energy_f64<<<replicas, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        ctx->d_row_ptr, ctx->d_col, ctx->d_val, ctx->has_h ? ctx->d_h : nullptr, ctx->N, spins,
        energy);
    return hqa_capture_note(cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA);
}

hqa_status hqa_launch_energy(hqa_ctx* ctx, int32_t R, const int8_t* spins, int64_t* energy,
                             int64_t* cut, cudaStream_t st)
{
    if (!ctx->integer) return HQA_ERR_UNSUPPORTED;
    if (R <= 0) return HQA_OK;
    k_energy_csr<<<R, kThreads, 0, st>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val_i8,
                                         ctx->has_h ? ctx->d_h_i32 : nullptr, ctx->N,
                                         ctx->sum_J_all, spins, energy, cut);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}
