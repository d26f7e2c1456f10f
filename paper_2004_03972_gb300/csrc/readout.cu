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
#include <vector>

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

// Integer energy for couplings in {-1, 0, +1} with many couplings per row
// (dense instances), from bit masks instead of per-coupling gathers.  With
// bit j of a spin mask set where s_j = -1, and per row i the masks of its
// nonzero couplings (nz) and of its negative ones (neg), a term J_ij s_j is
// -1 exactly where (neg_i XOR S) AND nz_i has a bit, so
//   g_i = sum_j J_ij s_j = deg_i - 2 popc((neg_i ^ S) & nz_i),
// and sum_i s_i g_i is summed in int64 as in energy_block.  The row masks are
// stored word-major ([word][row]), so the 32 lanes of a warp, one row each,
// read one coalesced 128-byte line per word; a warp owns one replica and
// builds its spin mask in shared memory by ballots.
constexpr int kBitsWarps = 8;

__global__ void __launch_bounds__(kBitsWarps * 32)
k_energy_bits(const uint32_t* __restrict__ nzT, const uint32_t* __restrict__ negT,
              const int32_t* __restrict__ deg, const int32_t* __restrict__ h, int N, int Wd,
              int Npad, int R, int64_t sumJ, const int8_t* __restrict__ spins, int64_t* energy,
              int64_t* cut)
{
    extern __shared__ uint32_t smask[];   // [kBitsWarps][Wd]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kBitsWarps + warp;
    if (r >= R) return;                   // whole warp: no block-wide barrier below
    uint32_t* S = smask + (size_t)warp * Wd;
    const int8_t* s = spins + (size_t)r * N;
    for (int w = 0; w < Wd; ++w) {
        const int j = 32 * w + lane;
        const uint32_t b = __ballot_sync(0xffffffffu, j < N && s[j] < 0);
        if (lane == 0) S[w] = b;
    }
    __syncwarp();
    long long ordered = 0, field = 0;
    for (int i0 = 0; i0 < N; i0 += 32) {
        const int i = i0 + lane;
        int cnt = 0;
        for (int w = 0; w < Wd; ++w)
            cnt += __popc((negT[(size_t)w * Npad + i] ^ S[w]) & nzT[(size_t)w * Npad + i]);
        if (i < N) {
            const int si = ((S[i >> 5] >> (i & 31)) & 1u) ? -1 : 1;
            ordered += (long long)si * (long long)(deg[i] - 2 * cnt);
            if (h) field += (long long)h[i] * si;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ordered += __shfl_xor_sync(0xffffffffu, ordered, o);
        field += __shfl_xor_sync(0xffffffffu, field, o);
    }
    if (lane == 0) {
        if (energy) energy[r] = ordered / 2 + field;
        if (cut) cut[r] = (sumJ - ordered) / 4;
    }
}

// Ising energy for real-valued couplings and fields (Results Eq. (1)), exact up
// to one rounding of J and h onto a fixed-point grid.  The context's shift s
// makes max_i (sum_j |J_ij| + 2 |h_i|) 2^s <= 2^61; every J_ij and h_i is rounded
// to the nearest multiple of 2^-s (J~, h~: integers), and per replica
//   2^(s+1) E = sum_i s_i (2 h~_i + sum_{j != i} J~_ij s_j)
// is summed exactly: int64 row sums, a 128-bit total, one rounding to double at
// the end.  Integer sums do not depend on their order, so the result is the
// same under any schedule, and integer J, h give the int64 energy exactly.
// A warp holds 32 replicas (a lane each) and walks each row once: lane k loads
// entry k of a 32-entry slice, converts it and fetches the 32-replica sign mask
// of its column; the slice is then broadcast entry by entry.
constexpr int kFxWarps = 8;

__device__ __forceinline__ long long fx_round(float v, int s)
{
    const uint32_t u = __float_as_uint(v);
    const int e = (int)((u >> 23) & 0xffu);
    long long m = (long long)(u & 0x7fffffu);
    int ex = -149;                       // subnormal: m 2^-149
    if (e != 0) {
        m |= 0x800000;
        ex = e - 150;                    // v = m 2^(e - 150)
    }
    const int sh = ex + s;
    long long q;
    if (sh >= 0) q = m << sh;            // |v| 2^s <= 2^61: no overflow
    else if (sh > -40) q = (m + (1ll << (-sh - 1))) >> (-sh);   // nearest, ties away from 0
    else q = 0;
    return (u >> 31) ? -q : q;
}

// masks[g][j] bit r: spin j of replica 32 g + r is -1 (replicas past R: +1)
__global__ void __launch_bounds__(kThreads) k_spin_masks(const int8_t* __restrict__ spins, int R,
                                                         int N, uint32_t* __restrict__ masks)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, g = blockIdx.y;
    if (j >= N) return;
    uint32_t m = 0;
    for (int r = 0; r < 32 && g * 32 + r < R; ++r)
        m |= (spins[(size_t)(g * 32 + r) * N + j] < 0 ? 1u : 0u) << r;
    masks[(size_t)g * N + j] = m;
}

// Block (chunk c, replica group g): rows [c rows, +rows) of the 32 replicas of
// group g; part[c][32 g + lane] = sum over those rows of s_i (2 h~_i + g~_i).
__global__ void __launch_bounds__(kFxWarps * 32) k_energy_fx(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ val, const float* __restrict__ h, int N, int rows, int s,
    const uint32_t* __restrict__ masks, __int128* __restrict__ part, int Rp)
{
    const int c = blockIdx.x, g = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* mk = masks + (size_t)g * N;
    const int i0 = c * rows, i1 = min(N, i0 + rows);
    __int128 acc = 0;
    for (int i = i0 + warp; i < i1; i += kFxWarps) {
        const int b = row_ptr[i], e = row_ptr[i + 1];
        long long T = 0, A = 0;          // row sum, and its part over this lane's -1 spins
        for (int base = b; base < e; base += 32) {
            const int k = base + lane;
            long long q = 0;
            uint32_t m = 0;
            if (k < e) {
                q = fx_round(val[k], s);
                m = mk[col[k]];
            }
            T += q;
            const int cnt = min(32, e - base);
#pragma unroll 4
            for (int kk = 0; kk < cnt; ++kk) {
                const long long qk = __shfl_sync(0xffffffffu, q, kk);
                const uint32_t mkk = __shfl_sync(0xffffffffu, m, kk);
                if ((mkk >> lane) & 1u) A += qk;
            }
        }
        for (int o = 16; o > 0; o >>= 1) T += __shfl_xor_sync(0xffffffffu, T, o);
        const long long x = T - 2 * A + (h ? 2 * fx_round(h[i], s) : 0);
        acc += ((mk[i] >> lane) & 1u) ? -(__int128)x : (__int128)x;
    }
    __shared__ __int128 sh[kFxWarps][32];
    sh[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        __int128 t = 0;
        for (int w = 0; w < kFxWarps; ++w) t += sh[w][lane];
        part[(size_t)c * Rp + g * 32 + lane] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_energy_fx_final(const __int128* __restrict__ part,
                                                              int chunks, int Rp, int R, int s,
                                                              double* __restrict__ energy)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    __int128 t = 0;
    for (int c = 0; c < chunks; ++c) t += part[(size_t)c * Rp + r];
    const bool neg = t < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
    const double d = (double)(unsigned long long)(a >> 64) * 18446744073709551616.0 +
                     (double)(unsigned long long)a;
    energy[r] = ldexp(neg ? -d : d, -(s + 1));
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
    const int N = ctx->N;
    if (ctx->fx_shift < 0) {
        // the grid: the largest row bound B = sum_j |J_ij| + 2 |h_i| gets B 2^s <= 2^61
        double B = 0.0;
        for (int i = 0; i < N; ++i) {
            double b = ctx->has_h ? 2.0 * std::fabs((double)ctx->h[i]) : 0.0;
            for (int64_t k = ctx->row_ptr[i]; k < ctx->row_ptr[i + 1]; ++k)
                b += std::fabs((double)ctx->val[k]);
            B = std::max(B, b);
        }
        ctx->fx_shift = B > 0.0 ? std::min(200, (int)std::floor(61.0 - std::log2(B))) : 0;
        if (ctx->fx_shift < 0) return HQA_ERR_UNSUPPORTED;   // |J| sums beyond 2^61
    }
    const int s = ctx->fx_shift;
    const int G = (replicas + 31) / 32, Rp = G * 32;
    if (G > 65535) return HQA_ERR_TOO_LARGE;   // grid y
    // about four blocks per SM over (row chunk, replica group)
    const int want = std::max(1, 4 * ctx->sm_count / G);
    const int chunks = std::min(want, (N + kFxWarps - 1) / kFxWarps);
    const int rows = (N + chunks - 1) / chunks;
    const int nchunks = (N + rows - 1) / rows;
    const size_t mask_bytes = ((size_t)G * N * 4 + 255) & ~(size_t)255;
    const size_t bytes = mask_bytes + (size_t)nchunks * Rp * sizeof(__int128);
    hqa_status st = hqa_reserve(ctx, &ctx->d_efx, &ctx->efx_cap, bytes);
    if (st != HQA_OK) return st;
    hqa_capture_touch(ctx);
    uint32_t* masks = static_cast<uint32_t*>(ctx->d_efx);
    __int128* part = reinterpret_cast<__int128*>(static_cast<char*>(ctx->d_efx) + mask_bytes);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    k_spin_masks<<<dim3((N + kThreads - 1) / kThreads, G), kThreads, 0, cs>>>(spins, replicas, N,
                                                                             masks);
    k_energy_fx<<<dim3(nchunks, G), kFxWarps * 32, 0, cs>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val,
                                                           ctx->has_h ? ctx->d_h : nullptr, N,
                                                           rows, s, masks, part, Rp);
    k_energy_fx_final<<<(replicas + kThreads - 1) / kThreads, kThreads, 0, cs>>>(
        part, nchunks, Rp, replicas, s, energy);
    return hqa_capture_note(cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA);
}

// Word-major row masks of the couplings (k_energy_bits), built on first use.
static hqa_status energy_bits_setup(hqa_ctx* ctx)
{
    if (ctx->d_ebits) return HQA_OK;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    const int N = ctx->N, Wd = (N + 31) / 32, Npad = Wd * 32;
    std::vector<uint32_t> nz((size_t)Wd * Npad, 0u), neg((size_t)Wd * Npad, 0u);
    std::vector<int32_t> deg(N, 0);
    for (int i = 0; i < N; ++i)
        for (int64_t k = ctx->row_ptr[i]; k < ctx->row_ptr[i + 1]; ++k) {
            const int j = ctx->col[k];
            nz[(size_t)(j >> 5) * Npad + i] |= 1u << (j & 31);
            if (ctx->val[k] < 0.f) neg[(size_t)(j >> 5) * Npad + i] |= 1u << (j & 31);
            ++deg[i];
        }
    const size_t mb = nz.size() * sizeof(uint32_t);
    void* d = nullptr;
    HQA_CUDA_TRY(cudaMalloc(&d, 2 * mb + (size_t)N * sizeof(int32_t)));
    char* b = static_cast<char*>(d);
    if (cudaMemcpy(b, nz.data(), mb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b + mb, neg.data(), mb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b + 2 * mb, deg.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaFree(d);
        (void)cudaGetLastError();
        return HQA_ERR_CUDA;
    }
    ctx->d_ebits = d;
    ++ctx->generation;
    return HQA_OK;
}

// The bit-mask energy pays where rows hold at least as many couplings as mask
// words (dense instances); sparse rows keep the per-coupling gather.
static bool energy_bits_wanted(const hqa_ctx* ctx)
{
    const int Wd = (ctx->N + 31) / 32;
    return ctx->unit && ctx->nnz >= (int64_t)ctx->N * Wd;
}

hqa_status hqa_launch_energy(hqa_ctx* ctx, int32_t R, const int8_t* spins, int64_t* energy,
                             int64_t* cut, cudaStream_t st)
{
    return hqa_launch_energy_ex(ctx, R, spins, energy, cut, st, true);
}

hqa_status hqa_launch_energy_ex(hqa_ctx* ctx, int32_t R, const int8_t* spins, int64_t* energy,
                                int64_t* cut, cudaStream_t st, bool may_allocate)
{
    if (!ctx->integer) return HQA_ERR_UNSUPPORTED;
    if (R <= 0) return HQA_OK;
    // without permission to allocate, the bit masks are used only if already built
    if (energy_bits_wanted(ctx) && (may_allocate || ctx->d_ebits)) {
        hqa_status s = energy_bits_setup(ctx);
        if (s != HQA_OK) return s;
        const int N = ctx->N, Wd = (N + 31) / 32, Npad = Wd * 32;
        const size_t mb = (size_t)Wd * Npad * sizeof(uint32_t);
        const char* b = static_cast<const char*>(ctx->d_ebits);
        const size_t smem = (size_t)kBitsWarps * Wd * sizeof(uint32_t);
        if (smem > 48 * 1024) return HQA_ERR_TOO_LARGE;   // N <= 49152
        k_energy_bits<<<(R + kBitsWarps - 1) / kBitsWarps, kBitsWarps * 32, smem, st>>>(
            reinterpret_cast<const uint32_t*>(b), reinterpret_cast<const uint32_t*>(b + mb),
            reinterpret_cast<const int32_t*>(b + 2 * mb), ctx->has_h ? ctx->d_h_i32 : nullptr, N,
            Wd, Npad, R, ctx->sum_J_all, spins, energy, cut);
        return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
    }
    k_energy_csr<<<R, kThreads, 0, st>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val_i8,
                                         ctx->has_h ? ctx->d_h_i32 : nullptr, ctx->N,
                                         ctx->sum_J_all, spins, energy, cut);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}
