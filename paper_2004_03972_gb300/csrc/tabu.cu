// tabu.cu -- tabu search on the reduced problem (HQA section, Eqs. (6)-(7)),
// for ambivalent sets too large to enumerate: the role QBSolv's tabu search
// plays in the paper's HQA(TS1000) runs.  Deterministic single-flip search
// (the oracle states the same definition and is matched bit for bit):
//   f_a = h_a + sum_{j != a} J_aj s_j; flipping a changes E by d_a = -2 s_a f_a.
//   Iteration it = 1..iters: among ambivalent a that are not tabu
//   (until[a] < it) or would give a new best (E + d_a < E_best), flip the
//   smallest (d_a, a), even uphill; update its neighbours' fields; make it
//   tabu until it + tenure; a strictly lower E becomes the best assignment.
// One CTA per replica; each of its 512 threads owns two positions q and
// q + 512 of the ascending ambivalent list (n <= 1024), so four CTAs share an
// SM.  Per flip: every thread forms the keys ((d_a + 2^31) << 32 | q << 1 |
// [s_a < 0]) of its positions; warps reduce them and every warp reduces the
// 16 warp minima itself, so all threads learn the winner, its energy change
// and its old spin (the bit below the position, which never decides a tie).
// The running and best energies are register copies kept identical in all
// threads.  The whole block then walks the winner's CSR row (unique,
// off-diagonal columns) and updates the neighbours' fields through a
// shared-memory map spin -> position: two barriers per flip.  When every
// |f_a| < 2^19 (the host bounds it by |h_a| + deg_a for unit couplings) a key
// fits 32 bits, ((d_a + 2^20) << 11 | q << 1 | [s_a < 0]), and both minima are
// one redux.sync each instead of five 64-bit shuffle rounds.
#include "hqa_internal.cuh"

namespace {

constexpr int kTabuThreads = 512;
constexpr int kTabuPer = 2;
constexpr int kTabuWarps = kTabuThreads / 32;
constexpr int kTabuMaxN = kTabuThreads * kTabuPer;

size_t tabu_smem(int N)
{
    // pos int16[N]; amb, f, until, rb, re int32[max n]; s, bs int8[max n]
    return (((size_t)N * 2 + 15) & ~(size_t)15) + (size_t)kTabuMaxN * (5 * 4 + 2);
}

// Keys of one candidate and of "no candidate": 64-bit, or 32-bit when narrow.
template <bool NARROW>
struct TabuKey;
template <>
struct TabuKey<false> {
    using T = unsigned long long;
    static constexpr T kNone = ~0ull;
    __device__ static T make(int d, int q, int sq)
    {
        return ((T)((uint32_t)d ^ 0x80000000u) << 32) | ((uint32_t)q << 1) | (sq < 0 ? 1u : 0u);
    }
    __device__ static T warp_min(T k)
    {
        for (int o = 16; o > 0; o >>= 1) {
            const T v = __shfl_xor_sync(0xffffffffu, k, o);
            k = v < k ? v : k;
        }
        return k;
    }
    __device__ static int delta(T k) { return (int)((uint32_t)(k >> 32) ^ 0x80000000u); }
    __device__ static uint32_t low(T k) { return (uint32_t)k; }
};
template <>
struct TabuKey<true> {
    using T = uint32_t;
    static constexpr T kNone = ~0u;
    __device__ static T make(int d, int q, int sq)
    {
        return ((uint32_t)(d + (1 << 20)) << 11) | ((uint32_t)q << 1) | (sq < 0 ? 1u : 0u);
    }
    __device__ static T warp_min(T k) { return __reduce_min_sync(0xffffffffu, k); }
    __device__ static int delta(T k) { return (int)(k >> 11) - (1 << 20); }
    __device__ static uint32_t low(T k) { return k & 0x7ffu; }
};

template <bool NARROW>
__global__ void __launch_bounds__(kTabuThreads, 4) k_sub_tabu(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const int8_t* __restrict__ val, const int32_t* __restrict__ h, int N, int nmax,
    const int8_t* __restrict__ spins, const uint8_t* __restrict__ frozen, int iters, int tenure,
    int8_t* __restrict__ out, uint32_t* status)
{
    extern __shared__ __align__(16) unsigned char sm[];
    int16_t* pos = reinterpret_cast<int16_t*>(sm);
    int32_t* amb = reinterpret_cast<int32_t*>(sm + (((size_t)N * 2 + 15) & ~(size_t)15));
    int32_t* f = amb + kTabuMaxN;
    int32_t* until = f + kTabuMaxN;
    int32_t* rb = until + kTabuMaxN;
    int32_t* re = rb + kTabuMaxN;
    int8_t* s = reinterpret_cast<int8_t*>(re + kTabuMaxN);
    int8_t* bs = s + kTabuMaxN;
    using K = TabuKey<NARROW>;
    using key_t = typename K::T;
    __shared__ int wsum[kTabuWarps];
    __shared__ key_t wmin[kTabuWarps];

    const int r = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int8_t* sin = spins + (size_t)r * N;
    const uint8_t* fr = frozen + (size_t)r * N;
    int8_t* so = out + (size_t)r * N;

    // ambivalent list in ascending index: a contiguous chunk per thread, then a
    // block-wide exclusive scan of the chunk counts (warp scans + warp totals)
    const int per = (N + kTabuThreads - 1) / kTabuThreads;
    const int lo = min(N, t * per), hi = min(N, lo + per);
    int c = 0;
    for (int i = lo; i < hi; ++i) c += fr[i] ? 0 : 1;
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int v = lane < kTabuWarps ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < kTabuWarps) wsum[lane] = v;
    }
    __syncthreads();
    const int n = wsum[kTabuWarps - 1];
    if (n > nmax || n > kTabuMaxN) {
        for (int i = t; i < N; i += kTabuThreads) so[i] = sin[i];
        if (t == 0) atomicOr(status, HQA_DEV_BAD_SUBPROBLEM);
        return;
    }
    {
        int k = (warp ? wsum[warp - 1] : 0) + x - c;
        for (int i = lo; i < hi; ++i) {
            if (fr[i]) {
                pos[i] = -1;
            } else {
                pos[i] = (int16_t)k;
                amb[k++] = i;
            }
        }
    }
    __syncthreads();
    // fields f_a = h_a + sum_j J_aj s_j: one warp per position, lanes across the row
    for (int q = warp; q < n; q += kTabuWarps) {
        const int a = amb[q];
        const int b = row_ptr[a], e = row_ptr[a + 1];
        int g = 0;
        for (int k = b + lane; k < e; k += 32) g += (int)val[k] * (int)sin[col[k]];
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) {
            f[q] = g + (h ? h[a] : 0);
            rb[q] = b;
            re[q] = e;
        }
    }
#pragma unroll
    for (int u = 0; u < kTabuPer; ++u) {
        const int q = t + u * kTabuThreads;
        if (q < n) {
            s[q] = sin[amb[q]];
            bs[q] = s[q];
            until[q] = 0;
        }
    }
    __syncthreads();

    long long rel = 0, best = 0;   // energies relative to the input assignment
    for (int it = 1; it <= iters; ++it) {
        // aspiration E + d < E_best as d < gap; |d| <= 2^22, so the clamp keeps the test exact
        const long long gl = best - rel;
        const int gap = gl < -(1ll << 31) + 1 ? INT_MIN + 1 : (int)gl;
        key_t key = K::kNone;
#pragma unroll
        for (int u = 0; u < kTabuPer; ++u) {
            const int q = t + u * kTabuThreads;
            if (q < n) {
                const int sq = s[q];
                const int d = -2 * sq * f[q];
                if (until[q] < it || d < gap) {
                    const key_t kq = K::make(d, q, sq);
                    key = kq < key ? kq : key;
                }
            }
        }
        key = K::warp_min(key);
        if (lane == 0) wmin[warp] = key;
        __syncthreads();
        const key_t win = K::warp_min(lane < kTabuWarps ? wmin[lane] : K::kNone);
        if (win != K::kNone) {   // uniform: every spin tabu and none aspirates skips the flip
            const uint32_t low = K::low(win);
            const int w = (int)(low >> 1);
            const int sw = (low & 1u) ? 1 : -1;   // the winner's new spin
            rel += K::delta(win);
            const bool improved = rel < best;
            if (improved) best = rel;
            if ((w & (kTabuThreads - 1)) == t) {
                s[w] = (int8_t)sw;
                until[w] = it + tenure;
            }
            for (int k = rb[w] + t; k < re[w]; k += kTabuThreads) {
                const int p = pos[col[k]];
                if (p >= 0) f[p] += 2 * (int)val[k] * sw;   // each neighbour once per row
            }
            if (improved) {
#pragma unroll
                for (int u = 0; u < kTabuPer; ++u) {
                    const int q = t + u * kTabuThreads;
                    if (q < n) bs[q] = s[q];
                }
            }
        }
        __syncthreads();
    }
    for (int i = t; i < N; i += kTabuThreads) so[i] = pos[i] >= 0 ? bs[pos[i]] : sin[i];
}

}  // namespace

extern "C" hqa_status hqa_solve_sub_tabu(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                                         const uint8_t* frozen, int32_t n, int32_t iters,
                                         int32_t tenure, int8_t* out_spins, int64_t* out_energy,
                                         void* stream)
{
    if (!ctx || replicas < 1 || !spins || !frozen || !out_spins) return HQA_ERR_INVALID_ARG;
    if (n < 0 || iters < 0 || tenure < 0 || ((uintptr_t)out_energy % 8)) return HQA_ERR_INVALID_ARG;
    if (iters > (1 << 30) || tenure > (1 << 30)) return HQA_ERR_INVALID_ARG;   // it + tenure < 2^31
    if (ctx->is_batch) return HQA_ERR_UNSUPPORTED;
    if (!ctx->integer || !ctx->unit) return HQA_ERR_UNSUPPORTED;
    if (n > kTabuMaxN) return HQA_ERR_TOO_LARGE;
    const size_t smem = tabu_smem(ctx->N);
    if (smem > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    // |f_a| <= |h_a| + deg_a (unit couplings); an integer context has |h| <= 2^20 and
    // N <= 2^16, so fields and energy changes stay far inside int32.  32-bit keys
    // need |f_a| < 2^19.
    int64_t fmax = 0;
    for (int i = 0; i < ctx->N; ++i) {
        const int64_t hb = ctx->has_h ? (int64_t)std::fabs((double)ctx->h[i]) : 0;
        fmax = std::max(fmax, hb + (ctx->row_ptr[i + 1] - ctx->row_ptr[i]));
    }
    const bool narrow = fmax < ((int64_t)1 << 19);
    hqa_capture_touch(ctx);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const void* fn = narrow ? (const void*)k_sub_tabu<true> : (const void*)k_sub_tabu<false>;
    if (hqa_smem_attr(fn, smem) != cudaSuccess) return HQA_ERR_CUDA;
    const int32_t* hp = ctx->has_h ? ctx->d_h_i32 : nullptr;
    if (narrow)
        k_sub_tabu<true><<<replicas, kTabuThreads, smem, st>>>(ctx->d_row_ptr, ctx->d_col,
                                                               ctx->d_val_i8, hp, ctx->N, n, spins,
                                                               frozen, iters, tenure, out_spins,
                                                               ctx->d_status);
    else
        k_sub_tabu<false><<<replicas, kTabuThreads, smem, st>>>(ctx->d_row_ptr, ctx->d_col,
                                                                ctx->d_val_i8, hp, ctx->N, n, spins,
                                                                frozen, iters, tenure, out_spins,
                                                                ctx->d_status);
    if (cudaGetLastError() != cudaSuccess) return HQA_ERR_CUDA;
    if (out_energy) return hqa_capture_note(hqa_launch_energy(ctx, replicas, out_spins, out_energy,
                                                              nullptr, st));
    return HQA_OK;
}
