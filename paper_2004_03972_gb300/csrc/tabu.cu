// tabu.cu -- tabu search on the reduced problem (HQA section, Eqs. (6)-(7)),
// for ambivalent sets too large to enumerate: the role QBSolv's tabu search
// plays in the paper's HQA(TS1000) runs.  Deterministic single-flip search
// (the oracle states the same definition and is matched bit for bit):
//   f_a = h_a + sum_{j != a} J_aj s_j; flipping a changes E by d_a = -2 s_a f_a.
//   Iteration it = 1..iters: among ambivalent a that are not tabu
//   (until[a] < it) or would give a new best (E + d_a < E_best), flip the
//   smallest (d_a, a), even uphill; update its neighbours' fields; make it
//   tabu until it + tenure; a strictly lower E becomes the best assignment.
// One CTA per replica, one thread per ambivalent spin (n <= 1024): the
// choice is a block-wide minimum of 64-bit keys ((d_a + 2^31) << 32 | a),
// then one warp updates the winner's neighbours through a shared-memory map
// spin -> position in the ambivalent list.
#include "hqa_internal.cuh"

namespace {

constexpr int kTabuThreads = 1024;
constexpr int kTabuMaxN = 1024;

size_t tabu_smem(int N)
{
    return (((size_t)N * 2 + 15) & ~(size_t)15) + (size_t)kTabuMaxN * (4 + 4 + 4 + 1 + 1);
}

__global__ void __launch_bounds__(kTabuThreads, 1) k_sub_tabu(
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
    int8_t* s = reinterpret_cast<int8_t*>(until + kTabuMaxN);
    int8_t* bs = s + kTabuMaxN;
    __shared__ int cnt[kTabuThreads];
    __shared__ int s_n;
    __shared__ unsigned long long wmin[kTabuThreads / 32];
    __shared__ unsigned long long s_win;
    __shared__ long long s_rel, s_best;
    __shared__ int s_improved;

    const int r = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int8_t* sin = spins + (size_t)r * N;
    const uint8_t* fr = frozen + (size_t)r * N;
    int8_t* so = out + (size_t)r * N;

    // ambivalent list in ascending index: a contiguous chunk per thread, then a scan
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int lo = t * per, hi = min(N, lo + per);
    int c = 0;
    for (int i = lo; i < hi; ++i) c += fr[i] ? 0 : 1;
    cnt[t] = c;
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const int v = cnt[k];
            cnt[k] = acc;
            acc += v;
        }
        s_n = acc;
        s_rel = 0;
        s_best = 0;
    }
    __syncthreads();
    const int n = s_n;
    if (n > nmax || n > kTabuMaxN) {
        for (int i = t; i < N; i += blockDim.x) so[i] = sin[i];
        if (t == 0) atomicOr(status, HQA_DEV_BAD_SUBPROBLEM);
        return;
    }
    {
        int k = cnt[t];
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
    if (t < n) {
        const int a = amb[t];
        int g = h ? h[a] : 0;
        for (int k = row_ptr[a]; k < row_ptr[a + 1]; ++k)
            if (col[k] != a) g += (int)val[k] * (int)sin[col[k]];
        f[t] = g;
        s[t] = sin[a];
        bs[t] = sin[a];
        until[t] = 0;
    }
    __syncthreads();

    for (int it = 1; it <= iters; ++it) {
        unsigned long long key = ~0ull;
        if (t < n) {
            const int d = -2 * (int)s[t] * f[t];
            if (until[t] < it || s_rel + d < s_best)
                key = ((unsigned long long)((uint32_t)d ^ 0x80000000u) << 32) | (uint32_t)t;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, key, o);
            key = v < key ? v : key;
        }
        if (lane == 0) wmin[warp] = key;
        __syncthreads();
        if (warp == 0) {
            unsigned long long v = lane < (int)(blockDim.x >> 5) ? wmin[lane] : ~0ull;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
                v = u < v ? u : v;
            }
            if (lane == 0) s_win = v;
        }
        __syncthreads();
        const unsigned long long win = s_win;
        if (win == ~0ull) continue;   // every spin tabu and none aspirates (uniform)
        const int w = (int)(win & 0xffffffffull);
        const int d = (int)((uint32_t)(win >> 32) ^ 0x80000000u);
        if (t == w) {
            s[w] = (int8_t)-s[w];
            until[w] = it + tenure;
        }
        if (t == 0) s_rel += d;
        __syncthreads();
        if (warp == 0) {
            const int a = amb[w];
            const int sw = s[w];
            for (int k = row_ptr[a] + lane; k < row_ptr[a + 1]; k += 32) {
                const int j = col[k];
                const int p = j != a ? pos[j] : -1;
                if (p >= 0) f[p] += 2 * (int)val[k] * sw;   // each neighbour once per row
            }
            if (lane == 0) {
                s_improved = s_rel < s_best ? 1 : 0;
                if (s_improved) s_best = s_rel;
            }
        }
        __syncthreads();
        if (s_improved && t < n) bs[t] = s[t];
    }
    __syncthreads();
    for (int i = t; i < N; i += blockDim.x) so[i] = pos[i] >= 0 ? bs[pos[i]] : sin[i];
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
    hqa_capture_touch(ctx);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (hqa_smem_attr((const void*)k_sub_tabu, smem) != cudaSuccess) return HQA_ERR_CUDA;
    k_sub_tabu<<<replicas, kTabuThreads, smem, st>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val_i8,
                                                     ctx->has_h ? ctx->d_h_i32 : nullptr, ctx->N, n,
                                                     spins, frozen, iters, tenure, out_spins,
                                                     ctx->d_status);
    if (cudaGetLastError() != cudaSuccess) return HQA_ERR_CUDA;
    if (out_energy) return hqa_capture_note(hqa_launch_energy(ctx, replicas, out_spins, out_energy,
                                                              nullptr, st));
    return HQA_OK;
}
