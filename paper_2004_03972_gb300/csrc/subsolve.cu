// subsolve.cu -- exact solution of the reduced Ising problem on the
// ambivalent spins (HQA section, Eqs. (6)-(7)) by Gray-code enumeration.
//
// Per replica, with the ambivalent spins a_0 < a_1 < ... < a_{n-1}:
//   h_eff_a = h_a + sum_{k frozen} J_ak s_k
//   H'(x)   = sum_{a<b} J_ab s_a s_b + sum_a h_eff_a s_a,  s_a = -1 iff bit a of x
// Couplings are in {-1, 0, +1}, so row a of J_eff is two bit masks over the
// ambivalent set: nz_a (J_ab != 0) and neg_a (J_ab < 0), and
//   g_a(x) = sum_b J_ab s_b = popc(nz_a) - 2 popc((neg_a ^ x) & nz_a).
// Flipping bit k changes H' by -2 s_k (g_k + h_eff_k), an O(1) update.  Each
// thread fixes the high n - LB bits of x and walks the low LB bits in Gray
// order (step t flips bit ctz(t)); the best (H', x) pair, ties to the
// smallest x, is reduced by warp shuffles and one 64-bit atomicMin per CTA
// on the key ((H' + 2^31) << 32 | x).
#include <atomic>
#include <mutex>

#include "hqa_internal.cuh"

namespace {

constexpr int kMaxN = 30;
constexpr int kPrepThreads = 256;
constexpr int kEnumThreads = 256;

struct SubPrep {
    int32_t n;          // ambivalent count, -1 if invalid
    int32_t amb[32];    // spin index of a_k
    int32_t heff[32];
    uint32_t nz[32];
    uint32_t neg[32];
};

// One CTA per replica: ambivalent list (ascending), h_eff and bit masks.
__global__ void __launch_bounds__(kPrepThreads) k_sub_prep(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const int8_t* __restrict__ val, const int32_t* __restrict__ h, int N, int nmax,
    const int8_t* __restrict__ spins, const uint8_t* __restrict__ frozen, SubPrep* prep,
    unsigned long long* keys, uint32_t* status)
{
    const int r = blockIdx.x;
    const int8_t* s = spins + (size_t)r * N;
    const uint8_t* f = frozen + (size_t)r * N;
    __shared__ int cnt[kPrepThreads];
    __shared__ int s_amb[32];
    __shared__ int s_n;
    // contiguous chunk per thread keeps the list ascending after the scan
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(N, lo + per);
    int c = 0;
    for (int i = lo; i < hi; ++i) c += f[i] ? 0 : 1;
    cnt[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int v = cnt[t];
            cnt[t] = acc;
            acc += v;
        }
        s_n = acc;
    }
    __syncthreads();
    const int n = s_n;
    const bool ok = n <= nmax && n <= kMaxN;
    if (ok) {
        int k = cnt[threadIdx.x];
        for (int i = lo; i < hi; ++i)
            if (!f[i]) s_amb[k++] = i;
    }
    __syncthreads();
    SubPrep* P = prep + r;
    if (!ok) {
        if (threadIdx.x == 0) {
            P->n = -1;
            keys[r] = ~0ull;
            atomicOr(status, HQA_DEV_BAD_SUBPROBLEM);
        }
        return;
    }
    // one warp per ambivalent spin
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = warp; a < n; a += nw) {
        const int i = s_amb[a];
        int he = 0;
        uint32_t nz = 0, ng = 0;
        for (int k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) {
            const int j = col[k];
            const int w = val[k];
            if (f[j]) {
                he += w * s[j];
            } else {
                int b = 0;
                while (b < n && s_amb[b] != j) ++b;  // j is ambivalent, so it is in the list
                if (b < n) {
                    if (w != 0) nz |= 1u << b;
                    if (w < 0) ng |= 1u << b;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            he += __shfl_xor_sync(0xffffffffu, he, o);
            nz |= __shfl_xor_sync(0xffffffffu, nz, o);
            ng |= __shfl_xor_sync(0xffffffffu, ng, o);
        }
        if (lane == 0) {
            P->amb[a] = i;
            P->heff[a] = he + (h ? h[i] : 0);
            P->nz[a] = nz;
            P->neg[a] = ng;
        }
    }
    if (threadIdx.x == 0) {
        P->n = n;
        keys[r] = ~0ull;
    }
}

__device__ __forceinline__ int gfield(uint32_t nz, uint32_t ng, int pc, uint32_t x)
{
    return pc - 2 * __popc((ng ^ x) & nz);
}

// grid (blocks per replica, R); thread index within the replica = high bits.
__global__ void __launch_bounds__(kEnumThreads) k_sub_enum(const SubPrep* __restrict__ prep,
                                                           int LBreq, unsigned long long* keys)
{
    const int r = blockIdx.y;
    __shared__ uint32_t s_nz[32], s_ng[32];
    __shared__ int s_he[32], s_pc[32];
    __shared__ unsigned long long s_best[kEnumThreads / 32];
    const SubPrep* P = prep + r;
    const int n = P->n;
    if (n < 0) return;
    for (int a = threadIdx.x; a < 32; a += blockDim.x) {
        const bool v = a < n;
        s_nz[a] = v ? P->nz[a] : 0u;
        s_ng[a] = v ? P->neg[a] : 0u;
        s_he[a] = v ? P->heff[a] : 0;
        s_pc[a] = v ? __popc(P->nz[a]) : 0;
    }
    __syncthreads();
    const int LB = LBreq < n ? LBreq : n;
    const int HB = n - LB;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long best = ~0ull;
    if (tid < (1u << HB)) {
        uint32_t x = tid << LB;
        // energy of the starting configuration
        int twice_pair = 0, lin = 0;
        for (int a = 0; a < n; ++a) {
            const int sa = ((x >> a) & 1u) ? -1 : 1;
            twice_pair += sa * gfield(s_nz[a], s_ng[a], s_pc[a], x);
            lin += sa * s_he[a];
        }
        int E = twice_pair / 2 + lin;
        int bE = E;
        uint32_t bx = x;
        // registers for the four lowest bits
        uint32_t rnz[4], rng[4];
        int rhe[4], rpc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            rnz[k] = s_nz[k];
            rng[k] = s_ng[k];
            rhe[k] = s_he[k];
            rpc[k] = s_pc[k];
        }
        auto flip = [&](int k, uint32_t nz, uint32_t ng, int pc, int he) {
            const int sk = ((x >> k) & 1u) ? -1 : 1;
            E -= 2 * sk * (gfield(nz, ng, pc, x) + he);
            x ^= 1u << k;
            if (E < bE || (E == bE && x < bx)) {
                bE = E;
                bx = x;
            }
        };
        const uint32_t steps = 1u << LB;
        if (LB >= 4) {
            for (uint32_t tb = 0;; tb += 16) {
#pragma unroll
                for (int u = 1; u < 16; ++u) {
                    const int k = __ffs(u) - 1;
                    flip(k, rnz[k], rng[k], rpc[k], rhe[k]);
                }
                const uint32_t t = tb + 16;
                if (t >= steps) break;
                const int k = __ffs(t) - 1;
                flip(k, s_nz[k], s_ng[k], s_pc[k], s_he[k]);
            }
        } else {
            for (uint32_t t = 1; t < steps; ++t) {
                const int k = __ffs(t) - 1;
                flip(k, s_nz[k], s_ng[k], s_pc[k], s_he[k]);
            }
        }
        best = ((unsigned long long)((uint32_t)bE ^ 0x80000000u) << 32) | bx;  // signed -> unsigned order
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v < best ? v : best;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_best[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = ~0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = s_best[w] < b ? s_best[w] : b;
        if (b != ~0ull) atomicMin(keys + r, b);
    }
}

// Writes the assembled configuration.
__global__ void k_sub_assemble(const SubPrep* __restrict__ prep,
                               const unsigned long long* __restrict__ keys, int N,
                               const int8_t* __restrict__ spins, int8_t* out)
{
    const int r = blockIdx.x;
    const SubPrep* P = prep + r;
    const int n = P->n;
    const uint32_t x = (uint32_t)(keys[r] & 0xffffffffull);
    for (int i = threadIdx.x; i < N; i += blockDim.x) out[(size_t)r * N + i] = spins[(size_t)r * N + i];
    __syncthreads();
    if (n > 0)
        for (int a = threadIdx.x; a < n; a += blockDim.x)
            out[(size_t)r * N + P->amb[a]] = ((x >> a) & 1u) ? -1 : 1;
}

}  // namespace

static int pick_lb(int32_t R, int n, int sm_count)
{
    // aim at ~2 waves of full occupancy: threads per replica ~ 2 * SMs * 2048 / R
    const double want = 2.0 * sm_count * 2048.0 / (double)R;
    int hb = 0;
    while (hb < n && (double)(1u << (hb + 1)) <= want) ++hb;
    return n - hb;
}

hqa_status hqa_launch_subsolve(hqa_ctx* ctx, int32_t R, const int8_t* spins,
                               const uint8_t* frozen, int32_t n, int8_t* out_spins,
                               int64_t* out_energy, cudaStream_t st)
{
    if (!ctx->integer || !ctx->unit) return HQA_ERR_UNSUPPORTED;
    if (n < 0 || n > kMaxN) return HQA_ERR_TOO_LARGE;
    if (R <= 0) return HQA_OK;
    // keys (64-bit atomics) start on a 256-byte boundary after the prep records
    const size_t keys_off = ((size_t)R * sizeof(SubPrep) + 255) & ~(size_t)255;
    const size_t need = keys_off + (size_t)R * sizeof(unsigned long long);
    hqa_status s = hqa_reserve(ctx, &ctx->d_sub, &ctx->sub_cap, need);
    if (s != HQA_OK) return s;
    SubPrep* prep = static_cast<SubPrep*>(ctx->d_sub);
    unsigned long long* keys =
        reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->d_sub) + keys_off);
    k_sub_prep<<<R, kPrepThreads, 0, st>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val_i8,
                                           ctx->has_h ? ctx->d_h_i32 : nullptr, ctx->N, n, spins,
                                           frozen, prep, keys, ctx->d_status);
    const int LB = pick_lb(R, n, ctx->sm_count);
    const int HB = n - LB;
    const uint32_t per = 1u << HB;
    const dim3 grid((per + kEnumThreads - 1) / kEnumThreads, R);
    k_sub_enum<<<grid, kEnumThreads, 0, st>>>(prep, LB, keys);
    k_sub_assemble<<<R, 256, 0, st>>>(prep, keys, ctx->N, spins, out_spins);
    if (cudaGetLastError() != cudaSuccess) return HQA_ERR_CUDA;
    if (out_energy) return hqa_launch_energy(ctx, R, out_spins, out_energy, nullptr, st);
    return HQA_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the sub-solve.
//
// Some callers cannot let the library call cudaMalloc: processes whose device
// memory is reserved up front by another allocator or arena (nothing is left
// to hand out), and latency-sensitive callers for whom cudaMalloc's implicit
// device-wide synchronisation is not acceptable.  This entry point runs the
// same three kernels as hqa_solve_sub, but its scratch (the per-replica
// reduced-problem records and the 64-bit argmin keys) lives in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.  The records and keys of each replica are rewritten by
// k_sub_prep before they are read, so stale contents from the previous call
// are never used.  All calls share the one array: calls whose kernels
// overlap on the GPU (e.g. on two streams) race and must be serialised by
// the caller.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoAllocMaxReplicas = 2048;
constexpr size_t kNoAllocKeysOff =
    ((size_t)kNoAllocMaxReplicas * sizeof(SubPrep) + 255) & ~(size_t)255;
constexpr size_t kNoAllocBytes = kNoAllocKeysOff + (size_t)kNoAllocMaxReplicas * 8;
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_sub_scratch[kNoAllocBytes];

// Device address of g_sub_scratch per device ordinal.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress once per device (with that device current).
static std::atomic<unsigned char*> g_sub_scratch_dev[kMaxDevices];
static std::mutex g_sub_scratch_mu;

static hqa_status sub_scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return HQA_ERR_UNSUPPORTED;
    unsigned char* p = g_sub_scratch_dev[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lk(g_sub_scratch_mu);
        p = g_sub_scratch_dev[dev].load(std::memory_order_relaxed);
        if (!p) {
            void* a = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&a, g_sub_scratch);
            if (e != cudaSuccess || !a) {
                (void)cudaGetLastError();
                return HQA_ERR_CUDA;
            }
            p = static_cast<unsigned char*>(a);
            g_sub_scratch_dev[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return HQA_OK;
}

extern "C" hqa_status hqa_solve_sub_noalloc(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                                            const uint8_t* frozen, int32_t n, int8_t* out_spins,
                                            int64_t* out_energy, void* stream)
{
    if (!ctx || replicas < 1 || !spins || !frozen || !out_spins || n < 0) return HQA_ERR_INVALID_ARG;
    if (ctx->is_batch) return HQA_ERR_UNSUPPORTED;  // a batch has no coupling arrays of its own
    if (out_energy && ((uintptr_t)out_energy % 8) != 0) return HQA_ERR_INVALID_ARG;
    if (replicas > kNoAllocMaxReplicas) return HQA_ERR_TOO_LARGE;  // scratch holds 2048 replicas
    if (!ctx->integer || !ctx->unit) return HQA_ERR_UNSUPPORTED;
    if (n > kMaxN) return HQA_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return HQA_ERR_CUDA;
    }
    if (dev != ctx->device) return HQA_ERR_INVALID_ARG;  // the scratch address is per device
    hqa_capture_touch(ctx);
    unsigned char* base = nullptr;
    hqa_status s = sub_scratch_address(dev, &base);
    if (s != HQA_OK) return s;
    SubPrep* prep = reinterpret_cast<SubPrep*>(base);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + kNoAllocKeysOff);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t R = replicas;
    k_sub_prep<<<R, kPrepThreads, 0, st>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val_i8,
                                           ctx->has_h ? ctx->d_h_i32 : nullptr, ctx->N, n, spins,
                                           frozen, prep, keys, ctx->d_status);
    const int LB = pick_lb(R, n, ctx->sm_count);
    const uint32_t per = 1u << (n - LB);
    const dim3 grid((per + kEnumThreads - 1) / kEnumThreads, R);
    k_sub_enum<<<grid, kEnumThreads, 0, st>>>(prep, LB, keys);
    k_sub_assemble<<<R, 256, 0, st>>>(prep, keys, ctx->N, spins, out_spins);
    if (cudaGetLastError() != cudaSuccess) return HQA_ERR_CUDA;
    if (out_energy) return hqa_launch_energy(ctx, R, out_spins, out_energy, nullptr, st);
    return HQA_OK;
}
