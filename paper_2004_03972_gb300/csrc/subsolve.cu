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
//
// Packed path (when every |H'| of the replica fits in 16 bits): bits 0 and 1
// of x are not walked but carried as four 16-bit lanes in two registers, so
// one flip of a walked bit k updates four configurations with two packed
// adds (add.s16x2) and tracks their minimum with min.s16x2.  Relative to the
// lane with bits 0, 1 clear, a lane (b0, b1) changes by
// 4 s_k (J_k0 b0 + J_k1 b1) on top of the common -2 s_k (g_k + h_eff_k).
// Phase 1 finds every thread's minimum and the replica minimum; phase 2
// re-walks only the threads that reached the replica minimum and keeps the
// smallest x attaining it.  Replicas outside the 16-bit bound, or with
// fewer than 3 walked bits, take the scalar walk.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "hqa_internal.cuh"

namespace {

constexpr int kMaxN = 30;
constexpr int kPrepThreads = 256;
constexpr int kEnumThreads = 256;

struct SubPrep {
    int32_t n;          // ambivalent count, -1 if invalid
    int32_t packed;     // 1: the packed 16-bit walk solves this replica
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
    unsigned long long* keys, uint32_t* status, int allow_packed, int* emin)
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
            P->packed = 0;
            keys[r] = ~0ull;
            atomicOr(status, HQA_DEV_BAD_SUBPROBLEM);
        }
        return;
    }
    __shared__ int s_bound;
    if (threadIdx.x == 0) s_bound = 0;
    __syncthreads();
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
            const int hf = he + (h ? h[i] : 0);
            P->amb[a] = i;
            P->heff[a] = hf;
            P->nz[a] = nz;
            P->neg[a] = ng;
            // |H'| <= sum |h_eff| + sum over pairs |J|: each row adds |h_eff| + popc / 2
            atomicAdd(&s_bound, (hf < 0 ? -hf : hf) + (__popc(nz) + 1) / 2);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        P->n = n;
        P->packed = (allow_packed && n >= 3 && s_bound < 30000) ? 1 : 0;
        keys[r] = ~0ull;
        if (emin) emin[r] = 0x7fffffff;
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
    if (n < 0 || P->packed) return;
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

__device__ __forceinline__ uint32_t add16x2(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("add.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t min16x2(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("min.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// both 16-bit halves = the low 16 bits of v
__device__ __forceinline__ uint32_t dup16(int v) { return __byte_perm((uint32_t)v, 0u, 0x1010); }

__device__ __forceinline__ uint32_t pack16(int lo, int hi)
{
    return ((uint32_t)lo & 0xffffu) | ((uint32_t)hi << 16);
}

__device__ __forceinline__ int lo16(uint32_t v) { return (int)(int16_t)(v & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t v) { return (int)(int16_t)(v >> 16); }

// nonzero iff one of the two 16-bit halves of v is zero
__device__ __forceinline__ uint32_t has_zero16(uint32_t v)
{
    return (v - 0x00010001u) & ~v & 0x80008000u;
}

// Per-bit constants of the packed walk (bits k >= 2).
struct PackedBit {
    uint32_t nz, ng;
    int pc, he;
    uint32_t cA, cB;       // lane corrections 4 (J_k0 b0 + J_k1 b1) for s_k = +1
    uint32_t nA, nB;       // the same, negated lane by lane (s_k = -1)
};

// Energy of x (bits >= 2 set as in x, bits 0, 1 from `lane`) from scratch.
__device__ int sub_energy(const uint32_t* nz, const uint32_t* ng, const int* pc, const int* he,
                          int n, uint32_t x)
{
    int twice_pair = 0, lin = 0;
    for (int a = 0; a < n; ++a) {
        const int sa = ((x >> a) & 1u) ? -1 : 1;
        twice_pair += sa * (pc[a] - 2 * __popc((ng[a] ^ x) & nz[a]));
        lin += sa * he[a];
    }
    return twice_pair / 2 + lin;
}

// One thread's packed Gray walk over bits 2 .. LB-1 (bits >= LB fixed by the
// thread index).  PHASE 1: returns the minimum over its 4 * 2^(LB-2)
// configurations.  PHASE 2: returns the smallest x whose energy is `target`
// (0xffffffff if none).
template <int PHASE>
__device__ uint32_t packed_walk(const uint32_t* s_nz, const uint32_t* s_ng, const int* s_pc,
                                const int* s_he, const uint32_t* s_cA, const uint32_t* s_cB,
                                const uint32_t* s_nA, const uint32_t* s_nB, int n, int LB,
                                uint32_t x, int target, int* minE)
{
    // starting energies of the four lanes (bits 0, 1 of x)
    const int e0 = sub_energy(s_nz, s_ng, s_pc, s_he, n, x);
    const int e1 = sub_energy(s_nz, s_ng, s_pc, s_he, n, x | 1u);
    const int e2 = sub_energy(s_nz, s_ng, s_pc, s_he, n, x | 2u);
    const int e3 = sub_energy(s_nz, s_ng, s_pc, s_he, n, x | 3u);
    uint32_t A = pack16(e0, e1), B = pack16(e2, e3);
    uint32_t mA = A, mB = B;
    const uint32_t tgt = dup16(target);
    uint32_t best = 0xffffffffu;
    auto check = [&](uint32_t xx) {
        if (PHASE == 2 && (has_zero16(A ^ tgt) | has_zero16(B ^ tgt))) {
            if (lo16(A) == target) best = min(best, xx);
            if (hi16(A) == target) best = min(best, xx | 1u);
            if (lo16(B) == target) best = min(best, xx | 2u);
            if (hi16(B) == target) best = min(best, xx | 3u);
        }
    };
    check(x);
    // walked bits 2..5 in registers
    PackedBit rb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = 2 + j;
        rb[j].nz = s_nz[k];
        rb[j].ng = s_ng[k];
        rb[j].pc = s_pc[k];
        rb[j].he = s_he[k];
        rb[j].cA = s_cA[k];
        rb[j].cB = s_cB[k];
        rb[j].nA = s_nA[k];
        rb[j].nB = s_nB[k];
    }
    auto flip = [&](int k, uint32_t nz, uint32_t ng, int pc, int he, uint32_t cA, uint32_t cB,
                    uint32_t nA, uint32_t nB) {
        const bool neg = (x >> k) & 1u;
        const int g = pc - 2 * __popc((ng ^ x) & nz);
        const int D = neg ? 2 * (g + he) : -2 * (g + he);
        const uint32_t Dp = dup16(D);
        // s_k = -1: the lane corrections change sign (negated lane by lane on the
        // host side of the walk: a 32-bit negation would borrow across the halves)
        A = add16x2(A, add16x2(Dp, neg ? nA : cA));
        B = add16x2(B, add16x2(Dp, neg ? nB : cB));
        x ^= 1u << k;
        if (PHASE == 1) {
            mA = min16x2(mA, A);
            mB = min16x2(mB, B);
        } else {
            check(x);
        }
    };
    const uint32_t steps = 1u << (LB - 2);
    if (LB - 2 >= 4) {
        for (uint32_t tb = 0;; tb += 16) {
#pragma unroll
            for (int u = 1; u < 16; ++u) {
                const int j = __ffs(u) - 1;
                flip(2 + j, rb[j].nz, rb[j].ng, rb[j].pc, rb[j].he, rb[j].cA, rb[j].cB, rb[j].nA,
                     rb[j].nB);
            }
            const uint32_t t = tb + 16;
            if (t >= steps) break;
            const int k = 2 + __ffs(t) - 1;
            flip(k, s_nz[k], s_ng[k], s_pc[k], s_he[k], s_cA[k], s_cB[k], s_nA[k], s_nB[k]);
        }
    } else {
        for (uint32_t t = 1; t < steps; ++t) {
            const int k = 2 + __ffs(t) - 1;
            flip(k, s_nz[k], s_ng[k], s_pc[k], s_he[k], s_cA[k], s_cB[k], s_nA[k], s_nB[k]);
        }
    }
    if (PHASE == 1) {
        const uint32_t m = min16x2(mA, mB);
        *minE = min(lo16(m), hi16(m));
    }
    return best;
}

// Loads a replica's reduced problem into shared memory with the packed lane
// corrections.  Returns false if this replica does not take the packed path.
__device__ __forceinline__ bool load_packed(const SubPrep* P, uint32_t* s_nz, uint32_t* s_ng,
                                            int* s_pc, int* s_he, uint32_t* s_cA, uint32_t* s_cB,
                                            uint32_t* s_nA, uint32_t* s_nB)
{
    const int n = P->n;
    if (n < 0 || !P->packed) return false;
    for (int a = threadIdx.x; a < 32; a += blockDim.x) {
        const bool v = a < n;
        const uint32_t nz = v ? P->nz[a] : 0u, ng = v ? P->neg[a] : 0u;
        s_nz[a] = nz;
        s_ng[a] = ng;
        s_he[a] = v ? P->heff[a] : 0;
        s_pc[a] = __popc(nz);
        const int j0 = (nz & 1u) ? ((ng & 1u) ? -1 : 1) : 0;
        const int j1 = (nz & 2u) ? ((ng & 2u) ? -1 : 1) : 0;
        s_cA[a] = pack16(0, 4 * j0);
        s_cB[a] = pack16(4 * j1, 4 * (j0 + j1));
        s_nA[a] = pack16(0, -4 * j0);
        s_nB[a] = pack16(-4 * j1, -4 * (j0 + j1));
    }
    return true;
}

// Phase 1: every thread's minimum (tmin) and the replica minimum (emin).
__global__ void __launch_bounds__(kEnumThreads) k_sub_enum16_min(const SubPrep* __restrict__ prep,
                                                                 int LBreq, int16_t* tmin, int* emin)
{
    const int r = blockIdx.y;
    __shared__ uint32_t s_nz[32], s_ng[32], s_cA[32], s_cB[32], s_nA[32], s_nB[32];
    __shared__ int s_he[32], s_pc[32];
    const SubPrep* P = prep + r;
    if (!load_packed(P, s_nz, s_ng, s_pc, s_he, s_cA, s_cB, s_nA, s_nB)) return;
    __syncthreads();
    const int n = P->n;
    const int LB = LBreq < n ? LBreq : n;
    const int HB = n - LB;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    int m = 0x7fffffff;
    if (LB >= 3 && tid < (1u << HB)) {
        packed_walk<1>(s_nz, s_ng, s_pc, s_he, s_cA, s_cB, s_nA, s_nB, n, LB, tid << LB, 0, &m);
        tmin[(size_t)r * gridDim.x * blockDim.x + tid] = (int16_t)m;
    }
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m != 0x7fffffff) atomicMin(emin + r, m);
}

// Phase 2: the threads that reached the replica minimum find its smallest x.
// A warp walks each of its candidates' ranges together: lane l takes the
// sub-range whose next five bits equal l, so a candidate costs 1/32 of its
// phase-1 walk; the smallest x attaining the minimum wins by atomicMin.
__global__ void __launch_bounds__(kEnumThreads) k_sub_enum16_arg(const SubPrep* __restrict__ prep,
                                                                 int LBreq, const int16_t* tmin,
                                                                 const int* emin,
                                                                 unsigned long long* keys)
{
    const int r = blockIdx.y;
    __shared__ uint32_t s_nz[32], s_ng[32], s_cA[32], s_cB[32], s_nA[32], s_nB[32];
    __shared__ int s_he[32], s_pc[32];
    const SubPrep* P = prep + r;
    if (!load_packed(P, s_nz, s_ng, s_pc, s_he, s_cA, s_cB, s_nA, s_nB)) return;
    __syncthreads();
    const int n = P->n;
    const int LB = LBreq < n ? LBreq : n;
    const int HB = n - LB;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    const int target = emin[r];
    if (LB < 3) return;
    const bool cand = tid < (1u << HB) &&
                      (int)tmin[(size_t)r * gridDim.x * blockDim.x + tid] == target;
    const unsigned long long hi = (unsigned long long)((uint32_t)target ^ 0x80000000u) << 32;
    if (LB < 8) {   // too few bits to share: each candidate walks its own range
        if (!cand) return;
        const uint32_t bx = packed_walk<2>(s_nz, s_ng, s_pc, s_he, s_cA, s_cB, s_nA, s_nB, n, LB,
                                           tid << LB, target, nullptr);
        if (bx != 0xffffffffu) atomicMin(keys + r, hi | bx);
        return;
    }
    const int SB = LB - 5;
    for (unsigned bal = __ballot_sync(0xffffffffu, cand); bal; bal &= bal - 1) {
        const uint32_t ct = (tid & ~31u) | (uint32_t)(__ffs(bal) - 1);   // the candidate
        const uint32_t bx = packed_walk<2>(s_nz, s_ng, s_pc, s_he, s_cA, s_cB, s_nA, s_nB, n, SB,
                                           (ct << LB) | (lane << SB), target, nullptr);
        const uint32_t m = __reduce_min_sync(0xffffffffu, bx);
        if (lane == 0 && m != 0xffffffffu) atomicMin(keys + r, hi | m);
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
    // at least 3 walked bits: the packed walk carries bits 0, 1 as lanes
    const int LB = std::max(pick_lb(R, n, ctx->sm_count), std::min(3, n));
    const int HB = n - LB;
    const uint32_t per = 1u << HB;
    const dim3 grid((per + kEnumThreads - 1) / kEnumThreads, R);
    // workspace: prep records | keys (64-bit atomics) | replica minima | thread minima,
    // each part on a 256-byte boundary
    const auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t keys_off = up((size_t)R * sizeof(SubPrep));
    const size_t emin_off = keys_off + up((size_t)R * sizeof(unsigned long long));
    const size_t tmin_off = emin_off + up((size_t)R * sizeof(int));
    const size_t need = tmin_off + (size_t)R * grid.x * kEnumThreads * sizeof(int16_t);
    hqa_status s = hqa_reserve(ctx, &ctx->d_sub, &ctx->sub_cap, need);
    if (s != HQA_OK) return s;
    char* w = static_cast<char*>(ctx->d_sub);
    SubPrep* prep = reinterpret_cast<SubPrep*>(w);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(w + keys_off);
    int* emin = reinterpret_cast<int*>(w + emin_off);
    int16_t* tmin = reinterpret_cast<int16_t*>(w + tmin_off);
    k_sub_prep<<<R, kPrepThreads, 0, st>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val_i8,
                                           ctx->has_h ? ctx->d_h_i32 : nullptr, ctx->N, n, spins,
                                           frozen, prep, keys, ctx->d_status, 1, emin);
    k_sub_enum16_min<<<grid, kEnumThreads, 0, st>>>(prep, LB, tmin, emin);
    k_sub_enum16_arg<<<grid, kEnumThreads, 0, st>>>(prep, LB, tmin, emin, keys);
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
// preparation, the scalar Gray-code walk and the assembly of hqa_solve_sub
// (plus the energy kernel when asked), but not its packed 16-bit walk: that
// walk's per-thread minima grow with the enumeration and do not fit a fixed
// array, so every replica takes the scalar walk, which is slower but reaches
// the same (H', x) minimum.  Its scratch (the per-replica reduced-problem
// records and the 64-bit argmin keys) lives in the file-scope array below,
// which every GPU that loads the library holds until the process exits.  The records and keys of each replica are rewritten by
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

static hqa_status solve_sub_noalloc_impl(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                                         const uint8_t* frozen, int32_t n, int8_t* out_spins,
                                         int64_t* out_energy, void* stream)
{
    // the checks of hqa_solve_sub, in its order, then the two of this variant
    if (ctx && ctx->is_batch) return HQA_ERR_UNSUPPORTED;  // a batch has no coupling arrays of its own
    if (!ctx || replicas < 1 || !spins || !frozen || !out_spins) return HQA_ERR_INVALID_ARG;
    if (n < 0 || (out_energy && ((uintptr_t)out_energy % 8) != 0)) return HQA_ERR_INVALID_ARG;
    if (!ctx->integer || !ctx->unit) return HQA_ERR_UNSUPPORTED;
    if (n > kMaxN) return HQA_ERR_TOO_LARGE;
    if (replicas > kNoAllocMaxReplicas) return HQA_ERR_TOO_LARGE;  // scratch holds 2048 replicas
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return HQA_ERR_CUDA;
    }
    if (dev != ctx->device) return HQA_ERR_INVALID_ARG;  // the scratch address is per device
    unsigned char* base = nullptr;
    hqa_status s = sub_scratch_address(dev, &base);
    if (s != HQA_OK) return s;
    SubPrep* prep = reinterpret_cast<SubPrep*>(base);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + kNoAllocKeysOff);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t R = replicas;
    k_sub_prep<<<R, kPrepThreads, 0, st>>>(ctx->d_row_ptr, ctx->d_col, ctx->d_val_i8,
                                           ctx->has_h ? ctx->d_h_i32 : nullptr, ctx->N, n, spins,
                                           frozen, prep, keys, ctx->d_status, 0, nullptr);
    const int LB = pick_lb(R, n, ctx->sm_count);
    const uint32_t per = 1u << (n - LB);
    const dim3 grid((per + kEnumThreads - 1) / kEnumThreads, R);
    k_sub_enum<<<grid, kEnumThreads, 0, st>>>(prep, LB, keys);
    k_sub_assemble<<<R, 256, 0, st>>>(prep, keys, ctx->N, spins, out_spins);
    if (cudaGetLastError() != cudaSuccess) return HQA_ERR_CUDA;
    if (out_energy) return hqa_launch_energy_ex(ctx, R, out_spins, out_energy, nullptr, st, false);
    return HQA_OK;
}

extern "C" hqa_status hqa_solve_sub_noalloc(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                                            const uint8_t* frozen, int32_t n, int8_t* out_spins,
                                            int64_t* out_energy, void* stream)
{
    hqa_capture_touch(ctx);
    return hqa_capture_note(
        solve_sub_noalloc_impl(ctx, replicas, spins, frozen, n, out_spins, out_energy, stream));
}
