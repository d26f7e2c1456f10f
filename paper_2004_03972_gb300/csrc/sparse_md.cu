// sparse_md.cu -- resident sparse HQA-MD kernel (local field + leapfrog).
//
// One CTA owns RB replicas of one instance for the whole trajectory.  The
// flux operand phi of those replicas lives in shared memory, replica-minor
// ([row][RB]), double-buffered across steps, so every step of Methods'
// leapfrog runs on chip:
//   L_i  = sum_{j != i} J_ij phi_j + 2 h_i |phi_i|          (local field)
//   p_i <- p_i - c_j h [alpha M phi_i^(M-1) + beta L_i]     (kick)
//   phi_i <- phi_i + h alpha' p_i                            (drift)
//   w_i <- w_i + phi_i   during the last W steps             (window sum, Eq. (5))
// with one __syncthreads() per step.  Couplings must be -1, 0 or +1: every
// row's neighbours are split into a "+" and a "-" list, so the field is a
// sum of gathered phi values minus another, without multiplies.
//
// A warp evaluates a tuple of G = 32 / RB rows at once, lane = (g, r): lane
// g*RB + r reads phi[neighbour][r].  Each position of a tuple's list is one
// 32-lane shared-memory load of G rows x RB consecutive replicas; the host
// orders neighbours so that the G rows read at one position sit in distinct
// bank groups (row j occupies banks (j*RB) mod 32 .. +RB-1), which makes the
// load a single wavefront.  Neighbour byte offsets are streamed from global
// memory (L1/L2 resident) as one uint4 (4 positions) per lane.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "hqa_internal.cuh"

namespace {

constexpr int kMaxThreads = 1024;

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t counter)
{
    // SplitMix64 (Steele, Lea, Flood 2014): output number counter+1 of the stream.
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void sts_f32(uint32_t addr, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

__device__ __forceinline__ float lds_bf16(uint32_t addr)
{
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return __uint_as_float(((uint32_t)v) << 16);
}

__device__ __forceinline__ void sts_bf16(uint32_t addr, float v)
{
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    unsigned short u = *reinterpret_cast<unsigned short*>(&b);
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"(u));
}

template <bool BF16>
__device__ __forceinline__ float ld_op(uint32_t addr)
{
    if constexpr (BF16) return lds_bf16(addr);
    else return lds_f32(addr);
}

// Sum over one tuple's neighbour lists for this lane: (+ section) - (- section).
template <int RB, bool BF16>
__device__ __forceinline__ float tuple_field(const uint4* __restrict__ e, int npos, int nneg,
                                             uint32_t base)
{
    constexpr int G = 32 / RB;
    float accp = 0.f, accn = 0.f;
    int c = 0;
#pragma unroll 2
    for (; c < npos; ++c) {
        const uint4 q = __ldg(e + (size_t)c * G);
        accp += (ld_op<BF16>(base + q.x) + ld_op<BF16>(base + q.y)) +
                (ld_op<BF16>(base + q.z) + ld_op<BF16>(base + q.w));
    }
    const int cend = npos + nneg;
#pragma unroll 2
    for (; c < cend; ++c) {
        const uint4 q = __ldg(e + (size_t)c * G);
        accn += (ld_op<BF16>(base + q.x) + ld_op<BF16>(base + q.y)) +
                (ld_op<BF16>(base + q.z) + ld_op<BF16>(base + q.w));
    }
    return accp - accn;
}

struct MDArgs {
    const uint4* entries;
    const int4* tuples;
    const int* tuple_rows;
    const StepCoef* sched;
    const float* h;        // null when h = 0
    const float* phi0;     // HQA_INIT_GIVEN
    const float* p0;       // HQA_INIT_GIVEN
    float* phi_out;
    float* p_out;
    float* phibar_out;
    float* gstate;         // p/w state in global memory when it does not fit on chip
    size_t gstride;        // floats per CTA slice of gstate (fixed across a batch)
    uint32_t* status;
    uint64_t seed;
    int64_t S;
    int32_t W;
    int32_t N, Npad, T, R;
    int32_t M;
    int32_t init;
    int32_t state_in_smem;
};

// Shared-memory layout (bytes), per CTA:
//   op[2]   : 2 buffers of Npad * RB operand elements (FP32 or BF16)
//   master  : N * RB FP32 (BF16 operand only: the FP32 flux)
//   p, w    : N * RB FP32 each (when state_in_smem)
// One replica block (replicas blk*RB .. +RB-1) of one instance, whole
// trajectory.  Called by the single-instance kernel (blk = blockIdx.x) and by
// the persistent batch kernel (blk from its work queue); `gslot` selects the
// CTA's slice of the global p/w state when it does not fit on chip.
template <int RB, bool BF16>
__device__ __forceinline__ void md_block(const MDArgs& a, int blk, int gslot)
{
    constexpr int G = 32 / RB;
    constexpr int ES = BF16 ? 2 : 4;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t buf_bytes = (uint32_t)a.Npad * RB * ES;
    const uint32_t op_bytes = ((2u * buf_bytes) + 15u) & ~15u;
    const uint32_t master = s0 + op_bytes;  // FP32 [N][RB] (BF16 only)
    const uint32_t state_s = master + (BF16 ? (uint32_t)a.N * RB * 4u : 0u);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int g = lane / RB, r = lane % RB;
    const int rep0 = blk * RB;
    const int NRB = a.N * RB;

    // p and w: shared (u32 addresses) or global (per-CTA slice), [row][RB]
    float* gp = a.gstate ? a.gstate + (size_t)gslot * a.gstride : nullptr;
    float* gw = gp ? gp + NRB : nullptr;
    const uint32_t sp = state_s, sw = state_s + (uint32_t)NRB * 4u;

    // ---- initial state ----
    for (uint32_t o = threadIdx.x * 4u; o < op_bytes; o += blockDim.x * 4u) sts_f32(s0 + o, 0.f);
    __syncthreads();
    for (int idx = threadIdx.x; idx < NRB; idx += blockDim.x) {
        const int row = idx / RB, rr = idx % RB, rep = rep0 + rr;
        float phi = 0.f, p = 0.f;
        if (rep < a.R) {
            const uint64_t c = ((uint64_t)rep << 32) | (uint64_t)row;
            if (a.init == HQA_INIT_GIVEN) {
                phi = a.phi0[(size_t)rep * a.N + row];
                p = a.p0[(size_t)rep * a.N + row];
            } else {
                p = (splitmix64_at(a.seed, c) >> 63) ? -1.f : 1.f;
                if (a.init == HQA_INIT_RANDOM_FLUX) {
                    const uint64_t z = splitmix64_at(a.seed, c | (1ull << 62));
                    phi = (float)((int64_t)(z >> 40) - (1 << 23)) * 0x1p-26f;
                }
            }
        }
        const uint32_t e = (uint32_t)idx;
        if constexpr (BF16) {
            sts_f32(master + e * 4u, phi);
            sts_bf16(s0 + e * 2u, phi);
        } else {
            sts_f32(s0 + e * 4u, phi);
        }
        if (a.state_in_smem) {
            sts_f32(sp + e * 4u, p);
            sts_f32(sw + e * 4u, 0.f);
        } else {
            gp[idx] = p;
            gw[idx] = 0.f;
        }
    }
    __syncthreads();

    const int64_t win0 = a.S - (int64_t)a.W;  // steps j >= win0 add phi^(j+1) to the window
    const int mhalf = (a.M - 2) / 2;
    for (int64_t j = 0; j < a.S; ++j) {
        const float4 cf = __ldg(reinterpret_cast<const float4*>(a.sched) + j);
        const uint32_t cur = s0 + (uint32_t)(j & 1) * buf_bytes;
        const uint32_t nxt = s0 + (uint32_t)((j & 1) ^ 1) * buf_bytes;
        const bool in_win = j >= win0;
        for (int t = warp; t < a.T; t += NW) {
            const int4 tp = __ldg(a.tuples + t);
            const float L0 = tuple_field<RB, BF16>(a.entries + (size_t)tp.x * G + g, tp.y, tp.z,
                                                   cur + (uint32_t)r * ES);
            const int row = __ldg(a.tuple_rows + t * G + g);
            if (row < 0) continue;
            const uint32_t e = (uint32_t)(row * RB + r);
            const float phi = BF16 ? lds_f32(master + e * 4u) : lds_f32(cur + e * 4u);
            float L = L0;
            if (a.h) L += 2.f * __ldg(a.h + row) * fabsf(phi);
            const float phi2 = phi * phi;
            const float pw = pot_pow(phi, phi2, mhalf);
            float p = a.state_in_smem ? lds_f32(sp + e * 4u) : gp[e];
            p = p - fmaf(cf.x, pw, cf.y * L);
            const float phin = fmaf(cf.z, p, phi);
            if (a.state_in_smem) sts_f32(sp + e * 4u, p);
            else gp[e] = p;
            if constexpr (BF16) {
                sts_f32(master + e * 4u, phin);
                sts_bf16(nxt + e * 2u, phin);
            } else {
                sts_f32(nxt + e * 4u, phin);
            }
            if (in_win) {
                if (a.state_in_smem) sts_f32(sw + e * 4u, lds_f32(sw + e * 4u) + phin);
                else gw[e] += phin;
            }
        }
        __syncthreads();
    }

    // ---- outputs, [R][N] layout, coalesced over rows ----
    const uint32_t fin = s0 + (uint32_t)(a.S & 1) * buf_bytes;
    const int64_t nwin = a.S < a.W ? a.S : a.W;
    const float inv_w = 1.0f / (float)nwin;
    bool bad = false;
    for (int idx = threadIdx.x; idx < NRB; idx += blockDim.x) {
        const int rr = idx / a.N, row = idx % a.N, rep = rep0 + rr;
        if (rep >= a.R) continue;
        const uint32_t e = (uint32_t)(row * RB + rr);
        const float phi = BF16 ? lds_f32(master + e * 4u) : lds_f32(fin + e * 4u);
        const float p = a.state_in_smem ? lds_f32(sp + e * 4u) : gp[e];
        const float w = a.state_in_smem ? lds_f32(sw + e * 4u) : gw[e];
        const size_t o = (size_t)rep * a.N + row;
        if (a.phi_out) a.phi_out[o] = phi;
        if (a.p_out) a.p_out[o] = p;
        if (a.phibar_out) a.phibar_out[o] = w * inv_w;
        bad |= !(isfinite(phi) && isfinite(p));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, HQA_DEV_NONFINITE);
}

template <int RB, bool BF16>
__global__ void __launch_bounds__(kMaxThreads, 1) k_sparse_md(const MDArgs a)
{
    md_block<RB, BF16>(a, blockIdx.x, blockIdx.x);
}

// Persistent batch kernel: work items (instance, replica block) in
// longest-first order, taken from a global counter; every item is a whole
// trajectory of one replica block of one instance.
struct BatchItem {
    int inst;
    int blk;
};

template <int RB, bool BF16>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_sparse_md_batch(const MDArgs* __restrict__ insts, const BatchItem* __restrict__ items, int nitems,
                  int* __restrict__ counter)
{
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const BatchItem w = items[it];
        const MDArgs a = insts[w.inst];
        __syncthreads();
        md_block<RB, BF16>(a, w.blk, blockIdx.x);
    }
}

struct FieldArgs {
    const uint4* entries;
    const int4* tuples;
    const int* tuple_rows;
    const float* h;
    const float* phi;
    float* L;
    int32_t N, Npad, T, R;
};

template <int RB, bool BF16>
__global__ void __launch_bounds__(kMaxThreads, 1) k_sparse_field(const FieldArgs a)
{
    constexpr int G = 32 / RB;
    constexpr int ES = BF16 ? 2 : 4;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t buf_bytes = ((uint32_t)a.Npad * RB * ES + 15u) & ~15u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int g = lane / RB, r = lane % RB;
    const int rep0 = blockIdx.x * RB;
    for (uint32_t o = threadIdx.x * 4u; o < buf_bytes; o += blockDim.x * 4u) sts_f32(s0 + o, 0.f);
    __syncthreads();
    for (int idx = threadIdx.x; idx < a.N * RB; idx += blockDim.x) {
        const int rr = idx / a.N, row = idx % a.N, rep = rep0 + rr;
        const float v = rep < a.R ? a.phi[(size_t)rep * a.N + row] : 0.f;
        const uint32_t e = (uint32_t)(row * RB + rr);
        if constexpr (BF16) sts_bf16(s0 + e * 2u, v);
        else sts_f32(s0 + e * 4u, v);
    }
    __syncthreads();
    for (int t = warp; t < a.T; t += NW) {
        const int4 tp = __ldg(a.tuples + t);
        float L = tuple_field<RB, BF16>(a.entries + (size_t)tp.x * G + g, tp.y, tp.z,
                                         s0 + (uint32_t)r * ES);
        const int row = __ldg(a.tuple_rows + t * G + g);
        const int rep = rep0 + r;
        if (row < 0 || rep >= a.R) continue;
        if (a.h) L += 2.f * __ldg(a.h + row) * fabsf(a.phi[(size_t)rep * a.N + row]);
        a.L[(size_t)rep * a.N + row] = L;
    }
}

// ---------------------------------------------------------------------------
// host: plan construction
// ---------------------------------------------------------------------------

}  // namespace

void hqa_schedule_bank_section(const std::vector<std::vector<int>>& lists, int P, int N, int K,
                               std::vector<int>& out /* [K][G] */, int64_t& wavefronts)
{
    const int G = (int)lists.size();
    out.assign((size_t)K * G, -1);
    // buckets[g][q] = rows of list g in bank group q
    std::vector<std::vector<std::vector<int>>> bk(G, std::vector<std::vector<int>>(P));
    std::vector<int> remaining(G, 0);
    for (int g = 0; g < G; ++g) {
        for (int j : lists[g]) bk[g][j % P].push_back(j);
        remaining[g] = (int)lists[g].size();
    }
    std::vector<int> order(P);
    std::vector<int> cnt(P);
    for (int pos = 0; pos < K; ++pos) {
        for (int ph = 0; ph < G / P; ++ph) {
            for (int u = 0; u < P; ++u) order[u] = ph * P + u;
            std::sort(order.begin(), order.end(),
                      [&](int x, int y) { return remaining[x] > remaining[y]; });
            uint64_t used = 0;
            std::fill(cnt.begin(), cnt.end(), 0);
            for (int g : order) {
                int pick = -1;
                if (remaining[g] > 0) {
                    int best_q = -1;
                    size_t best_n = 0;
                    for (int q = 0; q < P; ++q) {
                        if ((used >> q) & 1ull) continue;
                        if (bk[g][q].size() > best_n) { best_n = bk[g][q].size(); best_q = q; }
                    }
                    if (best_q < 0)  // every non-empty group already used: accept a conflict
                        for (int q = 0; q < P; ++q)
                            if (!bk[g][q].empty() && (best_q < 0 || bk[g][q].size() > best_n)) {
                                best_q = q;
                                best_n = bk[g][q].size();
                            }
                    pick = bk[g][best_q].back();
                    bk[g][best_q].pop_back();
                    --remaining[g];
                } else {
                    int q = 0;
                    while (q < P && ((used >> q) & 1ull)) ++q;
                    if (q == P) q = 0;
                    const int z = ((q - N % P) % P + P) % P;  // zero row N + z has group q
                    pick = N + z;
                }
                const int q = pick % P;
                used |= 1ull << q;
                ++cnt[q];
                out[(size_t)pos * G + g] = pick;
            }
            wavefronts += *std::max_element(cnt.begin(), cnt.end());
        }
    }
}

namespace {
}  // namespace

static size_t op_bytes(int Npad, int RB, int prec)
{
    const size_t es = prec == HQA_PREC_BF16 ? 2 : 4;
    return (2 * (size_t)Npad * RB * es + 15) & ~(size_t)15;
}

size_t hqa_sparse_smem_bytes(const hqa_ctx* ctx, int RB, int prec)
{
    const int G = 32 / RB;
    const size_t Npad = (size_t)ctx->N + G;
    size_t b = op_bytes((int)Npad, RB, prec);
    if (prec == HQA_PREC_BF16) b += (size_t)ctx->N * RB * 4;
    return b;
}

static size_t state_bytes(const hqa_ctx* ctx, int RB) { return (size_t)ctx->N * RB * 8; }

int hqa_sparse_pick_rb(const hqa_ctx* ctx, int32_t R, int prec)
{
    const int cands[6] = {32, 16, 8, 4, 2, 1};
    int best = 0;
    for (int RB : cands) {
        if (hqa_sparse_smem_bytes(ctx, RB, prec) > ctx->smem_optin) continue;
        const int64_t blocks = (R + RB - 1) / RB;
        if (blocks * 5 >= (int64_t)ctx->sm_count * 4) return RB;  // >= 80% of the SMs busy
        best = RB;  // smaller RB gives more blocks; keep going
    }
    return best;
}

hqa_status hqa_sparse_plan(hqa_ctx* ctx, int RB, int prec, const SparsePlan** out)
{
    if (!ctx->unit) return HQA_ERR_UNSUPPORTED;
    const int key = RB * 16 + prec;
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        *out = &it->second;
        return HQA_OK;
    }
    // building a plan allocates and uploads: not possible inside a capture
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    const int G = 32 / RB;
    const int N = ctx->N;
    const int es = prec == HQA_PREC_BF16 ? 2 : 4;
    // neighbour lists split by sign
    std::vector<std::vector<int>> P(N), Q(N);
    for (int i = 0; i < N; ++i)
        for (int64_t k = ctx->row_ptr[i]; k < ctx->row_ptr[i + 1]; ++k) {
            if (ctx->val[k] > 0) P[i].push_back(ctx->col[k]);
            else if (ctx->val[k] < 0) Q[i].push_back(ctx->col[k]);
        }
    std::vector<int> rows(N);
    std::iota(rows.begin(), rows.end(), 0);
    std::stable_sort(rows.begin(), rows.end(), [&](int x, int y) {
        if (P[x].size() != P[y].size()) return P[x].size() > P[y].size();
        return Q[x].size() > Q[y].size();
    });
    const int T = (N + G - 1) / G;
    struct Tup { std::vector<int> rows; int kp, kn; std::vector<int> pos, neg; };
    std::vector<Tup> tups(T);
    int64_t wave = 0, ideal = 0, stored = 0;
    for (int t = 0; t < T; ++t) {
        Tup& u = tups[t];
        u.rows.assign(G, -1);
        std::vector<std::vector<int>> lp(G), ln(G);
        size_t mp = 0, mn = 0;
        for (int g = 0; g < G; ++g) {
            const int k = t * G + g;
            if (k >= N) continue;
            const int row = rows[k];
            u.rows[g] = row;
            lp[g] = P[row];
            ln[g] = Q[row];
            mp = std::max(mp, lp[g].size());
            mn = std::max(mn, ln[g].size());
        }
        u.kp = (int)((mp + 3) / 4 * 4);
        u.kn = (int)((mn + 3) / 4 * 4);
        hqa_schedule_bank_section(lp, G, N, u.kp, u.pos, wave);
        hqa_schedule_bank_section(ln, G, N, u.kn, u.neg, wave);
        ideal += u.kp + u.kn;
        stored += (int64_t)(u.kp + u.kn) * G;
    }
    // longest tuples first: warps take tuples t = warp, warp + NW, ...
    std::vector<int> ord(T);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int x, int y) { return tups[x].kp + tups[x].kn > tups[y].kp + tups[y].kn; });
    int64_t chunks = 0;
    for (int t = 0; t < T; ++t) chunks += (tups[t].kp + tups[t].kn) / 4;
    std::vector<uint4> ent((size_t)std::max<int64_t>(chunks, 1) * G);
    std::vector<int4> tpl(T);
    std::vector<int> trows((size_t)T * G);
    int64_t c0 = 0;
    for (int ti = 0; ti < T; ++ti) {
        const Tup& u = tups[ord[ti]];
        tpl[ti] = make_int4((int)c0, u.kp / 4, u.kn / 4, 0);
        for (int g = 0; g < G; ++g) trows[(size_t)ti * G + g] = u.rows[g];
        auto emit = [&](const std::vector<int>& sec, int K) {
            for (int c = 0; c < K / 4; ++c) {
                for (int g = 0; g < G; ++g) {
                    uint32_t v[4];
                    for (int q = 0; q < 4; ++q)
                        v[q] = (uint32_t)sec[(size_t)(c * 4 + q) * G + g] * (uint32_t)(RB * es);
                    ent[(size_t)(c0 + c) * G + g] = make_uint4(v[0], v[1], v[2], v[3]);
                }
            }
            c0 += K / 4;
        };
        emit(u.pos, u.kp);
        emit(u.neg, u.kn);
    }
    SparsePlan pl;
    pl.RB = RB;
    pl.G = G;
    pl.T = T;
    pl.Npad = N + G;
    pl.prec = prec;
    pl.chunks = chunks;
    pl.pad_ratio = ctx->nnz > 0 ? (double)stored / (double)ctx->nnz : 0.0;
    pl.conflict_ratio = ideal > 0 ? (double)wave / (double)ideal : 1.0;
    HQA_CUDA_TRY(cudaMalloc(&pl.d_entries, ent.size() * sizeof(uint4)));
    HQA_CUDA_TRY(cudaMalloc(&pl.d_tuples, tpl.size() * sizeof(int4)));
    HQA_CUDA_TRY(cudaMalloc(&pl.d_tuple_rows, trows.size() * sizeof(int)));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_entries, ent.data(), ent.size() * sizeof(uint4), cudaMemcpyHostToDevice));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_tuples, tpl.data(), tpl.size() * sizeof(int4), cudaMemcpyHostToDevice));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_tuple_rows, trows.data(), trows.size() * sizeof(int), cudaMemcpyHostToDevice));
    auto ins = ctx->plans.emplace(key, pl);
    *out = &ins.first->second;
    return HQA_OK;
}

template <int RB, bool BF16>
static cudaError_t launch_md_t(const MDArgs& a, int threads, size_t smem, cudaStream_t st)
{
    cudaError_t e = hqa_smem_attr((const void*)k_sparse_md<RB, BF16>, smem);
    if (e != cudaSuccess) return e;
    const int blocks = (a.R + RB - 1) / RB;
    k_sparse_md<RB, BF16><<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int RB, bool BF16>
static cudaError_t launch_field_t(const FieldArgs& a, int threads, size_t smem, cudaStream_t st)
{
    cudaError_t e = hqa_smem_attr((const void*)k_sparse_field<RB, BF16>, smem);
    if (e != cudaSuccess) return e;
    const int blocks = (a.R + RB - 1) / RB;
    k_sparse_field<RB, BF16><<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

#define HQA_DISPATCH_RB(RBV, BF, FN, ...)                                      \
    ((RBV) == 32 ? (BF ? FN<32, true>(__VA_ARGS__) : FN<32, false>(__VA_ARGS__)) : \
     (RBV) == 16 ? (BF ? FN<16, true>(__VA_ARGS__) : FN<16, false>(__VA_ARGS__)) : \
     (RBV) == 8  ? (BF ? FN<8, true>(__VA_ARGS__) : FN<8, false>(__VA_ARGS__)) :   \
     (RBV) == 4  ? (BF ? FN<4, true>(__VA_ARGS__) : FN<4, false>(__VA_ARGS__)) :   \
     (RBV) == 2  ? (BF ? FN<2, true>(__VA_ARGS__) : FN<2, false>(__VA_ARGS__)) :   \
                   (BF ? FN<1, true>(__VA_ARGS__) : FN<1, false>(__VA_ARGS__)))

static int pick_threads(int T)
{
    int w = std::min(32, std::max(1, T));
    return w * 32;
}

hqa_status hqa_sparse_launch_md(hqa_ctx* ctx, const SparsePlan* pl, const StepCoef* d_sched,
                                int64_t S, int32_t W, int32_t R, uint64_t seed, int init,
                                const float* phi0, const float* p0, int M, float* phi_out,
                                float* p_out, float* phibar_out, cudaStream_t st)
{
    const int RB = pl->RB;
    const bool bf = pl->prec == HQA_PREC_BF16;
    size_t smem = hqa_sparse_smem_bytes(ctx, RB, pl->prec);
    const size_t sb = state_bytes(ctx, RB);
    MDArgs a{};
    a.entries = pl->d_entries;
    a.tuples = pl->d_tuples;
    a.tuple_rows = pl->d_tuple_rows;
    a.sched = d_sched;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.phi0 = phi0;
    a.p0 = p0;
    a.phi_out = phi_out;
    a.p_out = p_out;
    a.phibar_out = phibar_out;
    a.status = ctx->d_status;
    a.seed = seed;
    a.S = S;
    a.W = W;
    a.N = ctx->N;
    a.Npad = pl->Npad;
    a.T = pl->T;
    a.R = R;
    a.M = M;
    a.init = init;
    if (smem + sb <= ctx->smem_optin) {
        smem += sb;
        a.state_in_smem = 1;
        a.gstate = nullptr;
    } else {
        const int blocks = (R + RB - 1) / RB;
        hqa_status s = hqa_reserve(ctx, &ctx->d_state, &ctx->state_cap, (size_t)blocks * sb);
        if (s != HQA_OK) return s;
        a.state_in_smem = 0;
        a.gstate = static_cast<float*>(ctx->d_state);
        a.gstride = sb / sizeof(float);
    }
    if (smem > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    cudaError_t e = HQA_DISPATCH_RB(RB, bf, launch_md_t, a, pick_threads(pl->T), smem, st);
    return e == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_sparse_launch_field(hqa_ctx* ctx, const SparsePlan* pl, int32_t R,
                                   const float* phi, float* L, cudaStream_t st)
{
    const int RB = pl->RB;
    const bool bf = pl->prec == HQA_PREC_BF16;
    const size_t es = bf ? 2 : 4;
    const size_t smem = ((size_t)pl->Npad * RB * es + 15) & ~(size_t)15;
    if (smem > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    FieldArgs a{};
    a.entries = pl->d_entries;
    a.tuples = pl->d_tuples;
    a.tuple_rows = pl->d_tuple_rows;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.phi = phi;
    a.L = L;
    a.N = ctx->N;
    a.Npad = pl->Npad;
    a.T = pl->T;
    a.R = R;
    cudaError_t e = HQA_DISPATCH_RB(RB, bf, launch_field_t, a, pick_threads(pl->T), smem, st);
    return e == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Uneven batch: every member instance x ceil(R / RB) replica blocks becomes a
// work item; items are ordered longest-first (cost ~ stored positions per
// step + the per-element update) and pulled from a counter by a persistent
// grid of one CTA per SM.  Instance k's outputs start at R * (sum of the
// earlier members' N); its momenta use the stream seed + (k + 1) * 0x632BE59BD9B4E019.
// ---------------------------------------------------------------------------
template <int RB, bool BF16>
static cudaError_t launch_batch_t(const MDArgs* insts, const BatchItem* items, int nitems,
                                  int* counter, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = hqa_smem_attr((const void*)k_sparse_md_batch<RB, BF16>, smem);
    if (e != cudaSuccess) return e;
    k_sparse_md_batch<RB, BF16><<<grid, kMaxThreads, smem, st>>>(insts, items, nitems, counter);
    return cudaGetLastError();
}

hqa_status hqa_batch_launch_md(hqa_ctx* b, int RB, int prec, const StepCoef* d_sched, int64_t S,
                               int32_t W, int32_t R, uint64_t seed, int init, const float* phi0,
                               const float* p0, int M, float* phi_out, float* p_out,
                               float* phibar_out, cudaStream_t st)
{
    const int count = (int)b->members.size();
    const bool bf = prec == HQA_PREC_BF16;
    // shared memory: the largest member's operand buffers, plus p/w on chip where they
    // fit; 1 KB of the opt-in limit stays free for the kernel's static shared memory
    const size_t cap = b->smem_optin - 1024;
    size_t smem = 0;
    for (hqa_ctx* m : b->members) smem = std::max(smem, hqa_sparse_smem_bytes(m, RB, prec));
    if (smem > cap) return HQA_ERR_TOO_LARGE;
    size_t smem_dyn = smem;
    for (hqa_ctx* m : b->members) {
        const size_t need = hqa_sparse_smem_bytes(m, RB, prec) + state_bytes(m, RB);
        if (need <= cap) smem_dyn = std::max(smem_dyn, need);
    }
    std::vector<MDArgs> args(count);
    std::vector<BatchItem> items;
    std::vector<double> cost;
    size_t gslot = 0;
    const int blocks = (R + RB - 1) / RB;
    for (int k = 0; k < count; ++k) {
        hqa_ctx* m = b->members[k];
        const SparsePlan* pl = nullptr;
        hqa_status s = hqa_sparse_plan(m, RB, prec, &pl);
        if (s != HQA_OK) return s;
        MDArgs a;
        std::memset(&a, 0, sizeof a);   // padding too: the table is compared bytewise
        a.entries = pl->d_entries;
        a.tuples = pl->d_tuples;
        a.tuple_rows = pl->d_tuple_rows;
        a.sched = d_sched;
        a.h = m->has_h ? m->d_h : nullptr;
        const size_t off = (size_t)R * (size_t)b->member_off[k];
        a.phi0 = phi0 ? phi0 + off : nullptr;   // HQA_INIT_GIVEN: the same member blocks
        a.p0 = p0 ? p0 + off : nullptr;
        a.phi_out = phi_out ? phi_out + off : nullptr;
        a.p_out = p_out ? p_out + off : nullptr;
        a.phibar_out = phibar_out ? phibar_out + off : nullptr;
        a.status = b->d_status;
        a.seed = seed + (uint64_t)(k + 1) * 0x632BE59BD9B4E019ull;
        a.S = S;
        a.W = W;
        a.N = m->N;
        a.Npad = pl->Npad;
        a.T = pl->T;
        a.R = R;
        a.M = M;
        a.init = init;
        const size_t need = hqa_sparse_smem_bytes(m, RB, prec) + state_bytes(m, RB);
        a.state_in_smem = need <= smem_dyn ? 1 : 0;
        if (!a.state_in_smem) gslot = std::max(gslot, state_bytes(m, RB));
        args[k] = a;
        const double c = (double)pl->chunks * 4.0 * pl->G + 8.0 * m->N;  // positions + updates per step
        for (int blk = 0; blk < blocks; ++blk) {
            items.push_back({k, blk});
            cost.push_back(c);
        }
    }
    std::vector<int> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<BatchItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    const int grid = b->sm_count;
    // device work tables: instance args | items | counter
    const size_t off_items = (args.size() * sizeof(MDArgs) + 255) & ~(size_t)255;
    const size_t off_cnt = off_items + ((sorted.size() * sizeof(BatchItem) + 255) & ~(size_t)255);
    void* const held = b->d_bwork;
    hqa_status s = hqa_reserve(b, &b->d_bwork, &b->bwork_cap, off_cnt + 256);
    if (s != HQA_OK) return s;
    if (b->d_bwork != held) b->bwork_host.clear();
    if (gslot) {
        s = hqa_reserve(b, &b->d_state, &b->state_cap, (size_t)grid * gslot);
        if (s != HQA_OK) return s;
        for (auto& a : args)
            if (!a.state_in_smem) {
                a.gstate = static_cast<float*>(b->d_state);
                a.gstride = gslot / sizeof(float);   // the largest member's slice
            }
    }
    char* w = static_cast<char*>(b->d_bwork);
    // the tables are uploaded only when they differ from what the device holds (so a
    // repeated run, and a captured one, issues no host copy); the counter is reset always
    std::vector<char> tab(off_cnt, 0);
    const char* ab = reinterpret_cast<const char*>(args.data());
    const char* ib = reinterpret_cast<const char*>(sorted.data());
    std::copy(ab, ab + args.size() * sizeof(MDArgs), tab.begin());
    std::copy(ib, ib + sorted.size() * sizeof(BatchItem), tab.begin() + (std::ptrdiff_t)off_items);
    if (tab != b->bwork_host) {
        if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
        ++b->generation;
        b->bwork_host.clear();
        // pageable source: the copy is staged before cudaMemcpyAsync returns
        HQA_CUDA_TRY(cudaMemcpyAsync(w, tab.data(), tab.size(), cudaMemcpyHostToDevice, st));
        b->bwork_host.swap(tab);
    }
    HQA_CUDA_TRY(cudaMemsetAsync(w + off_cnt, 0, sizeof(int), st));
    cudaError_t e = HQA_DISPATCH_RB(RB, bf, launch_batch_t, reinterpret_cast<const MDArgs*>(w),
                                    reinterpret_cast<const BatchItem*>(w + off_items),
                                    (int)sorted.size(), reinterpret_cast<int*>(w + off_cnt), grid,
                                    smem_dyn, st);
    return e == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}
