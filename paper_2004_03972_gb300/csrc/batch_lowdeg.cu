// batch_lowdeg.cu -- uneven batches whose members have at most four couplings
// per spin (random 3-regular graphs and 2-D tori, the uneven-batch ensemble).
//
// Same method and work queue as k_sparse_md_batch (Methods, "Leapfrog
// algorithm": local field, kick, drift, window sum of Eq. (5); one work item =
// one member's block of RB replicas for the whole trajectory), with everything
// an item touches held on chip: its neighbour lists are staged in shared memory
// as four 16-bit entries per spin (neighbour index, bit 15 set for J = -1,
// padding pointing at a zero row of the operand), next to the double-buffered
// flux operand ([N + 1][RB], FP32 or BF16), the FP32 flux master (BF16
// operand only), the FP32 momentum and the window sums.  No global load is
// left in the step loop, which the list-streaming kernel spends waiting on L2.
// One thread per spin and pair of replicas (RB >= 2; one replica at RB = 1):
// a spin's list is decoded once for both, each neighbour is one 8-byte (FP32)
// or 4-byte (BF16) gather, and the state moves in pairs.  Every replica sees
// the same floating-point operations at every blocking.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "hqa_internal.cuh"

namespace {

constexpr int kLdThreads = 1024;
constexpr int kLdMaxN = 32767;   // 15-bit neighbour index; index N is the zero row
constexpr int kLdDeg = 4;

__host__ __device__ constexpr uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Shared-memory bytes of one item (member of N spins, RB replicas).
__host__ __device__ constexpr uint32_t ld_item_bytes(int N, int RB, bool bf16, bool has_h)
{
    return align16(2u * (uint32_t)(N + 1) * RB * (bf16 ? 2u : 4u)) +
           (bf16 ? align16((uint32_t)N * RB * 4u) : 0u) + 2u * align16((uint32_t)N * RB * 4u) +
           align16((uint32_t)N * 8u) + (has_h ? align16((uint32_t)N * 4u) : 0u);
}

struct LdMember {
    const uint2* lists;    // [N] four u16 entries
    const float* h;        // [N] or null
    const float* phi0;     // HQA_INIT_GIVEN: the member's [R][N] block
    const float* p0;
    float* phi_out;
    float* p_out;
    float* phibar_out;
    uint64_t seed;
    int32_t N;
    int32_t pad_;
};

struct LdArgs {
    const LdMember* mem;
    const int2* items;     // (member, replica block), longest member first
    int* counter;
    const StepCoef* sched;
    uint32_t* status;
    int64_t S;
    int32_t nitems, W, R, M, init;
};

__device__ __forceinline__ uint64_t ld_splitmix(uint64_t seed, uint64_t counter)
{
    // SplitMix64 (Steele, Lea, Flood 2014): output number counter+1 of the stream.
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float lds32(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts32(uint32_t a, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}

__device__ __forceinline__ uint2 lds64(uint32_t a)
{
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts64(uint32_t a, uint2 v)
{
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y));
}

template <bool BF16>
__device__ __forceinline__ float ld_op(uint32_t a)
{
    if constexpr (BF16) {
        unsigned short v;
        asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
        return __uint_as_float(((uint32_t)v) << 16);
    } else {
        return lds32(a);
    }
}

template <bool BF16>
__device__ __forceinline__ void st_op(uint32_t a, float v)
{
    if constexpr (BF16) {
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        const unsigned short u = *reinterpret_cast<const unsigned short*>(&b);
        asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(u));
    } else {
        sts32(a, v);
    }
}

// J_ij phi_j of one list entry u for replicas r0 .. r0 + PR - 1 (u & 0x8000:
// J = -1), added into v[]
template <int RB, int PR, bool BF16>
__device__ __forceinline__ void nb(uint32_t cur, uint32_t u, int r0, float* v)
{
    constexpr uint32_t ES = BF16 ? 2u : 4u;
    const uint32_t a = cur + ((u & 0x7fffu) * RB + (uint32_t)r0) * ES;
    const uint32_t sg = (u & 0x8000u) << 16;   // the FP32 sign bit
    if constexpr (PR == 2 && !BF16) {
        const uint2 x = lds64(a);
        v[0] = __uint_as_float(x.x ^ sg);
        v[1] = __uint_as_float(x.y ^ sg);
    } else if constexpr (PR == 2) {
        uint32_t x;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(x) : "r"(a));
        v[0] = __uint_as_float((x << 16) ^ sg);
        v[1] = __uint_as_float((x & 0xffff0000u) ^ sg);
    } else {
        v[0] = __uint_as_float(__float_as_uint(ld_op<BF16>(a)) ^ sg);
    }
}

// Packed FP32 pairs (Blackwell's f32x2 arithmetic: each half rounds like the
// scalar instruction, so a pair gets the bits of two scalar evaluations).
__device__ __forceinline__ uint64_t pk(float x, float y)
{
    return (uint64_t)__float_as_uint(x) | ((uint64_t)__float_as_uint(y) << 32);
}
__device__ __forceinline__ float lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <int RB, bool BF16>
__global__ void __launch_bounds__(kLdThreads, 1) k_batch_lowdeg(const LdArgs a)
{
    constexpr uint32_t ES = BF16 ? 2u : 4u;
    constexpr int PR = RB >= 2 ? 2 : 1;   // replicas per thread
    constexpr int TR = RB / PR;           // threads per spin
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    const int t = threadIdx.x;
    for (;;) {
        __syncthreads();
        if (t == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) break;
        const int2 wi = a.items[it];
        const LdMember m = a.mem[wi.x];
        const int N = m.N, NRB = N * RB, rep0 = wi.y * RB;
        const uint32_t buf = (uint32_t)(N + 1) * RB * ES;
        const uint32_t opb = align16(2u * buf);
        const uint32_t master = s0 + opb;
        const uint32_t sp = master + (BF16 ? align16((uint32_t)NRB * 4u) : 0u);
        const uint32_t sw = sp + align16((uint32_t)NRB * 4u);
        const uint32_t sl = sw + align16((uint32_t)NRB * 4u);
        const uint32_t sh = sl + align16((uint32_t)N * 8u);

        // both operand buffers zero (row N stays zero: the lists' padding), lists, h
        for (uint32_t o = (uint32_t)t * 16u; o < opb; o += kLdThreads * 16u) {
            sts64(s0 + o, make_uint2(0u, 0u));
            sts64(s0 + o + 8u, make_uint2(0u, 0u));
        }
        for (int i = t; i < N; i += kLdThreads) {
            sts64(sl + (uint32_t)i * 8u, __ldg(m.lists + i));
            if (m.h) sts32(sh + (uint32_t)i * 4u, __ldg(m.h + i));
        }
        __syncthreads();
        for (int idx = t; idx < NRB; idx += kLdThreads) {
            const int row = idx / RB, rr = idx % RB, rep = rep0 + rr;
            float phi = 0.f, p = 0.f;
            if (rep < a.R) {
                const uint64_t c = ((uint64_t)rep << 32) | (uint64_t)row;
                if (a.init == HQA_INIT_GIVEN) {
                    phi = m.phi0[(size_t)rep * N + row];
                    p = m.p0[(size_t)rep * N + row];
                } else {
                    p = (ld_splitmix(m.seed, c) >> 63) ? -1.f : 1.f;
                    if (a.init == HQA_INIT_RANDOM_FLUX) {
                        const uint64_t z = ld_splitmix(m.seed, c | (1ull << 62));
                        phi = (float)((int64_t)(z >> 40) - (1 << 23)) * 0x1p-26f;
                    }
                }
            }
            const uint32_t e = (uint32_t)idx;
            if constexpr (BF16) sts32(master + e * 4u, phi);
            st_op<BF16>(s0 + e * ES, phi);
            sts32(sp + e * 4u, p);
            sts32(sw + e * 4u, 0.f);
        }
        __syncthreads();

        const int64_t win0 = a.S - (int64_t)a.W;   // steps j >= win0 add phi^(j+1) to the window
        const int mhalf = (a.M - 2) / 2;
        for (int64_t j = 0; j < a.S; ++j) {
            const float4 cf = __ldg(reinterpret_cast<const float4*>(a.sched) + j);
            const uint32_t cur = s0 + (uint32_t)(j & 1) * buf;
            const uint32_t nxt = s0 + (uint32_t)((j & 1) ^ 1) * buf;
            const bool in_win = j >= win0;
            for (int idx = t; idx < N * TR; idx += kLdThreads) {
                const int row = idx / TR, r0 = (idx % TR) * PR;
                const uint2 l = lds64(sl + (uint32_t)row * 8u);
                float v0[PR], v1[PR], v2[PR], v3[PR];
                nb<RB, PR, BF16>(cur, l.x & 0xffffu, r0, v0);
                nb<RB, PR, BF16>(cur, l.x >> 16, r0, v1);
                nb<RB, PR, BF16>(cur, l.y & 0xffffu, r0, v2);
                nb<RB, PR, BF16>(cur, l.y >> 16, r0, v3);
                const uint32_t e = (uint32_t)(row * RB + r0);
                float phi[PR], p[PR], phin[PR];
                if constexpr (PR == 2) {
                    const uint2 f = lds64((BF16 ? master : cur) + e * 4u);
                    const uint2 q = lds64(sp + e * 4u);
                    phi[0] = __uint_as_float(f.x);
                    phi[1] = __uint_as_float(f.y);
                    p[0] = __uint_as_float(q.x);
                    p[1] = __uint_as_float(q.y);
                } else {
                    phi[0] = lds32((BF16 ? master : cur) + e * 4u);
                    p[0] = lds32(sp + e * 4u);
                }
                const float hr = m.h ? 2.f * lds32(sh + (uint32_t)row * 4u) : 0.f;
                // the same operations, in pairs or alone:
                //   L = (v0 + v1) + (v2 + v3) [+ 2h|phi| by fma]; pw = phi^(M-1)
                //   p -= fma(kA, pw, kB L); phi' = fma(dA, p, phi)
                if constexpr (PR == 2) {
                    const uint64_t f = pk(phi[0], phi[1]);
                    uint64_t L = add2(add2(pk(v0[0], v0[1]), pk(v1[0], v1[1])),
                                      add2(pk(v2[0], v2[1]), pk(v3[0], v3[1])));
                    if (m.h) L = fma2(pk(hr, hr), pk(fabsf(phi[0]), fabsf(phi[1])), L);
                    const uint64_t f2 = mul2(f, f);
                    uint64_t pw = f;
                    for (int q = 0; q < mhalf; ++q) pw = mul2(pw, f2);
                    const uint64_t pp = sub2(pk(p[0], p[1]),
                                             fma2(pk(cf.x, cf.x), pw, mul2(pk(cf.y, cf.y), L)));
                    const uint64_t fn = fma2(pk(cf.z, cf.z), pp, f);
                    p[0] = lo(pp);
                    p[1] = hi(pp);
                    phin[0] = lo(fn);
                    phin[1] = hi(fn);
                } else {
                    float L = (v0[0] + v1[0]) + (v2[0] + v3[0]);
                    if (m.h) L = fmaf(hr, fabsf(phi[0]), L);
                    const float phi2 = __fmul_rn(phi[0], phi[0]);
                    float pw = phi[0];
                    for (int q = 0; q < mhalf; ++q) pw = __fmul_rn(pw, phi2);
                    p[0] = __fsub_rn(p[0], fmaf(cf.x, pw, __fmul_rn(cf.y, L)));
                    phin[0] = fmaf(cf.z, p[0], phi[0]);
                }
                if constexpr (PR == 2) {
                    sts64(sp + e * 4u, make_uint2(__float_as_uint(p[0]), __float_as_uint(p[1])));
                    const uint2 fn = make_uint2(__float_as_uint(phin[0]), __float_as_uint(phin[1]));
                    if constexpr (BF16) {
                        sts64(master + e * 4u, fn);
                        st_op<BF16>(nxt + e * ES, phin[0]);
                        st_op<BF16>(nxt + (e + 1u) * ES, phin[1]);
                    } else {
                        sts64(nxt + e * 4u, fn);
                    }
                    if (in_win) {
                        const uint2 w = lds64(sw + e * 4u);
                        const uint64_t ws = add2((uint64_t)w.x | ((uint64_t)w.y << 32), pk(phin[0], phin[1]));
                        sts64(sw + e * 4u, make_uint2((uint32_t)ws, (uint32_t)(ws >> 32)));
                    }
                } else {
                    sts32(sp + e * 4u, p[0]);
                    if constexpr (BF16) sts32(master + e * 4u, phin[0]);
                    st_op<BF16>(nxt + e * ES, phin[0]);
                    if (in_win) sts32(sw + e * 4u, lds32(sw + e * 4u) + phin[0]);
                }
            }
            __syncthreads();
        }

        // outputs, [R][N] member block, coalesced over spins
        const uint32_t fin = s0 + (uint32_t)(a.S & 1) * buf;
        const int64_t nwin = a.S < a.W ? a.S : a.W;
        const float inv_w = 1.0f / (float)nwin;
        bool bad = false;
        for (int idx = t; idx < NRB; idx += kLdThreads) {
            const int rr = idx / N, row = idx % N, rep = rep0 + rr;
            if (rep >= a.R) continue;
            const uint32_t e = (uint32_t)(row * RB + rr);
            const float phi = BF16 ? lds32(master + e * 4u) : lds32(fin + e * 4u);
            const float p = lds32(sp + e * 4u);
            const size_t o = (size_t)rep * N + row;
            if (m.phi_out) m.phi_out[o] = phi;
            if (m.p_out) m.p_out[o] = p;
            if (m.phibar_out) m.phibar_out[o] = lds32(sw + e * 4u) * inv_w;
            bad |= !(isfinite(phi) && isfinite(p));
        }
        if (__syncthreads_or(bad) && t == 0) atomicOr(a.status, HQA_DEV_NONFINITE);
    }
}

template <int RB, bool BF16>
cudaError_t launch_ld(const LdArgs& a, int grid, size_t smem, cudaStream_t st)
{
    const cudaError_t e = hqa_smem_attr((const void*)k_batch_lowdeg<RB, BF16>, smem);
    if (e != cudaSuccess) return e;
    k_batch_lowdeg<RB, BF16><<<grid, kLdThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Every member has at most four couplings per spin, each -1 or +1, and fewer
// than 2^15 spins (host-only check, cached).
bool hqa_lowdeg_eligible(const hqa_ctx* b)
{
    if (!b->is_batch) return false;
    if (b->ld_state == 0) {
        bool ok = true;
        for (const hqa_ctx* m : b->members) {
            ok = ok && m->unit && m->N <= kLdMaxN;
            for (int i = 0; ok && i < m->N; ++i)
                ok = m->row_ptr[i + 1] - m->row_ptr[i] <= kLdDeg;
        }
        b->ld_state = ok ? 1 : -1;
    }
    return b->ld_state > 0;
}

size_t hqa_lowdeg_smem_bytes(const hqa_ctx* b, int RB, int prec)
{
    size_t need = 0;
    for (const hqa_ctx* m : b->members)
        need = std::max<size_t>(need, ld_item_bytes(m->N, RB, prec == HQA_PREC_BF16, m->has_h));
    return need;
}

// Largest replica blocking (4, 2, 1) whose items fit in shared memory and leave
// at least two items per SM; else the smallest that fits; 0 if none.
int hqa_lowdeg_pick_rb(const hqa_ctx* b, int32_t R, int prec)
{
    int pick = 0;
    for (int rb : {4, 2, 1}) {
        if (hqa_lowdeg_smem_bytes(b, rb, prec) > b->smem_optin - 1024) continue;
        const int64_t items = (int64_t)b->members.size() * ((R + rb - 1) / rb);
        pick = rb;
        if (items >= 2 * (int64_t)b->sm_count) break;
    }
    return pick;
}

hqa_status hqa_lowdeg_launch_md(hqa_ctx* b, int RB, int prec, const StepCoef* d_sched, int64_t S,
                                int32_t W, int32_t R, uint64_t seed, int init, const float* phi0,
                                const float* p0, int M, float* phi_out, float* p_out,
                                float* phibar_out, cudaStream_t st)
{
    if (!hqa_lowdeg_eligible(b) || prec == HQA_PREC_BF16X2) return HQA_ERR_UNSUPPORTED;
    if (RB != 1 && RB != 2 && RB != 4) return HQA_ERR_UNSUPPORTED;
    const size_t smem = hqa_lowdeg_smem_bytes(b, RB, prec);
    if (smem > b->smem_optin - 1024) return HQA_ERR_TOO_LARGE;
    const int count = (int)b->members.size();
    // compact lists of every member, built once (outside any capture)
    if (b->ld_off.empty()) {
        if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
        std::vector<uint2> lists;
        std::vector<int64_t> off(count);
        for (int k = 0; k < count; ++k) {
            const hqa_ctx* m = b->members[k];
            off[k] = (int64_t)lists.size();
            for (int i = 0; i < m->N; ++i) {
                uint32_t u[kLdDeg];
                int c = 0;
                for (int64_t q = m->row_ptr[i]; q < m->row_ptr[i + 1]; ++q)
                    u[c++] = (uint32_t)m->col[q] | (m->val[q] < 0.f ? 0x8000u : 0u);
                for (; c < kLdDeg; ++c) u[c] = (uint32_t)m->N;   // the zero row
                lists.push_back(make_uint2(u[0] | (u[1] << 16), u[2] | (u[3] << 16)));
            }
        }
        hqa_status s = hqa_reserve(b, &b->d_ld, &b->ld_cap, lists.size() * sizeof(uint2));
        if (s != HQA_OK) return s;
        HQA_CUDA_TRY(cudaMemcpy(b->d_ld, lists.data(), lists.size() * sizeof(uint2),
                                cudaMemcpyHostToDevice));
        b->ld_off = off;
    }
    std::vector<LdMember> mem(count);
    std::vector<int2> items;
    const int blocks = (R + RB - 1) / RB;
    for (int k = 0; k < count; ++k) {
        const hqa_ctx* m = b->members[k];
        LdMember x;
        std::memset(&x, 0, sizeof x);   // padding too: the table is compared bytewise
        const size_t o = (size_t)R * (size_t)b->member_off[k];
        x.lists = static_cast<const uint2*>(b->d_ld) + b->ld_off[k];
        x.h = m->has_h ? m->d_h : nullptr;
        x.phi0 = phi0 ? phi0 + o : nullptr;
        x.p0 = p0 ? p0 + o : nullptr;
        x.phi_out = phi_out ? phi_out + o : nullptr;
        x.p_out = p_out ? p_out + o : nullptr;
        x.phibar_out = phibar_out ? phibar_out + o : nullptr;
        x.seed = seed + (uint64_t)(k + 1) * 0x632BE59BD9B4E019ull;
        x.N = m->N;
        mem[k] = x;
        for (int blk = 0; blk < blocks; ++blk) items.push_back(make_int2(k, blk));
    }
    // longest member first (ties in member order)
    std::stable_sort(items.begin(), items.end(), [&](const int2& x, const int2& y) {
        return b->members[x.x]->N > b->members[y.x]->N;
    });
    const size_t off_items = (mem.size() * sizeof(LdMember) + 255) & ~(size_t)255;
    const size_t off_cnt = off_items + ((items.size() * sizeof(int2) + 255) & ~(size_t)255);
    void* const held = b->d_ldwork;
    hqa_status s = hqa_reserve(b, &b->d_ldwork, &b->ldwork_cap, off_cnt + 256);
    if (s != HQA_OK) return s;
    if (b->d_ldwork != held) b->ldwork_host.clear();
    char* w = static_cast<char*>(b->d_ldwork);
    // uploaded only when the tables differ from what the device holds (a repeated
    // run, and a captured one, issues no host copy); the counter is reset always
    std::vector<char> tab(off_cnt, 0);
    const char* mb = reinterpret_cast<const char*>(mem.data());
    const char* ib = reinterpret_cast<const char*>(items.data());
    std::copy(mb, mb + mem.size() * sizeof(LdMember), tab.begin());
    std::copy(ib, ib + items.size() * sizeof(int2), tab.begin() + (std::ptrdiff_t)off_items);
    if (tab != b->ldwork_host) {
        if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
        ++b->generation;
        b->ldwork_host.clear();
        // pageable source: the copy is staged before cudaMemcpyAsync returns
        HQA_CUDA_TRY(cudaMemcpyAsync(w, tab.data(), tab.size(), cudaMemcpyHostToDevice, st));
        b->ldwork_host.swap(tab);
    }
    HQA_CUDA_TRY(cudaMemsetAsync(w + off_cnt, 0, sizeof(int), st));
    LdArgs a;
    a.mem = reinterpret_cast<const LdMember*>(w);
    a.items = reinterpret_cast<const int2*>(w + off_items);
    a.counter = reinterpret_cast<int*>(w + off_cnt);
    a.sched = d_sched;
    a.status = b->d_status;
    a.S = S;
    a.nitems = (int)items.size();
    a.W = W;
    a.R = R;
    a.M = M;
    a.init = init;
    const bool bf = prec == HQA_PREC_BF16;
    cudaError_t e;
    if (RB == 4) e = bf ? launch_ld<4, true>(a, b->sm_count, smem, st) : launch_ld<4, false>(a, b->sm_count, smem, st);
    else if (RB == 2) e = bf ? launch_ld<2, true>(a, b->sm_count, smem, st) : launch_ld<2, false>(a, b->sm_count, smem, st);
    else e = bf ? launch_ld<1, true>(a, b->sm_count, smem, st) : launch_ld<1, false>(a, b->sm_count, smem, st);
    return e == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}
