// sparse_md_vec.cu -- vectorised resident sparse HQA-MD kernel.
//
// Same method as sparse_md.cu (Methods, "Leapfrog algorithm": local field,
// kick, drift, window sum; one CTA owns RB replicas for the whole run), laid
// out so that shared-memory bandwidth bounds it:
//   * every lane gathers 16 bytes per neighbour -- V = 4 FP32 or V = 8 BF16
//     replicas -- with one 128-bit shared load, so a warp reads G rows x RB
//     replicas per instruction (G = 32 * V / RB);
//   * the operand keeps phi and -phi ([+ slots | - slots]) so a coupling of
//     -1 is a gather from the negated copy: every position is a plain add;
//   * a 128-bit shared load is served in four 8-lane phases, each covering P
//     rows; a row's slot s lives in bank-quad group s mod P.  The host
//     (a) relabels slots by local search so that within every phase the
//     neighbour loads of the P groups are balanced, and (b) orders each
//     phase's lists by bipartite edge colouring (rows x groups, König), so a
//     position is one conflict-free wavefront per phase except where a group
//     is overloaded;
//   * neighbour lists are u16 offsets (units of 16 bytes) staged in shared
//     memory once per launch, 8 positions per 128-bit load;
//   * sums use Blackwell's packed FP32 add (add.rn.f32x2);
//   * tuples are assigned to warps on the host (longest-processing-time
//     first); one __syncthreads() per leapfrog step; window sums live in
//     global memory (touched only in the last W steps);
//   * a lane updates the same rows at every step (the tuple-to-warp map is
//     fixed for the launch), so when no warp owns more than four tuples
//     the FP32 flux and momentum of the lane's rows stay in its
//     registers for the whole trajectory: the kick reads no shared memory
//     and writes only the next operand buffer.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <numeric>

#include "hqa_internal.cuh"

namespace {

constexpr int kMaxThreads = 1024;
// Register-resident state: a warp owning at most `reg` tuples (1, 2 or 4) keeps
// its rows' flux and momentum in registers; the launch bound then allows
// reg_threads(reg, bf16) threads, chosen so that no variant spills
// (1024 / 896 threads -> 64 / 72 registers, 832 / 704 -> 72 / 88, 512 -> 128).
__host__ __device__ constexpr int reg_threads(int reg, bool bf16)
{
    return reg == 1 ? (bf16 ? 896 : 1024) : reg == 2 ? (bf16 ? 704 : 832) : 512;
}

__device__ __forceinline__ uint64_t smix(uint64_t seed, uint64_t counter)
{
    // SplitMix64 (Steele, Lea, Flood 2014): output number counter+1 of the stream.
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint4 lds128(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts128(uint32_t a, uint4 v)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w));
}

__device__ __forceinline__ void sts32(uint32_t a, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}

__device__ __forceinline__ void sts16(uint32_t a, unsigned short v)
{
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(v));
}

__device__ __forceinline__ uint64_t pack2(uint32_t lo, uint32_t hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ float lo_f(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_f(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

__device__ __forceinline__ unsigned short bf16_bits(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<unsigned short*>(&b);
}

// One 16-byte gather as NP = V/2 packed f32x2 values.
template <bool BF16>
struct Gather {
    static constexpr int NP = BF16 ? 4 : 2;
    uint64_t v[NP];
    __device__ __forceinline__ void load(uint32_t addr)
    {
        const uint4 w = lds128(addr);
        if constexpr (BF16) {
            // bf16 pair (lo = replica 2k, hi = replica 2k+1) -> two FP32
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = pack2(ws[k] << 16, ws[k] & 0xffff0000u);
        } else {
            v[0] = pack2(w.x, w.y);
            v[1] = pack2(w.z, w.w);
        }
    }
};

// Neighbour sum of one tuple for this lane.  ent: shared address of this
// lane's first uint4 of entries (8 u16 offsets), consecutive chunks G * 16
// bytes apart; nhalf: number of 4-position half-chunks; base: shared address
// of this lane's quad in the current operand buffer.
// acc[0..1] += bf16 pair in w (lo -> acc0, hi -> acc1): Blackwell's mixed
// add converts the BF16 operand and adds it to the FP32 sum in one instruction.
__device__ __forceinline__ void add_bf16x2(float& a0, float& a1, uint32_t w)
{
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "add.rn.f32.bf16 %0, l, %0;\n\tadd.rn.f32.bf16 %1, h, %1;\n\t}"
        : "+f"(a0), "+f"(a1) : "r"(w));
}

// BF16 operand: 8 FP32 accumulators, one per replica of the lane.
template <int G>
__device__ __forceinline__ void tuple_field_bf16(uint32_t ent, int nhalf, uint32_t base, float* acc)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    for (int hc = 0; hc < nhalf; hc += 2) {
        const uint4 e = lds128(ent + (uint32_t)(hc >> 1) * (G * 16u));
        const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && hc + 1 >= nhalf) break;
            uint4 v[4];
            v[0] = lds128(base + ((ew[2 * h] & 0xffffu) << 4));
            v[1] = lds128(base + ((ew[2 * h] >> 16) << 4));
            v[2] = lds128(base + ((ew[2 * h + 1] & 0xffffu) << 4));
            v[3] = lds128(base + ((ew[2 * h + 1] >> 16) << 4));
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                add_bf16x2(acc[0], acc[1], v[u].x);
                add_bf16x2(acc[2], acc[3], v[u].y);
                add_bf16x2(acc[4], acc[5], v[u].z);
                add_bf16x2(acc[6], acc[7], v[u].w);
            }
        }
    }
}

template <int G, bool BF16>
__device__ __forceinline__ void tuple_field_vec(uint32_t ent, int nhalf, uint32_t base,
                                                uint64_t* acc)
{
    using GT = Gather<BF16>;
#pragma unroll
    for (int k = 0; k < GT::NP; ++k) acc[k] = 0ull;
    for (int hc = 0; hc < nhalf; hc += 2) {
        const uint4 e = lds128(ent + (uint32_t)(hc >> 1) * (G * 16u));
        const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && hc + 1 >= nhalf) break;
            GT a, b, c, d;
            a.load(base + ((ew[2 * h] & 0xffffu) << 4));
            b.load(base + ((ew[2 * h] >> 16) << 4));
            c.load(base + ((ew[2 * h + 1] & 0xffffu) << 4));
            d.load(base + ((ew[2 * h + 1] >> 16) << 4));
#pragma unroll
            for (int k = 0; k < GT::NP; ++k)
                acc[k] = add2(acc[k], add2(add2(a.v[k], b.v[k]), add2(c.v[k], d.v[k])));
        }
    }
}

struct VArgs {
    const uint4* entries;   // global copy, staged into shared memory at start
    const int4* tuples;     // {first chunk, half-chunks, 0, 0}
    const int* tuple_rows;  // [T][G] row index or -1
    const int* slot_of_row; // [N]
    const int* warp_off;    // [NW + 1]
    const int* tuple_list;
    const StepCoef* sched;
    const float* h;
    const float* phi0;
    const float* p0;
    float* phi_out;
    float* p_out;
    float* phibar_out;
    float* gwin;            // window sums, [block][slot][RB]
    float* L_out;           // field-only mode
    const float* phi_in;    // field-only mode
    uint32_t* status;
    uint64_t seed;
    int64_t S;
    int32_t W, N, Npad, T, R, M, init;
    uint32_t ent_bytes;
    int32_t reg;            // 0, or state in registers: every warp owns <= reg tuples
};

// Shared-memory layout (bytes):
//   ent    : ent_bytes (packed u16 offsets)
//   op[2]  : 2 step buffers, each [+ slots | - slots], Npad * RB * ES per half
//   master : Npad * RB FP32 (BF16 operand only)
//   p      : Npad * RB FP32
template <int RB, bool BF16, int REG>
__global__ void __launch_bounds__(REG > 0 ? reg_threads(REG, BF16) : kMaxThreads, 1)
    k_sparse_md_vec(const VArgs a)
{
    constexpr int ES = BF16 ? 2 : 4;
    constexpr int V = 16 / ES;     // replicas per lane
    constexpr int LPR = RB / V;    // lanes per row
    constexpr int G = 32 / LPR;    // rows per warp instruction
    constexpr int NP = V / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t half_bytes = (uint32_t)a.Npad * RB * ES;
    const uint32_t buf_bytes = 2u * half_bytes;
    const uint32_t op0 = s0 + a.ent_bytes;
    const uint32_t master = op0 + 2u * buf_bytes;
    const uint32_t ps = master + (BF16 ? (uint32_t)a.Npad * RB * 4u : 0u);
    const int NRB = a.N * RB;
    float* gw = a.gwin + (size_t)blockIdx.x * a.Npad * RB;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / LPR, q = lane % LPR;
    const int rep0 = blockIdx.x * RB;

    // ---- stage entries, zero operand buffers and window sums, initial state ----
    for (uint32_t o = threadIdx.x * 16u; o < a.ent_bytes; o += blockDim.x * 16u)
        sts128(s0 + o, __ldg(a.entries + o / 16u));
    for (uint32_t o = threadIdx.x * 16u; o < 2u * buf_bytes; o += blockDim.x * 16u)
        sts128(op0 + o, make_uint4(0, 0, 0, 0));
    for (int o = threadIdx.x; o < a.Npad * RB; o += blockDim.x) gw[o] = 0.f;
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
                p = (smix(a.seed, c) >> 63) ? -1.f : 1.f;
                if (a.init == HQA_INIT_RANDOM_FLUX) {
                    const uint64_t z = smix(a.seed, c | (1ull << 62));
                    phi = (float)((int64_t)(z >> 40) - (1 << 23)) * 0x1p-26f;
                }
            }
        }
        const uint32_t e = (uint32_t)(__ldg(a.slot_of_row + row) * RB + rr);
        if constexpr (BF16) {
            sts32(master + e * 4u, phi);
            sts16(op0 + e * 2u, bf16_bits(phi));
            sts16(op0 + half_bytes + e * 2u, bf16_bits(-phi));
        } else {
            sts32(op0 + e * 4u, phi);
            sts32(op0 + half_bytes + e * 4u, -phi);
        }
        sts32(ps + e * 4u, p);
    }
    __syncthreads();

    const int wbeg = __ldg(a.warp_off + warp), wend = __ldg(a.warp_off + warp + 1);
    const int64_t win0 = a.S - (int64_t)a.W;
    const int mhalf = (a.M - 2) / 2;
    if constexpr (REG > 0) {
        // this lane's rows: flux and momentum in registers for the whole trajectory
        constexpr int RS = REG > 0 ? REG : 1;
        float rphi[RS][V], rp[RS][V];
        uint32_t rent[RS], re0[RS];
        int rnh[RS];
        float rhr[RS];
        bool rok[RS];
#pragma unroll
        for (int kk = 0; kk < RS; ++kk) {
            const int k = wbeg + kk;
            rok[kk] = false;
            rent[kk] = 0u;
            rnh[kk] = 0;
            re0[kk] = 0u;
            rhr[kk] = 0.f;
            if (k < wend) {
                const int t = __ldg(a.tuple_list + k);
                const int4 tp = __ldg(a.tuples + t);
                rent[kk] = s0 + ((uint32_t)tp.x * G + g) * 16u;
                rnh[kk] = tp.y;
                const int row = __ldg(a.tuple_rows + t * G + g);
                if (row >= 0) {
                    rok[kk] = true;
                    re0[kk] = (uint32_t)(__ldg(a.slot_of_row + row) * RB + q * V);
                    rhr[kk] = a.h ? 2.f * __ldg(a.h + row) : 0.f;
                }
            }
#pragma unroll
            for (int k4 = 0; k4 < V / 4; ++k4) {
                uint4 x = make_uint4(0, 0, 0, 0), y = make_uint4(0, 0, 0, 0);
                if (rok[kk]) {
                    x = lds128((BF16 ? master : op0) + (re0[kk] + 4 * k4) * 4u);
                    y = lds128(ps + (re0[kk] + 4 * k4) * 4u);
                }
                rphi[kk][4 * k4] = __uint_as_float(x.x); rphi[kk][4 * k4 + 1] = __uint_as_float(x.y);
                rphi[kk][4 * k4 + 2] = __uint_as_float(x.z); rphi[kk][4 * k4 + 3] = __uint_as_float(x.w);
                rp[kk][4 * k4] = __uint_as_float(y.x); rp[kk][4 * k4 + 1] = __uint_as_float(y.y);
                rp[kk][4 * k4 + 2] = __uint_as_float(y.z); rp[kk][4 * k4 + 3] = __uint_as_float(y.w);
            }
        }
        const int nk = wend - wbeg;
        for (int64_t j = 0; j < a.S; ++j) {
            const float4 cf = __ldg(reinterpret_cast<const float4*>(a.sched) + j);
            const uint32_t cur = op0 + (uint32_t)(j & 1) * buf_bytes;
            const uint32_t nxt = op0 + (uint32_t)((j & 1) ^ 1) * buf_bytes;
            const bool in_win = j >= win0;
#pragma unroll
            for (int kk = 0; kk < RS; ++kk) {
                if (kk >= nk) break;
                float Lsum[V];
                if constexpr (BF16) {
                    tuple_field_bf16<G>(rent[kk], rnh[kk], cur + (uint32_t)q * 16u, Lsum);
                } else {
                    uint64_t acc[NP];
                    tuple_field_vec<G, BF16>(rent[kk], rnh[kk], cur + (uint32_t)q * 16u, acc);
#pragma unroll
                    for (int u = 0; u < V; ++u) Lsum[u] = (u & 1) ? hi_f(acc[u >> 1]) : lo_f(acc[u >> 1]);
                }
                if (!rok[kk]) continue;
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    const float L = Lsum[u] + rhr[kk] * fabsf(rphi[kk][u]);
                    const float phi2 = rphi[kk][u] * rphi[kk][u];
                    const float pw = pot_pow(rphi[kk][u], phi2, mhalf);
                    rp[kk][u] = rp[kk][u] - fmaf(cf.x, pw, cf.y * L);
                    rphi[kk][u] = fmaf(cf.z, rp[kk][u], rphi[kk][u]);
                }
                if constexpr (BF16) {
                    uint32_t pk[4];
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) {
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(rphi[kk][2 * k2], rphi[kk][2 * k2 + 1]);
                        pk[k2] = *reinterpret_cast<uint32_t*>(&b2);
                    }
                    sts128(nxt + re0[kk] * 2u, make_uint4(pk[0], pk[1], pk[2], pk[3]));
                    sts128(nxt + half_bytes + re0[kk] * 2u,
                           make_uint4(pk[0] ^ 0x80008000u, pk[1] ^ 0x80008000u, pk[2] ^ 0x80008000u,
                                      pk[3] ^ 0x80008000u));
                } else {
                    const uint4 f = make_uint4(__float_as_uint(rphi[kk][0]), __float_as_uint(rphi[kk][1]),
                                               __float_as_uint(rphi[kk][2]), __float_as_uint(rphi[kk][3]));
                    sts128(nxt + re0[kk] * 4u, f);
                    sts128(nxt + half_bytes + re0[kk] * 4u,
                           make_uint4(f.x ^ 0x80000000u, f.y ^ 0x80000000u, f.z ^ 0x80000000u,
                                      f.w ^ 0x80000000u));
                }
                if (in_win) {
#pragma unroll
                    for (int k4 = 0; k4 < V / 4; ++k4) {
                        float4* wp = reinterpret_cast<float4*>(gw + re0[kk] + 4 * k4);
                        float4 w = *wp;
                        w.x += rphi[kk][4 * k4]; w.y += rphi[kk][4 * k4 + 1];
                        w.z += rphi[kk][4 * k4 + 2]; w.w += rphi[kk][4 * k4 + 3];
                        *wp = w;
                    }
                }
            }
            __syncthreads();
        }
        // final state back to the shared layout the output code reads
        const uint32_t fin = op0 + (uint32_t)(a.S & 1) * buf_bytes;
#pragma unroll
        for (int kk = 0; kk < RS; ++kk) {
            if (!rok[kk]) continue;
#pragma unroll
            for (int k4 = 0; k4 < V / 4; ++k4) {
                const uint32_t o = (re0[kk] + 4 * k4) * 4u;
                sts128(ps + o, make_uint4(__float_as_uint(rp[kk][4 * k4]), __float_as_uint(rp[kk][4 * k4 + 1]),
                                          __float_as_uint(rp[kk][4 * k4 + 2]),
                                          __float_as_uint(rp[kk][4 * k4 + 3])));
                sts128((BF16 ? master : fin) + o,
                       make_uint4(__float_as_uint(rphi[kk][4 * k4]), __float_as_uint(rphi[kk][4 * k4 + 1]),
                                  __float_as_uint(rphi[kk][4 * k4 + 2]),
                                  __float_as_uint(rphi[kk][4 * k4 + 3])));
            }
        }
        __syncthreads();
    } else
    for (int64_t j = 0; j < a.S; ++j) {
        const float4 cf = __ldg(reinterpret_cast<const float4*>(a.sched) + j);
        const uint32_t cur = op0 + (uint32_t)(j & 1) * buf_bytes;
        const uint32_t nxt = op0 + (uint32_t)((j & 1) ^ 1) * buf_bytes;
        const bool in_win = j >= win0;
        for (int k = wbeg; k < wend; ++k) {
            const int t = __ldg(a.tuple_list + k);
            const int4 tp = __ldg(a.tuples + t);
            float Lsum[V];
            if constexpr (BF16) {
                tuple_field_bf16<G>(s0 + ((uint32_t)tp.x * G + g) * 16u, tp.y,
                                    cur + (uint32_t)q * 16u, Lsum);
            } else {
                uint64_t acc[NP];
                tuple_field_vec<G, BF16>(s0 + ((uint32_t)tp.x * G + g) * 16u, tp.y,
                                         cur + (uint32_t)q * 16u, acc);
#pragma unroll
                for (int u = 0; u < V; ++u) Lsum[u] = (u & 1) ? hi_f(acc[u >> 1]) : lo_f(acc[u >> 1]);
            }
            const int row = __ldg(a.tuple_rows + t * G + g);
            if (row < 0) continue;
            const uint32_t e0 = (uint32_t)(__ldg(a.slot_of_row + row) * RB + q * V);
            const float hr = a.h ? 2.f * __ldg(a.h + row) : 0.f;
            // this lane's V replicas of `row`, 16-byte vectors
            float phi[V], p[V];
#pragma unroll
            for (int k4 = 0; k4 < V / 4; ++k4) {
                const uint4 x = lds128((BF16 ? master : cur) + (e0 + 4 * k4) * 4u);
                const uint4 y = lds128(ps + (e0 + 4 * k4) * 4u);
                phi[4 * k4] = __uint_as_float(x.x); phi[4 * k4 + 1] = __uint_as_float(x.y);
                phi[4 * k4 + 2] = __uint_as_float(x.z); phi[4 * k4 + 3] = __uint_as_float(x.w);
                p[4 * k4] = __uint_as_float(y.x); p[4 * k4 + 1] = __uint_as_float(y.y);
                p[4 * k4 + 2] = __uint_as_float(y.z); p[4 * k4 + 3] = __uint_as_float(y.w);
            }
#pragma unroll
            for (int u = 0; u < V; ++u) {
                const float L = Lsum[u] + hr * fabsf(phi[u]);
                const float phi2 = phi[u] * phi[u];
                const float pw = pot_pow(phi[u], phi2, mhalf);
                p[u] = p[u] - fmaf(cf.x, pw, cf.y * L);
                phi[u] = fmaf(cf.z, p[u], phi[u]);
            }
#pragma unroll
            for (int k4 = 0; k4 < V / 4; ++k4) {
                const uint32_t o = (e0 + 4 * k4) * 4u;
                sts128(ps + o, make_uint4(__float_as_uint(p[4 * k4]), __float_as_uint(p[4 * k4 + 1]),
                                          __float_as_uint(p[4 * k4 + 2]), __float_as_uint(p[4 * k4 + 3])));
                const uint4 f = make_uint4(__float_as_uint(phi[4 * k4]), __float_as_uint(phi[4 * k4 + 1]),
                                           __float_as_uint(phi[4 * k4 + 2]), __float_as_uint(phi[4 * k4 + 3]));
                if constexpr (BF16) {
                    sts128(master + o, f);
                } else {
                    sts128(nxt + o, f);
                    sts128(nxt + half_bytes + o, make_uint4(f.x ^ 0x80000000u, f.y ^ 0x80000000u,
                                                            f.z ^ 0x80000000u, f.w ^ 0x80000000u));
                }
                if (in_win) {
                    float4* wp = reinterpret_cast<float4*>(gw + e0 + 4 * k4);
                    float4 w = *wp;
                    w.x += phi[4 * k4]; w.y += phi[4 * k4 + 1];
                    w.z += phi[4 * k4 + 2]; w.w += phi[4 * k4 + 3];
                    *wp = w;
                }
            }
            if constexpr (BF16) {
                // 8 BF16 values (16 bytes) into both halves of the next operand buffer
                uint32_t pk[4];
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) {
                    __nv_bfloat162 b2 = __floats2bfloat162_rn(phi[2 * k2], phi[2 * k2 + 1]);
                    pk[k2] = *reinterpret_cast<uint32_t*>(&b2);
                }
                sts128(nxt + e0 * 2u, make_uint4(pk[0], pk[1], pk[2], pk[3]));
                sts128(nxt + half_bytes + e0 * 2u,
                       make_uint4(pk[0] ^ 0x80008000u, pk[1] ^ 0x80008000u, pk[2] ^ 0x80008000u,
                                  pk[3] ^ 0x80008000u));
            }
        }
        __syncthreads();
    }

    // ---- outputs, [R][N] layout, coalesced over rows ----
    const uint32_t fin = op0 + (uint32_t)(a.S & 1) * buf_bytes;
    const int64_t nwin = a.S < a.W ? a.S : a.W;
    const float inv_w = 1.0f / (float)nwin;
    bool bad = false;
    for (int idx = threadIdx.x; idx < NRB; idx += blockDim.x) {
        const int rr = idx / a.N, row = idx % a.N, rep = rep0 + rr;
        if (rep >= a.R) continue;
        const uint32_t e = (uint32_t)(__ldg(a.slot_of_row + row) * RB + rr);
        float phi, p;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(phi) : "r"((BF16 ? master : fin) + e * 4u));
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(p) : "r"(ps + e * 4u));
        const float w = gw[e];
        const size_t o = (size_t)rep * a.N + row;
        if (a.phi_out) a.phi_out[o] = phi;
        if (a.p_out) a.p_out[o] = p;
        if (a.phibar_out) a.phibar_out[o] = w * inv_w;
        bad |= !(isfinite(phi) && isfinite(p));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, HQA_DEV_NONFINITE);
}

// Field only: L = J phi (+ 2 h |phi|) with the same gather code.
template <int RB, bool BF16>
__global__ void __launch_bounds__(kMaxThreads, 1) k_sparse_field_vec(const VArgs a)
{
    constexpr int ES = BF16 ? 2 : 4;
    constexpr int V = 16 / ES;
    constexpr int LPR = RB / V;
    constexpr int G = 32 / LPR;
    constexpr int NP = V / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t half_bytes = (uint32_t)a.Npad * RB * ES;
    const uint32_t op0 = s0 + a.ent_bytes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / LPR, q = lane % LPR;
    const int rep0 = blockIdx.x * RB;
    for (uint32_t o = threadIdx.x * 16u; o < a.ent_bytes; o += blockDim.x * 16u)
        sts128(s0 + o, __ldg(a.entries + o / 16u));
    for (uint32_t o = threadIdx.x * 16u; o < 2u * half_bytes; o += blockDim.x * 16u)
        sts128(op0 + o, make_uint4(0, 0, 0, 0));
    __syncthreads();
    for (int idx = threadIdx.x; idx < a.N * RB; idx += blockDim.x) {
        const int rr = idx / a.N, row = idx % a.N, rep = rep0 + rr;
        const float v = rep < a.R ? a.phi_in[(size_t)rep * a.N + row] : 0.f;
        const uint32_t e = (uint32_t)(__ldg(a.slot_of_row + row) * RB + rr);
        if constexpr (BF16) {
            sts16(op0 + e * 2u, bf16_bits(v));
            sts16(op0 + half_bytes + e * 2u, bf16_bits(-v));
        } else {
            sts32(op0 + e * 4u, v);
            sts32(op0 + half_bytes + e * 4u, -v);
        }
    }
    __syncthreads();
    const int wbeg = __ldg(a.warp_off + warp), wend = __ldg(a.warp_off + warp + 1);
    for (int k = wbeg; k < wend; ++k) {
        const int t = __ldg(a.tuple_list + k);
        const int4 tp = __ldg(a.tuples + t);
        float Lsum[V];
        if constexpr (BF16) {
            tuple_field_bf16<G>(s0 + ((uint32_t)tp.x * G + g) * 16u, tp.y, op0 + (uint32_t)q * 16u,
                                Lsum);
        } else {
            uint64_t acc[NP];
            tuple_field_vec<G, BF16>(s0 + ((uint32_t)tp.x * G + g) * 16u, tp.y,
                                     op0 + (uint32_t)q * 16u, acc);
#pragma unroll
            for (int u = 0; u < V; ++u) Lsum[u] = (u & 1) ? hi_f(acc[u >> 1]) : lo_f(acc[u >> 1]);
        }
        const int row = __ldg(a.tuple_rows + t * G + g);
        if (row < 0) continue;
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int rep = rep0 + q * V + u;
            if (rep >= a.R) continue;
            float L = Lsum[u];
            if (a.h) L += 2.f * __ldg(a.h + row) * fabsf(a.phi_in[(size_t)rep * a.N + row]);
            a.L_out[(size_t)rep * a.N + row] = L;
        }
    }
}

int vec_width(int prec) { return prec == HQA_PREC_BF16 ? 8 : 4; }

// ---------------------------------------------------------------------------
// host: plan construction
// ---------------------------------------------------------------------------

// Small deterministic generator for the local search (SplitMix64 stream).
struct HostRng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// One phase: P lanes-rows, each with a list of (entry code, bank group);
// K positions.  Bipartite multigraph rows x group copies: a group whose load
// exceeds K is split into ceil(load / K) copies (those are the only places a
// position can hold two rows of one group).  The graph is completed to a
// K-regular one with pad edges (reads of the group's zero row) and dummy
// rows, then peeled into K perfect matchings (Kuhn's augmenting paths); each
// matching is one position.  out[pos * G + g0 + g] receives the codes.
struct PhaseEntry {
    int code;
    int grp;
};

void colour_phase(const std::vector<std::vector<PhaseEntry>>& lists, int P, int K,
                  const std::vector<int>& zero_code, int G, int g0, std::vector<int>& out,
                  int64_t& wavefronts)
{
    std::vector<int> load(P, 0);
    for (int g = 0; g < P; ++g)
        for (auto& e : lists[g]) ++load[e.grp];
    std::vector<int> ncopy(P), copy_grp, first_copy(P);
    for (int q = 0; q < P; ++q) {
        ncopy[q] = std::max(1, (load[q] + K - 1) / K);
        first_copy[q] = (int)copy_grp.size();
        for (int k = 0; k < ncopy[q]; ++k) copy_grp.push_back(q);
    }
    const int C = (int)copy_grp.size();
    const int Rn = C;  // P real rows + (C - P) dummy rows
    // real edges per (row, copy): lists of codes
    std::vector<std::vector<std::vector<int>>> real(P, std::vector<std::vector<int>>(C));
    std::vector<int> cload(C, 0);
    for (int g = 0; g < P; ++g)
        for (auto& e : lists[g]) {
            int k = first_copy[e.grp];
            while (cload[k] >= K) ++k;  // fill copies of the group in order
            real[g][k].push_back(e.code);
            ++cload[k];
        }
    std::vector<std::vector<int>> M(Rn, std::vector<int>(C, 0));
    std::vector<int> rdef(Rn, K), cdef(C);
    for (int g = 0; g < P; ++g)
        for (int k = 0; k < C; ++k) {
            M[g][k] = (int)real[g][k].size();
            rdef[g] -= M[g][k];
        }
    for (int k = 0; k < C; ++k) cdef[k] = K - cload[k];
    std::vector<std::vector<int>> pads(P, std::vector<int>(C, 0));
    // pad edges of real rows go to single-copy groups first
    for (int pass = 0; pass < 2; ++pass)
        for (int g = 0; g < P; ++g)
            for (int k = 0; k < C && rdef[g] > 0; ++k) {
                if (pass == 0 && ncopy[copy_grp[k]] > 1) continue;
                const int m = std::min(rdef[g], cdef[k]);
                if (m <= 0) continue;
                M[g][k] += m;
                pads[g][k] += m;
                rdef[g] -= m;
                cdef[k] -= m;
            }
    for (int r = P; r < Rn; ++r)
        for (int k = 0; k < C && rdef[r] > 0; ++k) {
            const int m = std::min(rdef[r], cdef[k]);
            M[r][k] += m;
            rdef[r] -= m;
            cdef[k] -= m;
        }
    std::vector<int> match_c(C), cnt(P);
    std::vector<char> seen(C);
    std::function<bool(int)> augment = [&](int r) -> bool {
        for (int k = 0; k < C; ++k) {
            if (M[r][k] <= 0 || seen[k]) continue;
            seen[k] = 1;
            if (match_c[k] < 0 || augment(match_c[k])) {
                match_c[k] = r;
                return true;
            }
        }
        return false;
    };
    for (int pos = 0; pos < K; ++pos) {
        std::fill(match_c.begin(), match_c.end(), -1);
        for (int r = 0; r < Rn; ++r) {
            std::fill(seen.begin(), seen.end(), 0);
            augment(r);  // a regular bipartite multigraph always has a perfect matching
        }
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int k = 0; k < C; ++k) {
            const int r = match_c[k];
            if (r < 0) continue;
            --M[r][k];
            if (r >= P) continue;
            int code;
            if (!real[r][k].empty()) {
                code = real[r][k].back();
                real[r][k].pop_back();
            } else {
                --pads[r][k];
                code = zero_code[copy_grp[k]];
            }
            out[(size_t)pos * G + g0 + r] = code;
            ++cnt[copy_grp[k]];
        }
        wavefronts += std::max(1, *std::max_element(cnt.begin(), cnt.end()));
    }
}

}  // namespace

bool hqa_vec_supported(const hqa_ctx* ctx, int RB, int prec)
{
    if (!ctx->unit) return false;
    const int V = vec_width(prec);
    if (RB < V || RB > 32) return false;
    const int es = prec == HQA_PREC_BF16 ? 2 : 4;
    const int P = std::max(1, 128 / (RB * es));
    const int64_t Npad = ((int64_t)ctx->N + P - 1) / P * P + P;
    // u16 offsets in units of 16 bytes over both halves of a step buffer
    return 2 * Npad * RB * es / 16 < 65536;
}

static int64_t vec_npad(const hqa_ctx* ctx, int RB, int prec)
{
    const int es = prec == HQA_PREC_BF16 ? 2 : 4;
    const int P = std::max(1, 128 / (RB * es));
    return ((int64_t)ctx->N + P - 1) / P * P + P;
}

size_t hqa_vec_smem_bytes(const hqa_ctx* ctx, int RB, int prec, size_t ent_bytes)
{
    const int es = prec == HQA_PREC_BF16 ? 2 : 4;
    const size_t Npad = (size_t)vec_npad(ctx, RB, prec);
    size_t b = ent_bytes + 4 * Npad * RB * es;  // 2 step buffers x (+, -)
    if (prec == HQA_PREC_BF16) b += Npad * RB * 4;
    b += Npad * RB * 4;  // p
    return b;
}

hqa_status hqa_vec_plan(hqa_ctx* ctx, int RB, int prec, const SparsePlan** out)
{
    if (!hqa_vec_supported(ctx, RB, prec)) return HQA_ERR_UNSUPPORTED;
    const int key = 1000 + RB * 16 + prec;
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        *out = &it->second;
        return HQA_OK;
    }
    // building a plan allocates and uploads: not possible inside a capture
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    const int es = prec == HQA_PREC_BF16 ? 2 : 4;
    const int V = vec_width(prec);
    const int LPR = RB / V;
    const int G = 32 / LPR;
    const int P = std::max(1, 128 / (RB * es));   // rows per 8-lane phase
    const int N = ctx->N;
    const int Npad = (int)vec_npad(ctx, RB, prec);
    const int unit = RB * es / 16;                // one slot in 16-byte units
    // all neighbours of each row with their sign
    std::vector<std::vector<std::pair<int, bool>>> nb(N);
    for (int i = 0; i < N; ++i)
        for (int64_t k = ctx->row_ptr[i]; k < ctx->row_ptr[i + 1]; ++k)
            if (ctx->val[k] != 0.f) nb[i].emplace_back(ctx->col[k], ctx->val[k] < 0.f);
    std::vector<int> rows(N);
    std::iota(rows.begin(), rows.end(), 0);
    std::stable_sort(rows.begin(), rows.end(),
                     [&](int x, int y) { return nb[x].size() > nb[y].size(); });
    const int T = (N + G - 1) / G;
    const int nph = G / P;
    // ---- bank-group (slot residue) labels: a permutation of 0..P-1 per phase ----
    std::vector<int> grp(N), phase_of(N);
    const int nphases = T * nph;
    std::vector<std::vector<int>> phase_rows(nphases);
    for (int k = 0; k < N; ++k) {
        grp[rows[k]] = k % P;
        phase_of[rows[k]] = k / P;
        phase_rows[k / P].push_back(rows[k]);
    }
    // terms: (tuple, phase) -> loads per group, floor K of the tuple
    std::vector<int> termK(nphases);
    std::vector<int> termL((size_t)nphases * P, 0);
    std::vector<std::vector<int>> occ(N);
    for (int t = 0; t < T; ++t) {
        size_t K = 0;
        for (int g = 0; g < G && t * G + g < N; ++g) K = std::max(K, nb[rows[t * G + g]].size());
        for (int ph = 0; ph < nph; ++ph) termK[t * nph + ph] = (int)K;
    }
    for (int i = 0; i < N; ++i) {
        const int ti = phase_of[i];
        for (auto& e : nb[i]) {
            ++termL[(size_t)ti * P + grp[e.first]];
            occ[e.first].push_back(ti);
        }
    }
    auto term_cost = [&](int ti) {
        int m = termK[ti];
        for (int q = 0; q < P; ++q) m = std::max(m, termL[(size_t)ti * P + q]);
        return m;
    };
    if (P > 1) {
        HostRng rng{0x5EEDull + (uint64_t)N * 131 + (uint64_t)RB};
        const int64_t iters = (int64_t)40 * N;
        std::vector<int> touched;
        for (int64_t itn = 0; itn < iters; ++itn) {
            const auto& pr = phase_rows[rng.next() % (uint64_t)nphases];
            if (pr.size() < 2) continue;
            const int a = pr[rng.next() % pr.size()];
            int b = pr[rng.next() % pr.size()];
            if (a == b) continue;
            const int qa = grp[a], qb = grp[b];
            touched.clear();
            for (int ti : occ[a]) touched.push_back(ti);
            for (int ti : occ[b]) touched.push_back(ti);
            std::sort(touched.begin(), touched.end());
            touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
            int before = 0;
            for (int ti : touched) before += term_cost(ti);
            for (int ti : occ[a]) { --termL[(size_t)ti * P + qa]; ++termL[(size_t)ti * P + qb]; }
            for (int ti : occ[b]) { --termL[(size_t)ti * P + qb]; ++termL[(size_t)ti * P + qa]; }
            int after = 0;
            for (int ti : touched) after += term_cost(ti);
            if (after <= before) {
                grp[a] = qb;
                grp[b] = qa;
            } else {
                for (int ti : occ[a]) { ++termL[(size_t)ti * P + qa]; --termL[(size_t)ti * P + qb]; }
                for (int ti : occ[b]) { ++termL[(size_t)ti * P + qb]; --termL[(size_t)ti * P + qa]; }
            }
        }
    }
    // slots: group q's members at q, q + P, q + 2P, ...; zero rows at the end
    std::vector<int> slot_of_row(N), fill(P, 0);
    for (int k = 0; k < N; ++k) {
        const int r = rows[k];
        slot_of_row[r] = grp[r] + P * fill[grp[r]]++;
    }
    const int zero_base = Npad - P;   // slots zero_base .. zero_base + P - 1, group q at zero_base + q
    std::vector<int> zero_code(P);
    for (int q = 0; q < P; ++q) zero_code[q] = (zero_base + q) * unit;
    // ---- per tuple: K positions (multiple of 4), phases coloured ----
    struct Tup { int K; std::vector<int> codes; std::vector<int> trow; };
    std::vector<Tup> tups(T);
    int64_t wave = 0, ideal = 0, stored = 0;
    for (int t = 0; t < T; ++t) {
        Tup& u = tups[t];
        u.trow.assign(G, -1);
        size_t K = 0;
        for (int g = 0; g < G && t * G + g < N; ++g) {
            u.trow[g] = rows[t * G + g];
            K = std::max(K, nb[u.trow[g]].size());
        }
        u.K = (int)((K + 3) / 4 * 4);
        if (u.K == 0) u.K = 4;
        u.codes.assign((size_t)u.K * G, 0);
        for (int ph = 0; ph < nph; ++ph) {
            std::vector<std::vector<PhaseEntry>> lists(P);
            for (int gg = 0; gg < P; ++gg) {
                const int r = u.trow[ph * P + gg];
                if (r < 0) continue;
                for (auto& e : nb[r]) {
                    const int slot = slot_of_row[e.first];
                    lists[gg].push_back({(slot + (e.second ? Npad : 0)) * unit, grp[e.first]});
                }
            }
            colour_phase(lists, P, u.K, zero_code, G, ph * P, u.codes, wave);
        }
        ideal += (int64_t)u.K * nph;
        stored += (int64_t)u.K * G;
    }
    int64_t chunks = 0;
    for (auto& u : tups) chunks += (u.K / 4 + 1) / 2;
    std::vector<uint4> ent((size_t)std::max<int64_t>(chunks, 1) * G, make_uint4(0, 0, 0, 0));
    std::vector<int4> tpl(T);
    std::vector<int> trows((size_t)T * G);
    int64_t c0 = 0;
    for (int t = 0; t < T; ++t) {
        const Tup& u = tups[t];
        const int H = u.K / 4;
        tpl[t] = make_int4((int)c0, H, 0, 0);
        for (int g = 0; g < G; ++g) trows[(size_t)t * G + g] = u.trow[g];
        for (int c = 0; c < (H + 1) / 2; ++c)
            for (int g = 0; g < G; ++g) {
                uint32_t w[4];
                for (int k = 0; k < 4; ++k) {
                    uint32_t hv[2];
                    for (int hh = 0; hh < 2; ++hh) {
                        const int pos = c * 8 + 2 * k + hh;
                        hv[hh] = pos < u.K ? (uint32_t)u.codes[(size_t)pos * G + g] : 0u;
                    }
                    w[k] = hv[0] | (hv[1] << 16);
                }
                ent[(size_t)(c0 + c) * G + g] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        c0 += (H + 1) / 2;
    }
    // longest-processing-time assignment of tuples to warps
    const size_t ent_bytes = ent.size() * sizeof(uint4);
    std::vector<int> order(T);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return tups[x].K > tups[y].K; });
    int64_t total = 0;
    for (auto& u : tups) total += u.K;
    int bestNW = 1;
    double best_score = -1.0;
    std::vector<std::vector<int>> best_lists;
    // When a warp owns at most `cap` tuples (cap = 1, 2, 4, with at most
    // reg_threads(cap, bf16) threads) the state stays in registers; such assignments
    // are preferred whenever one exists, else warps are unconstrained.
    std::vector<std::pair<int, int>> cand;   // (NW, cap)
    for (int cap : {1, 2, 4})
        for (int NW = std::min(reg_threads(cap, prec == HQA_PREC_BF16) / 32, T);
             NW >= (T + cap - 1) / cap && NW >= 1; --NW)
            cand.push_back({NW, cap});
    const bool reg = !cand.empty();
    if (!reg)
        for (int NW = std::min(32, T); NW >= 1; --NW) cand.push_back({NW, 0});
    for (const auto& nc : cand) {
        const int NW = nc.first, cap = nc.second;
        std::vector<int64_t> ld(NW, 0);
        std::vector<std::vector<int>> lists(NW);
        for (int t : order) {
            int w = -1;
            for (int c = 0; c < NW; ++c)
                if ((cap == 0 || (int)lists[c].size() < cap) && (w < 0 || ld[c] < ld[w])) w = c;
            ld[w] += tups[t].K;
            lists[w].push_back(t);
        }
        const int64_t mk = *std::max_element(ld.begin(), ld.end());
        const double bal = (double)total / ((double)NW * (double)mk);
        // warps hide the shared-memory latency: on ER N=800 BF16, 25 warps at balance
        // 0.63 ran faster (21.1 ms) than 13 warps at 0.98 or 16 at 0.83 (21.6 ms)
        const double score = bal * std::min(1.0, NW / 24.0);
        if (score > best_score + 1e-9) {
            best_score = score;
            bestNW = NW;
            best_lists = lists;
        }
    }
    std::vector<int> woff(bestNW + 1, 0), tlist;
    int64_t mk = 1;
    int max_wt = 0;
    for (int w = 0; w < bestNW; ++w) {
        max_wt = std::max(max_wt, (int)best_lists[w].size());
        int64_t ld = 0;
        for (int t : best_lists[w]) {
            tlist.push_back(t);
            ld += tups[t].K;
        }
        mk = std::max(mk, ld);
        woff[w + 1] = (int)tlist.size();
    }
    SparsePlan pl;
    pl.vec = true;
    pl.RB = RB;
    pl.G = G;
    pl.T = T;
    pl.P = P;
    pl.Npad = Npad;
    pl.prec = prec;
    pl.chunks = chunks;
    pl.NW = bestNW;
    pl.ent_bytes = ent_bytes;
    pl.balance = (double)total / ((double)bestNW * (double)mk);
    pl.max_wt = max_wt;
    pl.pad_ratio = ctx->nnz > 0 ? (double)stored / (double)ctx->nnz : 0.0;
    pl.conflict_ratio = ideal > 0 ? (double)wave / (double)ideal : 1.0;
    HQA_CUDA_TRY(cudaMalloc(&pl.d_entries, ent_bytes));
    HQA_CUDA_TRY(cudaMalloc(&pl.d_tuples, tpl.size() * sizeof(int4)));
    HQA_CUDA_TRY(cudaMalloc(&pl.d_tuple_rows, trows.size() * sizeof(int)));
    HQA_CUDA_TRY(cudaMalloc(&pl.d_slot_of_row, (size_t)N * sizeof(int)));
    HQA_CUDA_TRY(cudaMalloc(&pl.d_warp_off, woff.size() * sizeof(int)));
    HQA_CUDA_TRY(cudaMalloc(&pl.d_tuple_list, std::max<size_t>(tlist.size(), 1) * sizeof(int)));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_entries, ent.data(), ent_bytes, cudaMemcpyHostToDevice));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_tuples, tpl.data(), tpl.size() * sizeof(int4), cudaMemcpyHostToDevice));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_tuple_rows, trows.data(), trows.size() * sizeof(int), cudaMemcpyHostToDevice));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_slot_of_row, slot_of_row.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice));
    HQA_CUDA_TRY(cudaMemcpy(pl.d_warp_off, woff.data(), woff.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!tlist.empty())
        HQA_CUDA_TRY(cudaMemcpy(pl.d_tuple_list, tlist.data(), tlist.size() * sizeof(int), cudaMemcpyHostToDevice));
    auto ins = ctx->plans.emplace(key, pl);
    *out = &ins.first->second;
    return HQA_OK;
}

template <int RB, bool BF16>
static cudaError_t launch_vec_md(const VArgs& a, int threads, size_t smem, cudaStream_t st)
{
    if (a.reg) {
        if (threads > reg_threads(a.reg, BF16)) return cudaErrorInvalidValue;
        const void* fn = a.reg == 1 ? (const void*)k_sparse_md_vec<RB, BF16, 1>
                       : a.reg == 2 ? (const void*)k_sparse_md_vec<RB, BF16, 2>
                                    : (const void*)k_sparse_md_vec<RB, BF16, 4>;
        cudaError_t e = hqa_smem_attr(fn, smem);
        if (e != cudaSuccess) return e;
        const int blocks = (a.R + RB - 1) / RB;
        if (a.reg == 1) k_sparse_md_vec<RB, BF16, 1><<<blocks, threads, smem, st>>>(a);
        else if (a.reg == 2) k_sparse_md_vec<RB, BF16, 2><<<blocks, threads, smem, st>>>(a);
        else k_sparse_md_vec<RB, BF16, 4><<<blocks, threads, smem, st>>>(a);
        return cudaGetLastError();
    }
    cudaError_t e = hqa_smem_attr((const void*)k_sparse_md_vec<RB, BF16, 0>, smem);
    if (e != cudaSuccess) return e;
    k_sparse_md_vec<RB, BF16, 0><<<(a.R + RB - 1) / RB, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int RB, bool BF16>
static cudaError_t launch_vec_field(const VArgs& a, int threads, size_t smem, cudaStream_t st)
{
    cudaError_t e = hqa_smem_attr((const void*)k_sparse_field_vec<RB, BF16>, smem);
    if (e != cudaSuccess) return e;
    k_sparse_field_vec<RB, BF16><<<(a.R + RB - 1) / RB, threads, smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t dispatch_vec(bool field, int RB, bool bf, const VArgs& a, int threads,
                                size_t smem, cudaStream_t st)
{
#define HQA_VEC_CASE(R_)                                                                    \
    if (RB == R_) {                                                                         \
        if (bf) return field ? launch_vec_field<R_, true>(a, threads, smem, st)             \
                             : launch_vec_md<R_, true>(a, threads, smem, st);               \
        return field ? launch_vec_field<R_, false>(a, threads, smem, st)                    \
                     : launch_vec_md<R_, false>(a, threads, smem, st);                      \
    }
    HQA_VEC_CASE(32)
    HQA_VEC_CASE(16)
    HQA_VEC_CASE(8)
    if (RB == 4 && !bf) return field ? launch_vec_field<4, false>(a, threads, smem, st)
                                     : launch_vec_md<4, false>(a, threads, smem, st);
#undef HQA_VEC_CASE
    return cudaErrorInvalidValue;
}

static VArgs common_args(const hqa_ctx* ctx, const SparsePlan* pl, int32_t R)
{
    VArgs a{};
    a.entries = pl->d_entries;
    a.tuples = pl->d_tuples;
    a.tuple_rows = pl->d_tuple_rows;
    a.slot_of_row = pl->d_slot_of_row;
    a.warp_off = pl->d_warp_off;
    a.tuple_list = pl->d_tuple_list;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.status = ctx->d_status;
    a.N = ctx->N;
    a.Npad = pl->Npad;
    a.T = pl->T;
    a.R = R;
    a.ent_bytes = (uint32_t)pl->ent_bytes;
    return a;
}

hqa_status hqa_vec_launch_md(hqa_ctx* ctx, const SparsePlan* pl, const StepCoef* d_sched,
                             int64_t S, int32_t W, int32_t R, uint64_t seed, int init,
                             const float* phi0, const float* p0, int M, float* phi_out,
                             float* p_out, float* phibar_out, cudaStream_t st)
{
    const size_t smem = hqa_vec_smem_bytes(ctx, pl->RB, pl->prec, pl->ent_bytes);
    if (smem > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    const int blocks = (R + pl->RB - 1) / pl->RB;
    hqa_status s = hqa_reserve(ctx, &ctx->d_state, &ctx->state_cap,
                               (size_t)blocks * pl->Npad * pl->RB * sizeof(float));
    if (s != HQA_OK) return s;
    VArgs a = common_args(ctx, pl, R);
    a.sched = d_sched;
    a.phi0 = phi0;
    a.p0 = p0;
    a.phi_out = phi_out;
    a.p_out = p_out;
    a.phibar_out = phibar_out;
    a.gwin = static_cast<float*>(ctx->d_state);
    a.reg = 0;
    for (int r : {1, 2, 4})
        if (a.reg == 0 && pl->max_wt <= r && pl->NW * 32 <= reg_threads(r, pl->prec == HQA_PREC_BF16))
            a.reg = r;
    a.seed = seed;
    a.S = S;
    a.W = W;
    a.M = M;
    a.init = init;
    cudaError_t e = dispatch_vec(false, pl->RB, pl->prec == HQA_PREC_BF16, a, pl->NW * 32, smem, st);
    return e == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_vec_launch_field(hqa_ctx* ctx, const SparsePlan* pl, int32_t R, const float* phi,
                                float* L, cudaStream_t st)
{
    const int es = pl->prec == HQA_PREC_BF16 ? 2 : 4;
    const size_t smem = pl->ent_bytes + 2 * (size_t)pl->Npad * pl->RB * es;
    if (smem > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    VArgs a = common_args(ctx, pl, R);
    a.phi_in = phi;
    a.L_out = L;
    cudaError_t e = dispatch_vec(true, pl->RB, pl->prec == HQA_PREC_BF16, a, pl->NW * 32, smem, st);
    return e == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}
