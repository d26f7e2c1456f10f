// dense_md_kernel.cuh -- the persistent tcgen05 dense MD kernel, shared by the
// translation units that instantiate it for a BF16 (dense_md.cu) and an FP16
// (dense_md_f16.cu) operand.  Both formats run the same kind::f16 MMA; they
// differ in the instruction descriptor's A/B format and in how phi and J are
// rounded to 16 bits (FP16 keeps 11 significant bits against BF16's 8, with
// phi scaled by 2^6 and J by 2^10 so that the low half of a split operand
// stays clear of FP16's subnormal range; both scales are powers of two and
// the accumulator is scaled back by 2^-16 exactly).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "hqa_internal.cuh"
#include "tc_ptx.cuh"

namespace hqa_dense {

constexpr int BM = 128;
constexpr int BK = 64;                  // one 128-byte swizzle row of 16-bit elements
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on any wait
constexpr float kF16PhiScale = 64.f;    // 2^6
constexpr float kF16JScale = 1024.f;    // 2^10
constexpr float kF16LScale = 1.f / 65536.f;

template <bool F16>
__device__ __forceinline__ uint16_t cvt16(float x)
{
    if constexpr (F16) return __half_as_ushort(__float2half_rn(x));
    else return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

template <bool F16>
__device__ __forceinline__ float from16(uint16_t u)
{
    if constexpr (F16) return __half2float(__ushort_as_half(u));
    else return __bfloat162float(__ushort_as_bfloat16(u));
}

// ===========================================================================
// Persistent dense MD kernel.
//
// Grid: Mt x Nc CTAs, all co-resident (cooperative launch), 1 per SM.  CTA
// (mt, nc) owns spin rows [128 mt, +128) and replica columns [2 NH nc, +2 NH),
// split into two halves h = 0, 1 of NH columns with their own TMEM
// accumulator.  Per leapfrog step m and half h:
//   producer  waits until all Mt CTAs of column group (nc, h) finished the
//             epilogue of (m-1, h) (arrival counter >= Mt m), then streams the
//             J and Phi^(m) k-tiles through the shared-memory ring;
//   MMA       waits for accumulator h to be drained, accumulates L = J Phi;
//   epilogue  12 warps read L from TMEM and do the kick and drift of Methods'
//             leapfrog on the FP32 state in global memory ([R][Npad], one
//             owner per element), write the 16-bit Phi^(m+1) into the other
//             buffer and the window sum, release accumulator h and arrive on
//             the counter.
// While the epilogue drains half h, the MMA of the other half runs.
//
// PAIR: the CTAs of row tiles 2t and 2t+1 of a column group form a 2-CTA
// cluster and share one M = 256 MMA per K slice (cta_group::2), issued by the
// even CTA.  Each CTA stages its own 128-row J tiles but only half of each
// phi tile (NH/2 replicas); the MMA reads the other half from the peer's
// shared memory, so an SM takes in a third (KSEG 2) or a quarter (KSEG 1)
// fewer operand bytes from L2 per MMA cycle.  The odd CTA's MMA warp relays
// each landed stage to the even CTA (remote mbarrier arrive); the MMA commits
// arrive on both CTAs' barriers; the odd CTA's epilogue warps release the
// accumulator on the even CTA's barrier.  Requires phi in TMEM.
// ===========================================================================
// 12 epilogue warps: three per TMEM lane quarter, each taking every third
// 16-column chunk (1.5% faster than 8 on K2000 x 4096 in FP16X2 and FP16)
constexpr int kEpiWarps = 12;              // a multiple of 4: each TMEM lane quarter alike
constexpr int kCS = kEpiWarps / 4;         // chunk stride: warps per lane quarter
constexpr int kMDThreads = 64 + 32 * kEpiWarps;

// phi in TMEM, split operand (two 16-bit tiles per chunk): the epilogue stages
// each chunk's operand values in shared memory and writes them with TMA bulk
// stores, a group of four warps (one per TMEM lane quarter) per 16 replicas x
// 128 spins tile: whole rows of the operand instead of one 64-byte fragment
// per warp store (K2000 x 4096 FP16X2: 92.4 -> 90.0 ms per 2000 steps; the
// one-tile FP16 operand measured slower, 63.0 -> 65.7 ms, and keeps plain stores).
constexpr bool kTmaStore = true;
constexpr uint32_t kStgBytes = 16 * 128 * 2;   // one staging tile [16 replicas][128 spins]

__device__ __forceinline__ void sts_u16(uint32_t a, uint16_t v)
{
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(v) : "memory");
}

// Split-operand epilogue arithmetic on pairs of elements (Blackwell's packed
// FP32 add/mul/fma, each lane of a pair rounded as the scalar operation).
constexpr bool kPackedEpilogue = true;

__device__ __forceinline__ uint64_t pk2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo2(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi2(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// a - b as a + (-b): the same IEEE result
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) { return add2(a, b ^ 0x8000000080000000ull); }

template <bool F16>
__device__ __forceinline__ uint32_t cvt16x2(float lo, float hi)   // lo -> bits 0-15
{
    return (uint32_t)cvt16<F16>(lo) | ((uint32_t)cvt16<F16>(hi) << 16);
}

struct DenseMDArgs {
    float* phi;              // [Rpad][Npad] FP32 master
    float* p;                // [Rpad][Npad]
    float* w;                // [Rpad][Npad] window sums
    uint16_t* phib;          // [2][Rpad][Npad] operand buffers (BF16 or FP16 bits)
    const StepCoef* sched;
    const float* h;          // [N] or null
    unsigned int* gbar;      // [2 Nc] arrival counters
    uint32_t* status;
    int64_t S;
    int W, N, Npad, Rpad, R, KT, Mt, M;
    int rep0;                // global index of this launch's first replica (random draws)
    float oscale;            // operand = 16-bit(phi * oscale): 1 (BF16), 2^6 (FP16)
    float lscale;            // L = accumulator * lscale: 1 (BF16), 2^-16 (FP16: J * 2^10)
    // armed check of the bounded-wait path (hqa_arm_wait_check): before step
    // wait_step every producer waits for *wait_flag != 0, at most wait_ns
    const unsigned int* wait_flag;
    int64_t wait_step;
    uint64_t wait_ns;
};

static __device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int NH, int STAGES, int KSEG, bool FUSED, bool ONCHIP, bool F16, int KSUB, bool PHIT,
          bool PAIR>
__global__ void __launch_bounds__(kMDThreads, 1)
k_dense_md(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmB,
           const __grid_constant__ CUtensorMap tmS, const DenseMDArgs a)
{
    // a ring stage holds KSUB consecutive 64-wide k-tiles: the KSUB J tiles,
    // then the KSUB phi tiles, then (FUSED, SHAREJ) the KSUB second phi tiles
    constexpr uint32_t A_BYTES = BM * BK * 2;
    constexpr int NB = PAIR ? NH / 2 : NH;   // rows of a phi tile staged by this CTA
    constexpr uint32_t B_BYTES = NB * BK * 2;
    // fused: one J tile per stage feeds the MMAs of both column halves.
    // SHAREJ (split phi against an exact J): one J tile per stage feeds the
    // MMAs of both K segments, phi_hi and phi_lo, into the same accumulator
    constexpr bool SHAREJ = KSEG == 2 && !FUSED;
    constexpr uint32_t STAGE_BYTES = KSUB * (A_BYTES + ((FUSED || SHAREJ) ? 2u : 1u) * B_BYTES);
    constexpr uint32_t B2_OFF = KSUB * (A_BYTES + B_BYTES);   // second phi tiles
    constexpr int NPASS = FUSED ? 1 : 2;   // MMA passes (and counters) per step
    // on-chip state: p in TMEM columns [2 NH, 4 NH), phi in shared memory
    constexpr uint32_t TMEM_COLS = ONCHIP ? 512u
                                 : 2 * NH <= 64 ? 64 : 2 * NH <= 128 ? 128 : 2 * NH <= 256 ? 256 : 512;
    static_assert(NH % 16 == 0 && NH <= 256, "UMMA N");
    static_assert(!ONCHIP || (NH <= 128 && !FUSED), "on-chip state: 4 NH TMEM columns");
    static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
    static_assert((KSUB == 1 || KSUB == 2 || KSUB == 4) && (KSUB == 1 || !FUSED), "k-tiles per stage");
    static_assert(!PHIT || ONCHIP, "phi in TMEM is an on-chip state form");
    static_assert(!PAIR || (PHIT && !FUSED), "pair form: phi in TMEM, separate halves");
    // TS: operand values leave through shared-memory staging tiles and TMA
    // stores (tmS: the operand buffers, box 128 spins x 16 replicas); NSEG
    // distinct tiles per chunk (phi_hi, and phi_lo for split operands)
    constexpr bool TS = PHIT && kTmaStore && KSEG != 1;
    constexpr int NSEG = KSEG == 1 ? 1 : 2;
    static_assert(B_BYTES % 1024 == 0 && 24 * STAGES + 48 <= 1024, "tile alignment, barrier block");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t bar = base + STAGES * STAGE_BYTES;
    const uint32_t full0 = bar, empty0 = bar + 8 * STAGES;
    const uint32_t accf0 = bar + 16 * STAGES, acce0 = accf0 + 16;
    const uint32_t tmem_slot = acce0 + 16;
    const uint32_t done_bar = acce0 + 24;             // PAIR: the last MMA completed
    const uint32_t pfull0 = bar + 16 * STAGES + 48;   // PAIR: the odd CTA's stage landed
    // ONCHIP: TMEM columns [2 NH, 4 NH) hold one state word of the tile's 2 NH
    // replicas: p, with phi in a shared-memory tile [2 NH columns][128 rows]
    // FP32 at phis; or (PHIT) phi, with p in global memory and the whole
    // shared memory left to the ring
    const uint32_t phis = bar + 1024;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x % a.Mt, nc = blockIdx.x / a.Mt;
    // PAIR: rank 0 (the even row tile) issues the MMAs; clusters are consecutive CTAs
    const uint32_t crank = PAIR ? tc::cluster_rank() : 0u;
    const int m0 = mt * BM, n0 = nc * 2 * NH;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(full0 + 8 * s, 1);
            tc::mbar_init(empty0 + 8 * s, 1);
        }
        for (int hh = 0; hh < 2; ++hh) {
            tc::mbar_init(accf0 + 8 * hh, 1);
            // PAIR: both CTAs' epilogue warps release the even CTA's accumulators
            tc::mbar_init(acce0 + 8 * hh, PAIR ? 2 * kEpiWarps : kEpiWarps);
        }
        if constexpr (PAIR) {
            tc::mbar_init(done_bar, 1);
            for (int s = 0; s < STAGES; ++s) tc::mbar_init(pfull0 + 8 * s, 1);
        }
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmJ);
        tc::prefetch_tmap(&tmB);
        if constexpr (TS) tc::prefetch_tmap(&tmS);
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            tc::tmem_alloc2(tmem_slot, TMEM_COLS);
            tc::tmem_relinquish2();
        } else {
            tc::tmem_alloc(tmem_slot, TMEM_COLS);
            tc::tmem_relinquish();
        }
    }
    tc::tc_fence_before();
    if constexpr (PAIR) tc::cluster_sync();   // the peer's barriers exist before any remote arrive
    else __syncthreads();
    tc::tc_fence_after();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(tmem_slot));
    volatile int* abort = &s_abort;
    volatile uint32_t* gstatus = a.status;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            uint32_t it = 0;
            for (int64_t m = 0; m < a.S && !*abort; ++m) {
                for (int hh = 0; hh < NPASS && !*abort; ++hh) {
                    if (a.wait_flag && m == a.wait_step && hh == 0) {
                        const uint64_t t0 = tc::globaltimer();
                        uint32_t spins = 0;
                        while (ld_acquire(a.wait_flag) == 0u) {
                            if ((++spins & 63u) == 0 && tc::globaltimer() - t0 > a.wait_ns) {
                                *abort = 1;
                                break;
                            }
                        }
                        if (*abort) break;
                    }
                    if (m > 0) {
                        const unsigned int* g = a.gbar + 2 * nc + hh;
                        const unsigned int target = (unsigned int)(a.Mt * m);
                        const uint64_t t0 = tc::globaltimer();
                        uint32_t spins = 0;
                        while (ld_acquire(g) < target) {
                            if ((++spins & 63u) == 0) {
                                if (*abort || (*gstatus & HQA_DEV_TIMEOUT)) { *abort = 1; break; }
                                if (tc::globaltimer() - t0 > kWaitNs) { *abort = 1; break; }
                            }
                        }
                        if (*abort) break;
                        tc::fence_proxy_async_global();
                    }
                    // PAIR: this CTA stages rows [NH/2 rank, +NH/2) of each phi tile
                    const int brow = (int)(m & 1) * a.Rpad + n0 + hh * NH + (int)crank * NB;
                    // split operands: K runs over [hi | hi | lo] against
                    // [J_hi | J_lo | J_hi] (KSEG 3); with KSEG 2 a stage holds the
                    // J tile and the hi and lo tiles of the same k (columns kt and
                    // Npad + kt of the [hi | lo] operand rows)
                    const int KTT = SHAREJ ? a.KT : KSEG * a.KT;   // a multiple of KSUB
                    for (int kt = 0; kt < KTT; kt += KSUB, ++it) {
                        const int s = it % STAGES;
                        if (it >= STAGES) {
                            const uint32_t ph = ((it / STAGES) - 1) & 1;   // PAIR: freed by the even CTA
                            if (!(PAIR ? tc::mbar_wait_cl(empty0 + 8 * s, ph, abort, kWaitNs)
                                       : tc::mbar_wait(empty0 + 8 * s, ph, abort, kWaitNs)))
                                break;
                        }
                        const uint32_t sa = base + s * STAGE_BYTES;
                        tc::mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
#pragma unroll
                        for (int u = 0; u < KSUB; ++u) {
                            const int k = (kt + u) * BK;
                            tc::tma_load_2d(sa + u * A_BYTES, &tmJ, k, m0, full0 + 8 * s);
                            tc::tma_load_2d(sa + KSUB * A_BYTES + u * B_BYTES, &tmB, k, brow,
                                            full0 + 8 * s);
                            if constexpr (FUSED)
                                tc::tma_load_2d(sa + B2_OFF + u * B_BYTES, &tmB, k, brow + NH,
                                                full0 + 8 * s);
                            if constexpr (SHAREJ)
                                tc::tma_load_2d(sa + B2_OFF + u * B_BYTES, &tmB, a.Npad + k, brow,
                                                full0 + 8 * s);
                        }
                    }
                }
            }
            // drain: every issued stage must land before the CTA can exit
            if (*abort)
                for (uint32_t k = (it > STAGES ? it - STAGES : 0); k < it; ++k)
                    tc::mbar_wait(full0 + 8 * (k % STAGES), (k / STAGES) & 1, abort, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0 && PAIR && crank != 0) {
            // ---- PAIR, odd CTA: relay each landed stage to the MMA issuer ----
            uint32_t it = 0;
            const uint32_t peer_pfull0 = tc::mapa(pfull0, 0);
            for (int64_t m = 0; m < a.S && !*abort; ++m)
                for (int hh = 0; hh < NPASS && !*abort; ++hh) {
                    const int KTT = SHAREJ ? a.KT : KSEG * a.KT;
                    for (int kt = 0; kt < KTT; kt += KSUB, ++it) {
                        const int s = it % STAGES;
                        if (!tc::mbar_wait(full0 + 8 * s, (it / STAGES) & 1, abort, kWaitNs)) break;
                        tc::mbar_arrive_remote(peer_pfull0 + 8 * s);
                    }
                }
        } else if (lane == 0) {
            // ---- MMA issuer ----
            constexpr int MM = PAIR ? 2 * BM : BM;
            constexpr uint32_t idesc = F16 ? tc::idesc_f16(MM, NH) : tc::idesc_bf16(MM, NH);
            uint32_t it = 0;
            for (int64_t m = 0; m < a.S && !*abort; ++m) {
                for (int hh = 0; hh < NPASS && !*abort; ++hh) {
                    if (m > 0) {
                        const uint32_t ph = (uint32_t)((m - 1) & 1);
                        if (!(PAIR ? tc::mbar_wait_cl(acce0 + 8 * hh, ph, abort, kWaitNs)
                                   : tc::mbar_wait(acce0 + 8 * hh, ph, abort, kWaitNs)))
                            break;
                    }
                    tc::tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(hh * NH);
                    const int KTT = SHAREJ ? a.KT : KSEG * a.KT;
                    for (int kt = 0; kt < KTT; kt += KSUB, ++it) {
                        const int s = it % STAGES;
                        if (!tc::mbar_wait(full0 + 8 * s, (it / STAGES) & 1, abort, kWaitNs)) break;
                        if (PAIR && !tc::mbar_wait_cl(pfull0 + 8 * s, (it / STAGES) & 1, abort, kWaitNs))
                            break;
                        tc::tc_fence_after();
                        const uint32_t sa = base + s * STAGE_BYTES;
                        if constexpr (PAIR) {
#pragma unroll
                            for (int u = 0; u < KSUB; ++u) {
                                const uint64_t ad = tc::sdesc_k128(sa + u * A_BYTES);
                                const uint64_t bd = tc::sdesc_k128(sa + KSUB * A_BYTES + u * B_BYTES);
                                const bool first = (kt | u) == 0;
#pragma unroll
                                for (int kk = 0; kk < BK / 16; ++kk)
                                    tc::mma2_f16(d, ad + 2 * kk, bd + 2 * kk, idesc, !(first && kk == 0));
                                if constexpr (SHAREJ) {
                                    const uint64_t bd1 = tc::sdesc_k128(sa + B2_OFF + u * B_BYTES);
#pragma unroll
                                    for (int kk = 0; kk < BK / 16; ++kk)
                                        tc::mma2_f16(d, ad + 2 * kk, bd1 + 2 * kk, idesc, 1u);
                                }
                            }
                            tc::mma_commit2(empty0 + 8 * s, 3);   // both CTAs' stage s is free
                            continue;
                        }
#pragma unroll
                        for (int u = 0; u < KSUB; ++u) {
                            const uint64_t ad = tc::sdesc_k128(sa + u * A_BYTES);
                            const uint64_t bd = tc::sdesc_k128(sa + KSUB * A_BYTES + u * B_BYTES);
                            const bool first = (kt | u) == 0;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk)
                                tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, !(first && kk == 0));
                            if constexpr (FUSED) {
                                const uint64_t bd1 = tc::sdesc_k128(sa + B2_OFF + u * B_BYTES);
#pragma unroll
                                for (int kk = 0; kk < BK / 16; ++kk)
                                    tc::mma_bf16(d + (uint32_t)NH, ad + 2 * kk, bd1 + 2 * kk, idesc,
                                                 !(first && kk == 0));
                            }
                            if constexpr (SHAREJ) {   // J phi_lo into the same accumulator
                                const uint64_t bd1 = tc::sdesc_k128(sa + B2_OFF + u * B_BYTES);
#pragma unroll
                                for (int kk = 0; kk < BK / 16; ++kk)
                                    tc::mma_bf16(d, ad + 2 * kk, bd1 + 2 * kk, idesc, 1u);
                            }
                        }
                        tc::mma_commit(empty0 + 8 * s);
                    }
                    if constexpr (PAIR) tc::mma_commit2(accf0 + 8 * hh, 3);
                    else tc::mma_commit(accf0 + 8 * hh);
                }
            }
            if constexpr (PAIR) {
                // every MMA issued (into both CTAs' TMEM, from both CTAs' shared
                // memory) completes before either CTA frees them
                volatile int no_abort = 0;   // waited for even after an abort
                tc::mma_commit2(done_bar, 1);
                tc::mbar_wait_cl(done_bar, 0, &no_abort, kWaitNs);
            }
        }
    } else {
        // ---- epilogue warps: kick, drift, BF16 shadow, window ----
        const int ew = warp - 2;              // 0 .. kEpiWarps - 1
        const int quarter = warp & 3;         // TMEM lanes 32*quarter .. +31
        const int csel = ew >> 2;             // first chunk of this warp (chunks csel + kCS k)
        const int row = m0 + 32 * quarter + lane;
        const bool row_ok = row < a.N;
        const float hr = (a.h && row_ok) ? 2.f * a.h[row] : 0.f;
        const int mhalf = (a.M - 2) / 2;
        const int64_t win0 = a.S - (int64_t)a.W;
        const uint32_t tl = (uint32_t)(32 * quarter) << 16;   // this warp's TMEM lanes
        const uint32_t rloc = (uint32_t)(32 * quarter + lane);  // row within the tile
        // PAIR, odd CTA: accumulators are released on the even CTA's barrier
        const uint32_t acce_to = (PAIR && crank != 0) ? tc::mapa(acce0, 0) : acce0;
        // TS: the four warps sharing csel (one per lane quarter) form a group with
        // named barrier 2 + csel and staging tiles at stg; its first warp's lane 0
        // issues the group's TMA stores
        const uint32_t stg = bar + 1024 + (uint32_t)(csel * NSEG) * kStgBytes;
        const bool gleader = (ew & 3) == 0 && lane == 0;
        if constexpr (ONCHIP) {
            // the tile's state moves on chip for the whole trajectory
            for (int hh = 0; hh < 2; ++hh)
                for (int c = csel; c < NH / 16; c += kCS) {
                    const int col = hh * NH + c * 16;
                    uint32_t pv[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const size_t o = (size_t)(n0 + col + j) * a.Npad + row;
                        if constexpr (PHIT) {
                            pv[j] = __float_as_uint(a.phi[o]);
                        } else {
                            asm volatile("st.shared.f32 [%0], %1;"
                                         ::"r"(phis + (uint32_t)(col + j) * 512u + rloc * 4u), "f"(a.phi[o]));
                            pv[j] = __float_as_uint(a.p[o]);
                        }
                    }
                    tc::tmem_st16(tmem + tl + (uint32_t)(2 * NH + col), pv);
                }
            tc::tmem_wait_st();
        }
        bool stop = false;
        for (int64_t m = 0; m < a.S && !stop; ++m) {
            const float4 cf = __ldg(reinterpret_cast<const float4*>(a.sched) + m);
            const bool in_win = m >= win0;
            const int Kb = KSEG * a.Npad;   // operand row: [hi], [hi | lo] or [hi | hi | lo]
            uint16_t* nb = a.phib + (size_t)((m + 1) & 1) * a.Rpad * Kb;
            bool ok = true;
            for (int hh = 0; hh < 2 && !stop; ++hh) {
                // the state of this warp's first chunk does not depend on the MMA:
                // its loads are in flight while the accumulator is computed
                float ph[16], pp[16];
                if ((!ONCHIP || PHIT) && row_ok && csel < NH / 16) {
                    const int rb0 = n0 + hh * NH + csel * 16;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const size_t o = (size_t)(rb0 + j) * a.Npad + row;
                        if constexpr (!ONCHIP) ph[j] = a.phi[o];
                        pp[j] = a.p[o];
                    }
                }
                const int pass = FUSED ? 0 : hh;
                if (!FUSED || hh == 0) {
                    ok = __all_sync(0xffffffffu,
                                    PAIR ? tc::mbar_wait_cl(accf0 + 8 * pass, (uint32_t)(m & 1), abort, kWaitNs)
                                         : tc::mbar_wait(accf0 + 8 * pass, (uint32_t)(m & 1), abort, kWaitNs));
                    tc::tc_fence_after();
                    // the group enters the chunk loop (and its barriers) together
                    if constexpr (TS) ok = tc::named_bar_and(2 + csel, 128, ok);
                }
                if (ok && PHIT) {
                    // phi in TMEM next to the accumulators, p in global memory
#pragma unroll 1
                    for (int c = csel; c < NH / 16; c += kCS) {
                        const int col = hh * NH + c * 16;
                        uint32_t v[16], fv[16];
                        tc::tmem_ld16(tmem + tl + (uint32_t)col, v);
                        tc::tmem_ld16(tmem + tl + (uint32_t)(2 * NH + col), fv);
                        // the next chunk's momenta load while this chunk updates
                        float npp[16];
                        const bool more = row_ok && c + kCS < NH / 16;
                        if (more) {
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                npp[j] = a.p[(size_t)(n0 + col + 16 * kCS + j) * a.Npad + row];
                        }
                        if constexpr (TS) {
                            // the group's staging tiles are free once the stores of
                            // its previous chunk have read them
                            if (gleader) tc::bulk_wait_read0();
                            tc::named_bar(2 + csel, 128);
                        }
                        tc::tmem_wait_ld();
                        if (TS && kPackedEpilogue && row_ok) {
                            // pairs of replica columns: L = hr |phi| + acc lscale (fused),
                            // then the kick, drift, split and stores as below
                            const uint64_t ls2 = pk2(a.lscale, a.lscale), hr2 = pk2(hr, hr);
                            const uint64_t cx2 = pk2(cf.x, cf.x), cy2 = pk2(cf.y, cf.y);
                            const uint64_t cz2 = pk2(cf.z, cf.z), os2 = pk2(a.oscale, a.oscale);
#pragma unroll
                            for (int j = 0; j < 16; j += 2) {
                                const size_t o0 = (size_t)(n0 + col + j) * a.Npad + row;
                                const size_t o1 = o0 + a.Npad;
                                const uint64_t f2 = pk2(__uint_as_float(fv[j]), __uint_as_float(fv[j + 1]));
                                const uint64_t af2 = f2 & 0x7fffffff7fffffffull;   // |phi|
                                const uint64_t L2 = fma2(hr2, af2, mul2(pk2(__uint_as_float(v[j]),
                                                                            __uint_as_float(v[j + 1])), ls2));
                                const uint64_t sq2 = mul2(f2, f2);
                                uint64_t pw2 = f2;
#pragma unroll
                                for (int q = 0; q < kMaxMHalf; ++q)
                                    if (q < mhalf) pw2 = mul2(pw2, sq2);
                                const uint64_t pn2 = sub2(pk2(pp[j], pp[j + 1]), fma2(cx2, pw2, mul2(cy2, L2)));
                                const uint64_t fn2 = fma2(cz2, pn2, f2);
                                a.p[o0] = lo2(pn2);
                                a.p[o1] = hi2(pn2);
                                fv[j] = __float_as_uint(lo2(fn2));
                                fv[j + 1] = __float_as_uint(hi2(fn2));
                                const uint64_t fs2 = mul2(fn2, os2);
                                const uint32_t h2 = cvt16x2<F16>(lo2(fs2), hi2(fs2));
                                const uint64_t r2 = sub2(fs2, pk2(from16<F16>((uint16_t)h2),
                                                                  from16<F16>((uint16_t)(h2 >> 16))));
                                const uint32_t l2 = cvt16x2<F16>(lo2(r2), hi2(r2));
                                const uint32_t sb = stg + (uint32_t)(j * 128) * 2u + rloc * 2u;
                                sts_u16(sb, (uint16_t)h2);
                                sts_u16(sb + 256u, (uint16_t)(h2 >> 16));
                                sts_u16(sb + kStgBytes, (uint16_t)l2);
                                sts_u16(sb + kStgBytes + 256u, (uint16_t)(l2 >> 16));
                                if (in_win) {
                                    a.w[o0] += lo2(fn2);
                                    a.w[o1] += hi2(fn2);
                                }
                            }
                        } else if (row_ok) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const size_t o = (size_t)(n0 + col + j) * a.Npad + row;
                                const float f = __uint_as_float(fv[j]);
                                const float L = __uint_as_float(v[j]) * a.lscale + hr * fabsf(f);
                                const float phi2 = f * f;
                                const float pw = pot_pow(f, phi2, mhalf);
                                const float pn = pp[j] - fmaf(cf.x, pw, cf.y * L);
                                const float fn = fmaf(cf.z, pn, f);
                                a.p[o] = pn;
                                fv[j] = __float_as_uint(fn);
                                const float fs = fn * a.oscale;
                                const uint16_t hi = cvt16<F16>(fs);
                                if constexpr (TS) {
                                    const uint32_t sb = stg + (uint32_t)(j * 128) * 2u + rloc * 2u;
                                    sts_u16(sb, hi);
                                    if constexpr (KSEG != 1)
                                        sts_u16(sb + kStgBytes, cvt16<F16>(fs - from16<F16>(hi)));
                                } else {
                                    const size_t ob = (size_t)(n0 + col + j) * Kb + row;
                                    nb[ob] = hi;
                                    if (KSEG == 2) nb[ob + a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
                                    if (KSEG == 3) {
                                        nb[ob + a.Npad] = hi;
                                        nb[ob + 2 * a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
                                    }
                                }
                                if (in_win) a.w[o] += fn;
                            }
                        } else if constexpr (TS) {
                            // spin rows beyond N keep a zero operand
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const uint32_t sb = stg + (uint32_t)(j * 128) * 2u + rloc * 2u;
                                sts_u16(sb, 0);
                                if constexpr (KSEG != 1) sts_u16(sb + kStgBytes, 0);
                            }
                        }
                        // .sync.aligned: every lane of the warp, outside the row_ok branch
                        tc::tmem_st16(tmem + tl + (uint32_t)(2 * NH + col), fv);
                        tc::tmem_wait_st();
                        if constexpr (TS) {
                            tc::fence_proxy_async_smem();
                            tc::named_bar(2 + csel, 128);
                            if (gleader) {
                                const int y = (int)((m + 1) & 1) * a.Rpad + n0 + col;
                                tc::tma_store_2d(&tmS, m0, y, stg);
                                if (KSEG == 2) tc::tma_store_2d(&tmS, a.Npad + m0, y, stg + kStgBytes);
                                if (KSEG == 3) {
                                    tc::tma_store_2d(&tmS, a.Npad + m0, y, stg);
                                    tc::tma_store_2d(&tmS, 2 * a.Npad + m0, y, stg + kStgBytes);
                                }
                                tc::bulk_commit();
                            }
                        }
                        if (more) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) pp[j] = npp[j];
                        }
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (PAIR && crank != 0) tc::mbar_arrive_remote(acce_to + 8 * pass);
                        else tc::mbar_arrive(acce0 + 8 * pass);
                    }
                } else if (ok && ONCHIP) {
#pragma unroll 1
                    for (int c = csel; c < NH / 16; c += kCS) {
                        const int col = hh * NH + c * 16;
                        uint32_t v[16], pv[16];
                        tc::tmem_ld16(tmem + tl + (uint32_t)col, v);
                        tc::tmem_ld16(tmem + tl + (uint32_t)(2 * NH + col), pv);
                        float phl[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            asm volatile("ld.shared.f32 %0, [%1];"
                                         : "=f"(phl[j]) : "r"(phis + (uint32_t)(col + j) * 512u + rloc * 4u));
                        tc::tmem_wait_ld();
                        if (row_ok) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float L = __uint_as_float(v[j]) * a.lscale + hr * fabsf(phl[j]);
                                const float phi2 = phl[j] * phl[j];
                                const float pw = pot_pow(phl[j], phi2, mhalf);
                                const float pn = __uint_as_float(pv[j]) - fmaf(cf.x, pw, cf.y * L);
                                const float fn = fmaf(cf.z, pn, phl[j]);
                                pv[j] = __float_as_uint(pn);
                                asm volatile("st.shared.f32 [%0], %1;"
                                             ::"r"(phis + (uint32_t)(col + j) * 512u + rloc * 4u), "f"(fn));
                                const size_t ob = (size_t)(n0 + col + j) * Kb + row;
                                const float fs = fn * a.oscale;
                                const uint16_t hi = cvt16<F16>(fs);
                                nb[ob] = hi;
                                if (KSEG == 2) nb[ob + a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
                                if (KSEG == 3) {
                                    nb[ob + a.Npad] = hi;
                                    nb[ob + 2 * a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
                                }
                                if (in_win) a.w[(size_t)(n0 + col + j) * a.Npad + row] += fn;
                            }
                        }
                        // .sync.aligned: every lane of the warp, outside the row_ok branch
                        tc::tmem_st16(tmem + tl + (uint32_t)(2 * NH + col), pv);
                        tc::tmem_wait_st();
                    }
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(acce0 + 8 * pass);
                } else if (ok) {
#pragma unroll 1
                    for (int c = csel; c < NH / 16; c += kCS) {
                        uint32_t v[16];
                        tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(hh * NH + c * 16), v);
                        // the next chunk's state loads overlap this chunk's update
                        float nph[16], npp[16];
                        const bool more = row_ok && c + kCS < NH / 16;
                        if (more) {
                            const int rb1 = n0 + hh * NH + (c + kCS) * 16;
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const size_t o = (size_t)(rb1 + j) * a.Npad + row;
                                nph[j] = a.phi[o];
                                npp[j] = a.p[o];
                            }
                        }
                        tc::tmem_wait_ld();
                        if (row_ok) {
                            const int rbase = n0 + hh * NH + c * 16;
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const size_t o = (size_t)(rbase + j) * a.Npad + row;
                                const float L = __uint_as_float(v[j]) * a.lscale + hr * fabsf(ph[j]);
                                const float phi2 = ph[j] * ph[j];
                                const float pw = pot_pow(ph[j], phi2, mhalf);
                                const float pn = pp[j] - fmaf(cf.x, pw, cf.y * L);
                                const float fn = fmaf(cf.z, pn, ph[j]);
                                a.p[o] = pn;
                                a.phi[o] = fn;
                                const size_t ob = (size_t)(rbase + j) * Kb + row;
                                const float fs = fn * a.oscale;
                                const uint16_t hi = cvt16<F16>(fs);
                                nb[ob] = hi;
                                if (KSEG == 2) nb[ob + a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
                                if (KSEG == 3) {
                                    nb[ob + a.Npad] = hi;
                                    nb[ob + 2 * a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
                                }
                                if (in_win) a.w[o] += fn;
                            }
                        }
                        if (more) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                ph[j] = nph[j];
                                pp[j] = npp[j];
                            }
                        }
                    }
                    // the accumulator may be overwritten once every epilogue warp has read it
                    if (!FUSED || hh == 1) {
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(acce0 + 8 * pass);
                    }
                }
                if (FUSED && hh == 0) continue;
                // TS: this half's operand stores complete in global memory
                if constexpr (TS) {
                    if (gleader) tc::bulk_wait0();
                }
                // Phi^(m+1) of this half -> visible to the other CTAs' TMA loads
                tc::fence_proxy_async_global();
                // all epilogue warps meet here every half-step; the barrier also
                // ORs the abort flags so every warp leaves at the same point
                uint32_t any;
                asm volatile(
                    "{\n\t.reg .pred q, r;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                    "barrier.red.or.pred r, 1, %2, q;\n\tselp.u32 %0, 1, 0, r;\n\t}"
                    : "=r"(any) : "r"((uint32_t)(!ok || *abort)), "n"(32 * kEpiWarps) : "memory");
                if (any) {
                    *abort = 1;
                    stop = true;
                } else if (ew == 0 && lane == 0) {
                    __threadfence();
                    atomicAdd(a.gbar + 2 * nc + pass, 1u);
                }
            }
        }
        if constexpr (ONCHIP) {
            // final state back to global memory (the output kernel reads it there)
            for (int hh = 0; hh < 2; ++hh)
                for (int c = csel; c < NH / 16; c += kCS) {
                    const int col = hh * NH + c * 16;
                    uint32_t pv[16];
                    tc::tmem_ld16(tmem + tl + (uint32_t)(2 * NH + col), pv);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const size_t o = (size_t)(n0 + col + j) * a.Npad + row;
                        if constexpr (PHIT) {   // p is already in global memory
                            a.phi[o] = __uint_as_float(pv[j]);
                        } else {
                            float f;
                            asm volatile("ld.shared.f32 %0, [%1];"
                                         : "=f"(f) : "r"(phis + (uint32_t)(col + j) * 512u + rloc * 4u));
                            a.phi[o] = f;
                            a.p[o] = __uint_as_float(pv[j]);
                        }
                    }
                }
        }
    }
    tc::tc_fence_before();
    __syncwarp();
    // PAIR: neither CTA frees its shared memory or TMEM while the pair's MMAs
    // or remote arrives may still touch them
    if constexpr (PAIR) tc::cluster_sync();
    else __syncthreads();
    if (*abort && threadIdx.x == 0) atomicOr(a.status, HQA_DEV_TIMEOUT);
    if (warp == 1) {
        tc::tc_fence_after();
        if constexpr (PAIR) tc::tmem_dealloc2(tmem, TMEM_COLS);
        else tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// State set-up: phi(0), p(0) (SplitMix64 or caller-given), window 0, BF16
// operand buffer 0; padding rows/replicas zero in every array.
template <bool F16>
__global__ void k_dense_init(DenseMDArgs a, uint64_t seed, int init, const float* phi0,
                             const float* p0, int kseg)
{
    const int Kb = kseg * a.Npad;
    const size_t total = (size_t)a.Rpad * a.Npad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / a.Npad), i = (int)(idx % a.Npad);
        float phi = 0.f, p = 0.f;
        if (r < a.R && i < a.N) {
            const uint64_t c = ((uint64_t)(a.rep0 + r) << 32) | (uint64_t)i;
            if (init == HQA_INIT_GIVEN) {
                phi = phi0[(size_t)r * a.N + i];
                p = p0[(size_t)r * a.N + i];
            } else {
                uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;  // SplitMix64
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                z ^= z >> 31;
                p = (z >> 63) ? -1.f : 1.f;
                if (init == HQA_INIT_RANDOM_FLUX) {
                    uint64_t y = seed + ((c | (1ull << 62)) + 1ull) * 0x9E3779B97F4A7C15ull;
                    y = (y ^ (y >> 30)) * 0xBF58476D1CE4E5B9ull;
                    y = (y ^ (y >> 27)) * 0x94D049BB133111EBull;
                    y ^= y >> 31;
                    phi = (float)((int64_t)(y >> 40) - (1 << 23)) * 0x1p-26f;
                }
            }
        }
        a.phi[idx] = phi;
        a.p[idx] = p;
        a.w[idx] = 0.f;
        const size_t ob = (size_t)r * Kb + i;
        const size_t buf = (size_t)a.Rpad * Kb;
        const float fs = phi * a.oscale;
        const uint16_t hi = cvt16<F16>(fs);
        a.phib[ob] = hi;
        a.phib[buf + ob] = 0;   // +0 in both formats
        if (kseg == 2) {
            a.phib[ob + a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
            a.phib[buf + ob + a.Npad] = 0;
        }
        if (kseg == 3) {
            a.phib[ob + a.Npad] = hi;
            a.phib[ob + 2 * a.Npad] = cvt16<F16>(fs - from16<F16>(hi));
            a.phib[buf + ob + a.Npad] = 0;
            a.phib[buf + ob + 2 * a.Npad] = 0;
        }
    }
}

static __global__ void k_dense_out(DenseMDArgs a, float inv_w, float* phi_out, float* p_out,
                            float* phibar_out)
{
    const size_t total = (size_t)a.R * a.N;
    bool bad = false;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / a.N), i = (int)(idx % a.N);
        const size_t o = (size_t)r * a.Npad + i;
        const float phi = a.phi[o], p = a.p[o];
        if (phi_out) phi_out[idx] = phi;
        if (p_out) p_out[idx] = p;
        if (phibar_out) phibar_out[idx] = a.w[o] * inv_w;
        bad |= !(isfinite(phi) && isfinite(p));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, HQA_DEV_NONFINITE);
}

// Shared memory after the barrier block: the phi tile (on chip, not PHIT) or
// the epilogue's operand staging tiles (PHIT with TMA stores).
constexpr int md_tail(int nh, int kseg, bool onchip, bool phit)
{
    return onchip && !phit ? 2 * nh * BM * 4
         : phit && kTmaStore && kseg != 1 ? kCS * 2 * (int)kStgBytes
                             : 0;
}

template <int NH, int STAGES, bool TWOB, int KSUB, bool PAIR, int TAIL>
size_t md_smem()
{
    // alignment slack, ring (KSUB J tiles and KSUB or 2 KSUB phi tiles per
    // stage, a pair's CTA staging half of each phi tile), barrier block
    // (1 KB), tail
    constexpr int NB = PAIR ? NH / 2 : NH;
    return 1024 + (size_t)STAGES * KSUB * (BM * BK * 2 + (TWOB ? 2 : 1) * NB * BK * 2) + 1024 + TAIL;
}

// The tile's state (phi, p) stays on chip for the whole trajectory when its
// p fits next to the accumulators in TMEM (4 NH <= 512 columns) and its phi
// next to at least 3 ring stages in shared memory.
constexpr bool onchip_ok(int nh) { return nh <= 128; }

// Fused halves (both column halves from one J tile per stage, which halves the
// J stream from L2, the epilogue draining both halves after one accumulator
// wait) measured slower on K2000 x 2048 replicas (57 vs 40 us per step): the
// epilogue of one half no longer overlaps the MMA of the other.  Kept as an
// option, off.
constexpr bool kFusedHalves = false;

// Ring depth: as many stages as fit in the 227 KB opt-in shared memory next to
// the alignment slack, the barrier block and the on-chip phi tile, at most 4.
// Deeper rings measured no faster on K2000 x 4096: with the state in global
// memory instead (freeing the 128 KB phi tile), 4 and 7 stages ran FP16X2 in
// 115.5 ms per 2000 steps against 114.2 on chip, FP16 in 84.3 and 87.6 against 77.8.
constexpr int md_stages(int nh, bool twob, int tail, int ksub, bool phit, bool pair)
{
    const int stage = ksub * (BM * BK * 2 + (twob ? 2 : 1) * (pair ? nh / 2 : nh) * BK * 2);
    const int n = (227 * 1024 - 2048 - 64 - tail) / stage;
    const int cap = phit ? 8 : 4;
    return n > cap ? cap : n;
}

// On-chip state form for NH <= 128: phi in TMEM next to the accumulators and
// p in global memory (L2-resident), so that the ring gets the 128 KB a
// shared-memory phi tile would take; and two 64-wide k-tiles per ring stage.
// The MMA-issuing thread pays a fixed cost per stage (observing the full
// barrier, the commit) that a 64-wide stage of N = 128 MMAs does not hide;
// on K2000 x 4096, 2000 steps: FP16X2 114.7 -> 108.3 ms (phi in TMEM, 4
// stages of one k-tile) -> 105.8 ms (2 stages of two), FP16 78.0 -> 84.0 ->
// 69.3 ms, all bitwise identical.
constexpr bool kPhiInTmem = true;
constexpr int kKSub = 4;

constexpr int md_ksub(int nh, bool twob, int tail, bool phit, bool pair)
{
    // 4 only for pairs: their row tiles pair up, so Npad is a multiple of 256
    return kKSub >= 4 && phit && pair && md_stages(nh, twob, tail, 4, phit, pair) >= 2 ? 4
         : kKSub >= 2 && phit && md_stages(nh, twob, tail, 2, phit, pair) >= 2      ? 2
                                                                                   : 1;
}

// CTA pairs (one cta_group::2 MMA per K slice for two row tiles) wherever phi
// is in TMEM and the row tiles pair up.
constexpr bool kPairMMA = true;

inline bool use_pair(int nh, int Mt)
{
    return kPairMMA && kPhiInTmem && !kFusedHalves && onchip_ok(nh) && Mt % 2 == 0;
}

// Column halves: NH replicas (multiple of 16, <= 256); Nc = ceil(R / 2NH) with
// Mt * Nc <= SMs.  Only instantiated widths are offered.
constexpr int kNHs[] = {256, 240, 224, 192, 160, 128, 96, 64, 32, 16};

inline int pick_nh(int Mt, int R, int sms)
{
    const int nc_max = sms / Mt;
    if (nc_max < 1) return 0;
    int best = 0;
    double best_t = 1e30;
    for (int nh : kNHs) {
        const int nc = (R + 2 * nh - 1) / (2 * nh);
        if (nc > nc_max) continue;
        // time ~ columns per CTA (all CTAs run concurrently); prefer fewer padded columns
        const double t = (double)nh + 1e-3 * (double)(nc * 2 * nh - R);
        if (t < best_t) { best_t = t; best = nh; }
    }
    return best;
}

template <int NH, int KSEG, bool F16, bool PAIR>
hqa_status launch_dense_md_p(hqa_ctx* ctx, const DenseMDArgs& a, int grid, cudaStream_t st,
                             const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmS)
{
    constexpr bool ONCHIP = onchip_ok(NH) && !kFusedHalves;
    constexpr bool TWOB = kFusedHalves || KSEG == 2;   // two phi tiles per ring stage
    constexpr bool PHIT = ONCHIP && kPhiInTmem;
    constexpr int TAIL = md_tail(NH, KSEG, ONCHIP, PHIT);
    constexpr int KSUB = kFusedHalves ? 1 : md_ksub(NH, TWOB, TAIL, PHIT, PAIR);
    constexpr int STAGES = md_stages(NH, TWOB, TAIL, KSUB, PHIT, PAIR);
    static_assert(STAGES >= 2, "ring depth");
    const size_t smem = md_smem<NH, STAGES, TWOB, KSUB, PAIR, TAIL>();
    if (smem > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    if (a.KT % KSUB != 0) return HQA_ERR_INVALID_ARG;   // Npad is a multiple of 128
    if (PAIR && (grid % 2 != 0 || a.Mt % 2 != 0)) return HQA_ERR_INVALID_ARG;
    const void* fn =
        (const void*)k_dense_md<NH, STAGES, KSEG, kFusedHalves, ONCHIP, F16, KSUB, PHIT, PAIR>;
    if (hqa_smem_attr(fn, smem) != cudaSuccess) return HQA_ERR_CUDA;
    void* args[] = {const_cast<CUtensorMap*>(&tmA), const_cast<CUtensorMap*>(&tmB),
                    const_cast<CUtensorMap*>(&tmS), const_cast<DenseMDArgs*>(&a)};
    // every CTA must be co-resident: the column-group counters are waited on
    // across CTAs.  One-CTA form: a cooperative launch, issued through the
    // launch-attribute form so that a stream capture records it as a
    // cooperative kernel node.  PAIR: a cluster launch (2 CTAs per cluster)
    // after checking that all clusters fit at once; the cooperative form of a
    // cluster launch is refused under the profiler.  Every wait in the kernel
    // is bounded, so a grid that were not all resident would end in
    // HQA_DEV_TIMEOUT, not hang.
    cudaLaunchAttribute attr[1];
    if constexpr (PAIR) {
        attr[0].id = cudaLaunchAttributeClusterDimension;   // row tiles 2t, 2t+1
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
    } else {
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kMDThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (PAIR) {
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            return HQA_ERR_CUDA;
        }
        if (ncl < grid / 2) return HQA_ERR_TOO_LARGE;
    }
    cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        (void)cudaGetLastError();
        return HQA_ERR_TOO_LARGE;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return hqa_capture_note(hqa_capturing() ? HQA_ERR_UNSUPPORTED : HQA_ERR_CUDA);
    }
    return HQA_OK;
}

template <int NH, int KSEG, bool F16>
hqa_status launch_dense_md_t(hqa_ctx* ctx, const DenseMDArgs& a, int grid, cudaStream_t st,
                             const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmS)
{
    if constexpr (onchip_ok(NH) && !kFusedHalves && kPhiInTmem) {
        if (use_pair(NH, a.Mt))
            return launch_dense_md_p<NH, KSEG, F16, true>(ctx, a, grid, st, tmA, tmB, tmS);
    }
    return launch_dense_md_p<NH, KSEG, F16, false>(ctx, a, grid, st, tmA, tmB, tmS);
}

// Launches the persistent kernel for column width NH and K segments kseg.
template <bool F16>
hqa_status dense_md_dispatch(hqa_ctx* ctx, const DenseMDArgs& a, int NH, int kseg, int grid,
                             cudaStream_t st, const CUtensorMap& tmA, const CUtensorMap& tmB,
                             const CUtensorMap& tmS)
{
#define HQA_NH_CASE(V)                                                                        \
    case V:                                                                                    \
        return kseg == 3 ? launch_dense_md_t<V, 3, F16>(ctx, a, grid, st, tmA, tmB, tmS)            \
             : kseg == 2 ? launch_dense_md_t<V, 2, F16>(ctx, a, grid, st, tmA, tmB, tmS)            \
                         : launch_dense_md_t<V, 1, F16>(ctx, a, grid, st, tmA, tmB, tmS);
    switch (NH) {
        HQA_NH_CASE(256)
        HQA_NH_CASE(240)
        HQA_NH_CASE(224)
        HQA_NH_CASE(192)
        HQA_NH_CASE(160)
        HQA_NH_CASE(128)
        HQA_NH_CASE(96)
        HQA_NH_CASE(64)
        HQA_NH_CASE(32)
        HQA_NH_CASE(16)
    default: return HQA_ERR_TOO_LARGE;
    }
#undef HQA_NH_CASE
}

extern template hqa_status dense_md_dispatch<false>(hqa_ctx*, const DenseMDArgs&, int, int, int,
                                                    cudaStream_t, const CUtensorMap&,
                                                    const CUtensorMap&, const CUtensorMap&);
extern template hqa_status dense_md_dispatch<true>(hqa_ctx*, const DenseMDArgs&, int, int, int,
                                                   cudaStream_t, const CUtensorMap&,
                                                   const CUtensorMap&, const CUtensorMap&);

}  // namespace hqa_dense
