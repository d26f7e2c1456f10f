// dense_md.cu -- dense local field on the tcgen05 tensor cores.
//
// For dense couplings the field of all replicas is one GEMM per step,
//   L[i][r] = sum_j J[i][j] Phi[j][r]   (Methods, "Leapfrog algorithm"),
// with J (N x N, exactly representable in BF16, e.g. +-1) as the A operand
// and the BF16 copy of phi, replica-major ([R][K], K contiguous), as the B
// operand; both are K-major.  A CTA owns a 128-row x BN-replica output tile:
//   warp 0      TMA producer (one elected thread): 128 x 64 tile of J and
//               BN x 64 tile of Phi per stage, 128-byte swizzle, mbarrier
//               completion with transaction bytes;
//   warp 1      TMEM allocation and the MMA issuer (one elected thread):
//               4 x tcgen05.mma (M=128, N=BN, K=16) per stage into an FP32
//               accumulator in tensor memory, tcgen05.commit frees the stage;
//   warps 2..5  epilogue: tcgen05.ld 32 lanes x 16 columns, warp w reading
//               TMEM lanes 32*(w%4) .. +31 (rows), coalesced FP32 stores.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "hqa_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;                  // one 128-byte swizzle row of BF16
constexpr int kFieldBN = 128;
constexpr int kFieldStages = 4;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on any wait

__global__ void k_phi_to_bf16(const float* __restrict__ phi, int R, int N, int Rpad, int Kpad,
                              __nv_bfloat16* __restrict__ out)
{
    const size_t total = (size_t)Rpad * Kpad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / Kpad), k = (int)(idx % Kpad);
        const float v = (r < R && k < N) ? phi[(size_t)r * N + k] : 0.f;
        out[idx] = __float2bfloat16_rn(v);
    }
}

struct FieldArgs {
    float* L;            // [R][N]
    const float* phi;    // [R][N], for the 2 h |phi| term
    const float* h;      // [N] or null
    uint32_t* status;
    int N, R, KT;        // KT = Kpad / BK
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(192, 1)
k_dense_field(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmB,
              const FieldArgs a)
{
    constexpr uint32_t A_BYTES = BM * BK * 2;
    constexpr uint32_t B_BYTES = BN * BK * 2;
    constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand region
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar = base + STAGES * STAGE_BYTES;   // full[S], empty[S], accf
    const uint32_t full0 = bar, empty0 = bar + 8 * STAGES, accf = bar + 16 * STAGES;
    const uint32_t tmem_slot = accf + 8;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(full0 + 8 * s, 1);
            tc::mbar_init(empty0 + 8 * s, 1);
        }
        tc::mbar_init(accf, 1);
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmJ);
        tc::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(tmem_slot));
    volatile int* abort = &s_abort;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer ----
        for (int kt = 0; kt < a.KT; ++kt) {
            const int s = kt % STAGES;
            if (kt >= STAGES && !tc::mbar_wait(empty0 + 8 * s, ((kt / STAGES) - 1) & 1, abort, kWaitNs))
                break;
            const uint32_t sa = base + s * STAGE_BYTES;
            tc::mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
            tc::tma_load_2d(sa, &tmJ, kt * BK, m0, full0 + 8 * s);
            tc::tma_load_2d(sa + A_BYTES, &tmB, kt * BK, n0, full0 + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        constexpr uint32_t idesc = tc::idesc_bf16(BM, BN);
        for (int kt = 0; kt < a.KT; ++kt) {
            const int s = kt % STAGES;
            if (!tc::mbar_wait(full0 + 8 * s, (kt / STAGES) & 1, abort, kWaitNs)) break;
            tc::tc_fence_after();
            const uint32_t sa = base + s * STAGE_BYTES;
            const uint64_t ad = tc::sdesc_k128(sa), bd = tc::sdesc_k128(sa + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)  // 16 BF16 = 32 bytes per MMA along K
                tc::mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kt | kk) != 0);
            tc::mma_commit(empty0 + 8 * s);
        }
        tc::mma_commit(accf);
    } else if (warp >= 2) {
        // ---- epilogue: TMEM -> registers -> global ----
        const int quarter = warp & 3;
        // warp-uniform outcome: tcgen05.ld is a whole-warp instruction
        const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(accf, 0, abort, kWaitNs));
        tc::tc_fence_after();
        if (ok) {
            const int row = m0 + 32 * quarter + lane;
            const float hr = (a.h && row < a.N) ? 2.f * a.h[row] : 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0, v);
                tc::tmem_wait_ld();
                if (row < a.N) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const int r = n0 + c0 + c;
                        if (r < a.R) {
                            float L = __uint_as_float(v[c]);
                            if (hr != 0.f) L += hr * fabsf(a.phi[(size_t)r * a.N + row]);
                            a.L[(size_t)r * a.N + row] = L;
                        }
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (*abort && threadIdx.x == 0) atomicOr(a.status, HQA_DEV_TIMEOUT);
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D BF16 tensor [rows][cols] (cols contiguous, cols * 2 bytes a multiple of
// 16), box {64 cols, box_rows}, 128-byte swizzle.
bool make_tmap_bf16(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows)
{
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, int STAGES>
size_t field_smem()
{
    return 1024 + (size_t)STAGES * (BM * BK * 2 + BN * BK * 2) + 16 * STAGES + 64;
}

}  // namespace

// Builds the BF16 tensor-core operands of J (zero padded to [Mpad][Mpad]) and
// their tensor maps: J rounded to BF16 (exact for +-1 couplings) and, when
// rounding is not exact (real-valued J), the split operand [J_hi | J_lo | J_hi]
// with J_lo = BF16(J - J_hi), which with Phi split the same way gives
// J_hi Phi_hi + J_lo Phi_hi + J_hi Phi_lo: J and Phi to ~16 significant bits.
hqa_status hqa_dense_setup(hqa_ctx* ctx, const float* J)
{
    const int N = ctx->N;
    const int Mpad = (N + BM - 1) / BM * BM;
    std::vector<__nv_bfloat16> jb((size_t)Mpad * Mpad, __float2bfloat16_rn(0.f));
    std::vector<__nv_bfloat16> jl((size_t)Mpad * Mpad, __float2bfloat16_rn(0.f));
    bool exact = true;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            const float v = (i == j) ? 0.f : J[(size_t)i * N + j];
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            const float r = v - __bfloat162float(b);
            exact = exact && r == 0.f;
            jb[(size_t)i * Mpad + j] = b;
            jl[(size_t)i * Mpad + j] = __float2bfloat16_rn(r);
        }
    if (!get_encode()) return HQA_OK;
    void* d = nullptr;
    HQA_CUDA_TRY(cudaMalloc(&d, jb.size() * sizeof(__nv_bfloat16)));
    ctx->d_Jbf = d;
    HQA_CUDA_TRY(cudaMemcpy(d, jb.data(), jb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
    ctx->Mpad = Mpad;
    if (!make_tmap_bf16(&ctx->tmJ, d, Mpad, Mpad, BM)) return HQA_ERR_CUDA;
    if (!exact) {
        std::vector<__nv_bfloat16> jc((size_t)Mpad * 3 * Mpad);
        for (size_t i = 0; i < (size_t)Mpad; ++i)
            for (size_t j = 0; j < (size_t)Mpad; ++j) {
                const __nv_bfloat16 hi = jb[i * Mpad + j], lo = jl[i * Mpad + j];
                jc[i * 3 * Mpad + j] = hi;
                jc[i * 3 * Mpad + Mpad + j] = lo;
                jc[i * 3 * Mpad + 2 * Mpad + j] = hi;
            }
        void* dc = nullptr;
        HQA_CUDA_TRY(cudaMalloc(&dc, jc.size() * sizeof(__nv_bfloat16)));
        ctx->d_Jcat = dc;
        HQA_CUDA_TRY(cudaMemcpy(dc, jc.data(), jc.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
        if (!make_tmap_bf16(&ctx->tmJ3, dc, Mpad, (uint64_t)3 * Mpad, BM)) return HQA_ERR_CUDA;
    }
    ctx->dense_exact = exact;
    ctx->dense_tc = true;
    return HQA_OK;
}

hqa_status hqa_dense_field(hqa_ctx* ctx, int32_t R, const float* phi, float* L, cudaStream_t st)
{
    if (!ctx->dense_tc) return HQA_ERR_UNSUPPORTED;
    const int Kpad = ctx->Mpad;
    const int Rpad = (R + kFieldBN - 1) / kFieldBN * kFieldBN;
    const size_t bytes = (size_t)Rpad * Kpad * sizeof(__nv_bfloat16);
    hqa_status s = hqa_reserve(ctx, &ctx->d_ws, &ctx->ws_cap, bytes);
    if (s != HQA_OK) return s;
    __nv_bfloat16* phib = static_cast<__nv_bfloat16*>(ctx->d_ws);
    k_phi_to_bf16<<<std::min<size_t>(4096, (bytes / 2 + 255) / 256), 256, 0, st>>>(phi, R, ctx->N, Rpad,
                                                                                   Kpad, phib);
    CUtensorMap tmB;
    if (!make_tmap_bf16(&tmB, phib, Rpad, Kpad, kFieldBN)) return HQA_ERR_CUDA;
    FieldArgs a{};
    a.L = L;
    a.phi = phi;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.status = ctx->d_status;
    a.N = ctx->N;
    a.R = R;
    a.KT = Kpad / BK;
    const size_t smem = field_smem<kFieldBN, kFieldStages>();
    cudaError_t e = hqa_smem_attr((const void*)k_dense_field<kFieldBN, kFieldStages>, smem);
    if (e != cudaSuccess) return HQA_ERR_CUDA;
    const dim3 grid(ctx->Mpad / BM, Rpad / kFieldBN);
    k_dense_field<kFieldBN, kFieldStages><<<grid, 192, smem, st>>>(ctx->tmJ, tmB, a);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
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
//   epilogue  8 warps read L from TMEM and do the kick and drift of Methods'
//             leapfrog on the FP32 state in global memory ([R][Npad], one
//             owner per element), write the BF16 Phi^(m+1) into the other
//             buffer and the window sum, release accumulator h and arrive on
//             the counter.
// While the epilogue drains half h, the MMA of the other half runs.
// ===========================================================================
namespace {

constexpr int kEpiWarps = 8;
constexpr int kMDThreads = 64 + 32 * kEpiWarps;

struct DenseMDArgs {
    float* phi;              // [Rpad][Npad] FP32 master
    float* p;                // [Rpad][Npad]
    float* w;                // [Rpad][Npad] window sums
    __nv_bfloat16* phib;     // [2][Rpad][Npad] operand buffers
    const StepCoef* sched;
    const float* h;          // [N] or null
    unsigned int* gbar;      // [2 Nc] arrival counters
    uint32_t* status;
    int64_t S;
    int W, N, Npad, Rpad, R, KT, Mt, M;
    int rep0;                // global index of this launch's first replica (random draws)
    // armed check of the bounded-wait path (hqa_arm_wait_check): before step
    // wait_step every producer waits for *wait_flag != 0, at most wait_ns
    const unsigned int* wait_flag;
    int64_t wait_step;
    uint64_t wait_ns;
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int NH, int STAGES, int KSEG, bool FUSED, bool ONCHIP>
__global__ void __launch_bounds__(kMDThreads, 1)
k_dense_md(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmB,
           const DenseMDArgs a)
{
    constexpr uint32_t A_BYTES = BM * BK * 2;
    constexpr uint32_t B_BYTES = NH * BK * 2;
    // fused: one J tile per stage feeds the MMAs of both column halves
    constexpr uint32_t STAGE_BYTES = A_BYTES + (FUSED ? 2u : 1u) * B_BYTES;
    constexpr int NPASS = FUSED ? 1 : 2;   // MMA passes (and counters) per step
    // on-chip state: p in TMEM columns [2 NH, 4 NH), phi in shared memory
    constexpr uint32_t TMEM_COLS = ONCHIP ? 512u
                                 : 2 * NH <= 64 ? 64 : 2 * NH <= 128 ? 128 : 2 * NH <= 256 ? 256 : 512;
    static_assert(NH % 16 == 0 && NH <= 256, "UMMA N");
    static_assert(!ONCHIP || (NH <= 128 && !FUSED), "on-chip state: 4 NH TMEM columns");
    static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t bar = base + STAGES * STAGE_BYTES;
    const uint32_t full0 = bar, empty0 = bar + 8 * STAGES;
    const uint32_t accf0 = bar + 16 * STAGES, acce0 = accf0 + 16;
    const uint32_t tmem_slot = acce0 + 16;
    const uint32_t phis = bar + 1024;   // ONCHIP: phi tile [2 NH columns][128 rows] FP32
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x % a.Mt, nc = blockIdx.x / a.Mt;
    const int m0 = mt * BM, n0 = nc * 2 * NH;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(full0 + 8 * s, 1);
            tc::mbar_init(empty0 + 8 * s, 1);
        }
        for (int hh = 0; hh < 2; ++hh) {
            tc::mbar_init(accf0 + 8 * hh, 1);
            tc::mbar_init(acce0 + 8 * hh, kEpiWarps);
        }
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmJ);
        tc::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
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
                    const int brow = (int)(m & 1) * a.Rpad + n0 + hh * NH;
                    // split operands: K runs over [hi | lo] with J reused (KSEG 2), or
                    // over [hi | hi | lo] against [J_hi | J_lo | J_hi] (KSEG 3)
                    const int KTT = KSEG * a.KT;
                    for (int kt = 0; kt < KTT; ++kt, ++it) {
                        const int s = it % STAGES;
                        if (it >= STAGES &&
                            !tc::mbar_wait(empty0 + 8 * s, ((it / STAGES) - 1) & 1, abort, kWaitNs))
                            break;
                        const uint32_t sa = base + s * STAGE_BYTES;
                        tc::mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
                        tc::tma_load_2d(sa, &tmJ, (KSEG == 2 ? kt % a.KT : kt) * BK, m0, full0 + 8 * s);
                        tc::tma_load_2d(sa + A_BYTES, &tmB, kt * BK, brow, full0 + 8 * s);
                        if constexpr (FUSED)
                            tc::tma_load_2d(sa + A_BYTES + B_BYTES, &tmB, kt * BK, brow + NH,
                                            full0 + 8 * s);
                    }
                }
            }
            // drain: every issued stage must land before the CTA can exit
            if (*abort)
                for (uint32_t k = (it > STAGES ? it - STAGES : 0); k < it; ++k)
                    tc::mbar_wait(full0 + 8 * (k % STAGES), (k / STAGES) & 1, abort, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            constexpr uint32_t idesc = tc::idesc_bf16(BM, NH);
            uint32_t it = 0;
            for (int64_t m = 0; m < a.S && !*abort; ++m) {
                for (int hh = 0; hh < NPASS && !*abort; ++hh) {
                    if (m > 0 && !tc::mbar_wait(acce0 + 8 * hh, (uint32_t)((m - 1) & 1), abort, kWaitNs))
                        break;
                    tc::tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(hh * NH);
                    const int KTT = KSEG * a.KT;
                    for (int kt = 0; kt < KTT; ++kt, ++it) {
                        const int s = it % STAGES;
                        if (!tc::mbar_wait(full0 + 8 * s, (it / STAGES) & 1, abort, kWaitNs)) break;
                        tc::tc_fence_after();
                        const uint32_t sa = base + s * STAGE_BYTES;
                        const uint64_t ad = tc::sdesc_k128(sa), bd = tc::sdesc_k128(sa + A_BYTES);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, (kt | kk) != 0);
                        if constexpr (FUSED) {
                            const uint64_t bd1 = tc::sdesc_k128(sa + A_BYTES + B_BYTES);
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk)
                                tc::mma_bf16(d + (uint32_t)NH, ad + 2 * kk, bd1 + 2 * kk, idesc,
                                             (kt | kk) != 0);
                        }
                        tc::mma_commit(empty0 + 8 * s);
                    }
                    tc::mma_commit(accf0 + 8 * hh);
                }
            }
        }
    } else {
        // ---- epilogue warps: kick, drift, BF16 shadow, window ----
        const int ew = warp - 2;              // 0..7
        const int quarter = warp & 3;         // TMEM lanes 32*quarter .. +31
        const int csel = ew >> 2;             // chunk parity handled by this warp
        const int row = m0 + 32 * quarter + lane;
        const bool row_ok = row < a.N;
        const float hr = (a.h && row_ok) ? 2.f * a.h[row] : 0.f;
        const int mhalf = (a.M - 2) / 2;
        const int64_t win0 = a.S - (int64_t)a.W;
        const uint32_t tl = (uint32_t)(32 * quarter) << 16;   // this warp's TMEM lanes
        const uint32_t rloc = (uint32_t)(32 * quarter + lane);  // row within the tile
        if constexpr (ONCHIP) {
            // the tile's state moves on chip for the whole trajectory
            for (int hh = 0; hh < 2; ++hh)
                for (int c = csel; c < NH / 16; c += 2) {
                    const int col = hh * NH + c * 16;
                    uint32_t pv[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const size_t o = (size_t)(n0 + col + j) * a.Npad + row;
                        asm volatile("st.shared.f32 [%0], %1;" ::"r"(phis + (uint32_t)(col + j) * 512u + rloc * 4u),
                                     "f"(a.phi[o]));
                        pv[j] = __float_as_uint(a.p[o]);
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
            __nv_bfloat16* nb = a.phib + (size_t)((m + 1) & 1) * a.Rpad * Kb;
            bool ok = true;
            for (int hh = 0; hh < 2 && !stop; ++hh) {
                // the state of this warp's first chunk does not depend on the MMA:
                // its loads are in flight while the accumulator is computed
                float ph[16], pp[16];
                if (!ONCHIP && row_ok && csel < NH / 16) {
                    const int rb0 = n0 + hh * NH + csel * 16;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const size_t o = (size_t)(rb0 + j) * a.Npad + row;
                        ph[j] = a.phi[o];
                        pp[j] = a.p[o];
                    }
                }
                const int pass = FUSED ? 0 : hh;
                if (!FUSED || hh == 0) {
                    ok = __all_sync(0xffffffffu,
                                    tc::mbar_wait(accf0 + 8 * pass, (uint32_t)(m & 1), abort, kWaitNs));
                    tc::tc_fence_after();
                }
                if (ok && ONCHIP) {
#pragma unroll 1
                    for (int c = csel; c < NH / 16; c += 2) {
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
                                const float L = __uint_as_float(v[j]) + hr * fabsf(phl[j]);
                                const float phi2 = phl[j] * phl[j];
                                float pw = phl[j];
                                for (int q = 0; q < mhalf; ++q) pw *= phi2;
                                const float pn = __uint_as_float(pv[j]) - fmaf(cf.x, pw, cf.y * L);
                                const float fn = fmaf(cf.z, pn, phl[j]);
                                pv[j] = __float_as_uint(pn);
                                asm volatile("st.shared.f32 [%0], %1;"
                                             ::"r"(phis + (uint32_t)(col + j) * 512u + rloc * 4u), "f"(fn));
                                const size_t ob = (size_t)(n0 + col + j) * Kb + row;
                                const __nv_bfloat16 hi = __float2bfloat16_rn(fn);
                                nb[ob] = hi;
                                if (KSEG == 2) nb[ob + a.Npad] = __float2bfloat16_rn(fn - __bfloat162float(hi));
                                if (KSEG == 3) {
                                    nb[ob + a.Npad] = hi;
                                    nb[ob + 2 * a.Npad] = __float2bfloat16_rn(fn - __bfloat162float(hi));
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
                    for (int c = csel; c < NH / 16; c += 2) {
                        uint32_t v[16];
                        tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(hh * NH + c * 16), v);
                        // the next chunk's state loads overlap this chunk's update
                        float nph[16], npp[16];
                        const bool more = row_ok && c + 2 < NH / 16;
                        if (more) {
                            const int rb1 = n0 + hh * NH + (c + 2) * 16;
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
                                const float L = __uint_as_float(v[j]) + hr * fabsf(ph[j]);
                                const float phi2 = ph[j] * ph[j];
                                float pw = ph[j];
                                for (int q = 0; q < mhalf; ++q) pw *= phi2;
                                const float pn = pp[j] - fmaf(cf.x, pw, cf.y * L);
                                const float fn = fmaf(cf.z, pn, ph[j]);
                                a.p[o] = pn;
                                a.phi[o] = fn;
                                const size_t ob = (size_t)(rbase + j) * Kb + row;
                                const __nv_bfloat16 hi = __float2bfloat16_rn(fn);
                                nb[ob] = hi;
                                if (KSEG == 2) nb[ob + a.Npad] = __float2bfloat16_rn(fn - __bfloat162float(hi));
                                if (KSEG == 3) {
                                    nb[ob + a.Npad] = hi;
                                    nb[ob + 2 * a.Npad] = __float2bfloat16_rn(fn - __bfloat162float(hi));
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
                for (int c = csel; c < NH / 16; c += 2) {
                    const int col = hh * NH + c * 16;
                    uint32_t pv[16];
                    tc::tmem_ld16(tmem + tl + (uint32_t)(2 * NH + col), pv);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const size_t o = (size_t)(n0 + col + j) * a.Npad + row;
                        float f;
                        asm volatile("ld.shared.f32 %0, [%1];"
                                     : "=f"(f) : "r"(phis + (uint32_t)(col + j) * 512u + rloc * 4u));
                        a.phi[o] = f;
                        a.p[o] = __uint_as_float(pv[j]);
                    }
                }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (*abort && threadIdx.x == 0) atomicOr(a.status, HQA_DEV_TIMEOUT);
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// State set-up: phi(0), p(0) (SplitMix64 or caller-given), window 0, BF16
// operand buffer 0; padding rows/replicas zero in every array.
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
        const __nv_bfloat16 hi = __float2bfloat16_rn(phi);
        a.phib[ob] = hi;
        a.phib[buf + ob] = __float2bfloat16_rn(0.f);
        if (kseg == 2) {
            a.phib[ob + a.Npad] = __float2bfloat16_rn(phi - __bfloat162float(hi));
            a.phib[buf + ob + a.Npad] = __float2bfloat16_rn(0.f);
        }
        if (kseg == 3) {
            a.phib[ob + a.Npad] = hi;
            a.phib[ob + 2 * a.Npad] = __float2bfloat16_rn(phi - __bfloat162float(hi));
            a.phib[buf + ob + a.Npad] = __float2bfloat16_rn(0.f);
            a.phib[buf + ob + 2 * a.Npad] = __float2bfloat16_rn(0.f);
        }
    }
}

__global__ void k_dense_out(DenseMDArgs a, float inv_w, float* phi_out, float* p_out,
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

template <int NH, int STAGES, bool FUSED, bool ONCHIP>
size_t md_smem()
{
    // alignment slack, ring, barrier block (1 KB), on-chip phi tile
    return 1024 + (size_t)STAGES * (BM * BK * 2 + (FUSED ? 2 : 1) * NH * BK * 2) + 1024 +
           (ONCHIP ? (size_t)2 * NH * BM * 4 : 0);
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
// the alignment slack, the barrier block and the on-chip phi tile, at most 4
// (6 stages measured no faster on K2000 x 2048 replicas).
constexpr int md_stages(int nh, bool fused, bool onchip)
{
    const int stage = BM * BK * 2 + (fused ? 2 : 1) * nh * BK * 2;
    const int n = (227 * 1024 - 2048 - 64 - (onchip ? 2 * nh * BM * 4 : 0)) / stage;
    return n > 4 ? 4 : n;
}

// Column halves: NH replicas (multiple of 16, <= 256); Nc = ceil(R / 2NH) with
// Mt * Nc <= SMs.  Only instantiated widths are offered.
constexpr int kNHs[] = {256, 240, 224, 192, 160, 128, 96, 64, 32, 16};

int pick_nh(int Mt, int R, int sms)
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

}  // namespace

template <int NH, int KSEG>
static hqa_status launch_dense_md_t(hqa_ctx* ctx, const DenseMDArgs& a, int grid, cudaStream_t st,
                                    const CUtensorMap& tmA, const CUtensorMap& tmB)
{
    constexpr bool ONCHIP = onchip_ok(NH) && !kFusedHalves;
    constexpr int STAGES = md_stages(NH, kFusedHalves, ONCHIP);
    static_assert(STAGES >= 2, "ring depth");
    const size_t smem = md_smem<NH, STAGES, kFusedHalves, ONCHIP>();
    if (smem > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    // a cooperative launch is not captured into graphs here
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    const void* fn = (const void*)k_dense_md<NH, STAGES, KSEG, kFusedHalves, ONCHIP>;
    if (hqa_smem_attr(fn, smem) != cudaSuccess) return HQA_ERR_CUDA;
    void* args[] = {const_cast<CUtensorMap*>(&tmA), const_cast<CUtensorMap*>(&tmB),
                    const_cast<DenseMDArgs*>(&a)};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kMDThreads), args, smem, st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        (void)cudaGetLastError();
        return HQA_ERR_TOO_LARGE;
    }
    return e == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

bool hqa_dense_md_possible(const hqa_ctx* ctx, int32_t R)
{
    if (!ctx->dense_tc || R < 1) return false;
    return pick_nh(ctx->Mpad / BM, 1, ctx->sm_count) > 0;   // larger R runs in chunks
}

namespace {

// K segments of the tensor-core product: 1 (BF16 operand), 2 (split Phi
// against an exact J, J reused), 3 (split Phi against a split real-valued J).
int kseg_of(const hqa_ctx* ctx, bool split) { return split ? (ctx->dense_exact ? 2 : 3) : 1; }

// Bytes one step touches for R replicas: FP32 phi and p, the two BF16 operand
// buffers (kseg segments each) and the coupling operand.
size_t dense_step_bytes(const hqa_ctx* ctx, int32_t R, int kseg)
{
    int NH = 0, grid = 0;
    if (!hqa_dense_md_geometry(ctx, R, &NH, &grid)) return SIZE_MAX;
    const size_t Rpad = (size_t)(grid / (ctx->Mpad / BM)) * 2 * NH;
    const size_t n = Rpad * (size_t)ctx->Mpad;
    const size_t J = (size_t)ctx->Mpad * ctx->Mpad * 2 * (kseg == 3 ? 3 : 1);
    return n * (8 + 4 * (size_t)kseg) + J;
}

// Replica chunks run one after another, each a full trajectory.  A CTA's step
// costs its MMA columns (NH per half, doubled for the split operand) plus a
// fixed part worth ~150 columns (streaming its 128-row coupling tile through
// shared memory, the column-group barrier, pipeline fill), measured on K2000;
// a chunk whose step touches more than ~70% of L2 streams its state from HBM
// every step, which about doubles the step.  C minimises the sum over chunks.
int dense_chunks(const hqa_ctx* ctx, int32_t R, bool split)
{
    const int kseg = kseg_of(ctx, split);
    const double budget = 0.7 * (double)(ctx->l2_bytes ? ctx->l2_bytes : (size_t)96 << 20);
    int best = 1;
    double best_t = 1e300;
    for (int C = 1; C <= 16 && C <= R; ++C) {
        const int Rc = (R + C - 1) / C;
        int NH = 0, grid = 0;
        if (!hqa_dense_md_geometry(ctx, Rc, &NH, &grid)) continue;
        const double spill = (double)dense_step_bytes(ctx, Rc, kseg) > budget ? 2.0 : 1.0;
        const double t = (double)C * ((double)kseg * NH + 150.0) * spill;
        if (t < best_t - 1e-9) {
            best_t = t;
            best = C;
        }
    }
    return best;
}

}  // namespace

int hqa_dense_md_geometry(const hqa_ctx* ctx, int32_t R, int* nh, int* grid)
{
    const int Mt = ctx->Mpad / BM;
    const int h = pick_nh(Mt, R, ctx->sm_count);
    if (h == 0) return 0;
    const int nc = (R + 2 * h - 1) / (2 * h);
    *nh = h;
    *grid = Mt * nc;
    return 1;
}

static hqa_status dense_md_chunk(hqa_ctx* ctx, const StepCoef* d_sched, int64_t S, int32_t W,
                                 int32_t R, int32_t rep0, uint64_t seed, int init,
                                 const float* phi0, const float* p0, int M, float* phi_out,
                                 float* p_out, float* phibar_out, bool split, cudaStream_t st)
{
    int NH = 0, grid = 0;
    if (!hqa_dense_md_geometry(ctx, R, &NH, &grid)) return HQA_ERR_TOO_LARGE;
    const int Mt = ctx->Mpad / BM;
    const int Nc = grid / Mt;
    const int Rpad = Nc * 2 * NH;
    const int Npad = ctx->Mpad;
    const size_t n = (size_t)Rpad * Npad;
    const int kseg = kseg_of(ctx, split);
    const size_t nb = (size_t)kseg * n;   // operand elements per buffer
    // state: phi, p, w (FP32), two BF16 operand buffers, 2 Nc counters
    const size_t off_p = n * 4, off_w = 2 * n * 4, off_b = 3 * n * 4, off_g = off_b + 2 * nb * 2;
    const size_t need = off_g + (size_t)2 * Nc * sizeof(unsigned int);
    hqa_status s = hqa_reserve(ctx, &ctx->d_state, &ctx->state_cap, need);
    if (s != HQA_OK) return s;
    char* b = static_cast<char*>(ctx->d_state);
    DenseMDArgs a{};
    a.phi = reinterpret_cast<float*>(b);
    a.p = reinterpret_cast<float*>(b + off_p);
    a.w = reinterpret_cast<float*>(b + off_w);
    a.phib = reinterpret_cast<__nv_bfloat16*>(b + off_b);
    a.gbar = reinterpret_cast<unsigned int*>(b + off_g);
    a.sched = d_sched;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.status = ctx->d_status;
    a.S = S;
    a.W = W;
    a.N = ctx->N;
    a.Npad = Npad;
    a.Rpad = Rpad;
    a.R = R;
    a.KT = Npad / BK;
    a.Mt = Mt;
    a.M = M;
    a.rep0 = rep0;
    if (ctx->wait_flag) {   // one-shot: the first chunk of the next launch
        a.wait_flag = static_cast<const unsigned int*>(ctx->wait_flag);
        a.wait_step = ctx->wait_step;
        a.wait_ns = ctx->wait_ns;
        ctx->wait_flag = nullptr;
    }
    CUtensorMap tmB;
    if (!make_tmap_bf16(&tmB, a.phib, (uint64_t)2 * Rpad, (uint64_t)kseg * Npad, NH))
        return HQA_ERR_CUDA;
    const CUtensorMap& tmA = kseg == 3 ? ctx->tmJ3 : ctx->tmJ;
    k_dense_init<<<std::min<size_t>(8192, (n + 255) / 256), 256, 0, st>>>(a, seed, init, phi0, p0,
                                                                         kseg);
    if (cudaMemsetAsync(a.gbar, 0, (size_t)2 * Nc * sizeof(unsigned int), st) != cudaSuccess)
        return HQA_ERR_CUDA;
#define HQA_NH_CASE(V)                                                                        \
    case V:                                                                                    \
        s = kseg == 3 ? launch_dense_md_t<V, 3>(ctx, a, grid, st, tmA, tmB)                    \
          : kseg == 2 ? launch_dense_md_t<V, 2>(ctx, a, grid, st, tmA, tmB)                    \
                      : launch_dense_md_t<V, 1>(ctx, a, grid, st, tmA, tmB);                   \
        break;
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
    if (s != HQA_OK) return s;
    const int64_t nwin = S < W ? S : W;
    k_dense_out<<<std::min<size_t>(8192, ((size_t)R * ctx->N + 255) / 256), 256, 0, st>>>(
        a, 1.0f / (float)nwin, phi_out, p_out, phibar_out);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

int hqa_dense_md_chunks(const hqa_ctx* ctx, int32_t R, bool split)
{
    return dense_chunks(ctx, R, split);
}

hqa_status hqa_dense_launch_md(hqa_ctx* ctx, const StepCoef* d_sched, int64_t S, int32_t W,
                               int32_t R, uint64_t seed, int init, const float* phi0,
                               const float* p0, int M, float* phi_out, float* p_out,
                               float* phibar_out, bool split, cudaStream_t st)
{
    const int C = dense_chunks(ctx, R, split);
    const int Rc = (R + C - 1) / C;
    const size_t N = (size_t)ctx->N;
    for (int r0 = 0; r0 < R; r0 += Rc) {
        const int Rk = std::min(Rc, R - r0);
        const size_t o = (size_t)r0 * N;
        hqa_status s = dense_md_chunk(ctx, d_sched, S, W, Rk, r0, seed, init,
                                      phi0 ? phi0 + o : nullptr, p0 ? p0 + o : nullptr, M,
                                      phi_out ? phi_out + o : nullptr, p_out ? p_out + o : nullptr,
                                      phibar_out ? phibar_out + o : nullptr, split, st);
        if (s != HQA_OK) return s;
    }
    return HQA_OK;
}

extern "C" hqa_status hqa_arm_wait_check(hqa_ctx* ctx, const uint32_t* flag, int64_t step,
                                         int64_t limit_ns)
{
    if (!ctx || !flag || step < 0 || limit_ns < 1 || limit_ns > 10000000000ll ||
        ((uintptr_t)flag % 4))
        return HQA_ERR_INVALID_ARG;
    if (!ctx->dense_tc) return HQA_ERR_UNSUPPORTED;
    ctx->wait_flag = flag;
    ctx->wait_step = step;
    ctx->wait_ns = (uint64_t)limit_ns;
    return HQA_OK;
}
