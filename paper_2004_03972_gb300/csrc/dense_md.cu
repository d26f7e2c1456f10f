// dense_md.cu -- dense local field and MD on the tcgen05 tensor cores: the
// coupling operands, the one-shot field kernel and the host side of the
// persistent MD kernel (dense_md_kernel.cuh), instantiated here for a BF16
// operand and in dense_md_f16.cu for an FP16 one.
//
// For dense couplings the field of all replicas is one GEMM per step,
//   L[i][r] = sum_j J[i][j] Phi[j][r]   (Methods, "Leapfrog algorithm"),
// with J (N x N) as the A operand and the 16-bit copy of phi, replica-major
// ([R][K], K contiguous), as the B operand; both are K-major.  In the one-shot
// field kernel a CTA owns a 128-row x BN-replica output tile:
//   warp 0      TMA producer (one elected thread): 128 x 64 tile of J and
//               BN x 64 tile of Phi per stage, 128-byte swizzle, mbarrier
//               completion with transaction bytes;
//   warp 1      TMEM allocation and the MMA issuer (one elected thread):
//               4 x tcgen05.mma (M=128, N=BN, K=16) per stage into an FP32
//               accumulator in tensor memory, tcgen05.commit frees the stage;
//   warps 2..5  epilogue: tcgen05.ld 32 lanes x 16 columns, warp w reading
//               TMEM lanes 32*(w%4) .. +31 (rows), coalesced FP32 stores.
// Operand formats: BF16 (J and phi rounded to BF16, 8 significant bits), FP16
// (11 bits; phi scaled by 2^6 and J by 2^10 before rounding, the accumulator
// scaled back by 2^-16), and their splits x = hi + lo (BF16X2, FP16X2) run as
// extra K segments of the same product.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "dense_md_kernel.cuh"

using hqa_dense::BK;
using hqa_dense::BM;
using hqa_dense::DenseMDArgs;
using hqa_dense::kWaitNs;

namespace {

constexpr int kFieldBN = 128;
constexpr int kFieldStages = 4;

template <bool F16>
__global__ void k_phi_to_16(const float* __restrict__ phi, int R, int N, int Rpad, int Kpad,
                            float oscale, uint16_t* __restrict__ out)
{
    const size_t total = (size_t)Rpad * Kpad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / Kpad), k = (int)(idx % Kpad);
        const float v = (r < R && k < N) ? phi[(size_t)r * N + k] : 0.f;
        out[idx] = hqa_dense::cvt16<F16>(v * oscale);
    }
}

struct FieldArgs {
    float* L;            // [R][N]
    const float* phi;    // [R][N], for the 2 h |phi| term
    const float* h;      // [N] or null
    uint32_t* status;
    float lscale;        // L = accumulator * lscale
    int N, R, KT;        // KT = Kpad / BK
};

template <int BN, int STAGES, bool F16>
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
        constexpr uint32_t idesc = F16 ? tc::idesc_f16(BM, BN) : tc::idesc_bf16(BM, BN);
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
                            float L = __uint_as_float(v[c]) * a.lscale;
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

// 2-D 16-bit tensor [rows][cols] (BF16, or FP16 when f16; cols contiguous,
// cols * 2 bytes a multiple of 16), box {64 cols, box_rows}, 128-byte swizzle.
// A [rows][cols] 16-bit array; box_cols x box_rows boxes, 128-byte swizzle
// (MMA operand tiles) or none (row-major staging tiles).
bool make_tmap16_box(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols,
                     uint32_t box_cols, uint32_t box_rows, bool swizzle, bool f16)
{
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_tmap16(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows,
                 bool f16)
{
    return make_tmap16_box(m, ptr, rows, cols, BK, box_rows, true, f16);
}

template <int BN, int STAGES>
size_t field_smem()
{
    return 1024 + (size_t)STAGES * (BM * BK * 2 + BN * BK * 2) + 16 * STAGES + 64;
}

// Uploads a [rows][cols] 16-bit operand and encodes its tensor map.
hqa_status upload16(const std::vector<uint16_t>& host, uint64_t rows, uint64_t cols, bool f16,
                    void** dptr, CUtensorMap* map)
{
    void* d = nullptr;
    HQA_CUDA_TRY(cudaMalloc(&d, host.size() * sizeof(uint16_t)));
    *dptr = d;
    HQA_CUDA_TRY(cudaMemcpy(d, host.data(), host.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    return make_tmap16(map, d, rows, cols, BM, f16) ? HQA_OK : HQA_ERR_CUDA;
}

// [J_hi | J_lo | J_hi] rows of the split product J_hi Phi_hi + J_lo Phi_hi + J_hi Phi_lo.
std::vector<uint16_t> concat3(const std::vector<uint16_t>& hi, const std::vector<uint16_t>& lo,
                              size_t Mpad)
{
    std::vector<uint16_t> jc(Mpad * 3 * Mpad);
    for (size_t i = 0; i < Mpad; ++i)
        for (size_t j = 0; j < Mpad; ++j) {
            jc[i * 3 * Mpad + j] = hi[i * Mpad + j];
            jc[i * 3 * Mpad + Mpad + j] = lo[i * Mpad + j];
            jc[i * 3 * Mpad + 2 * Mpad + j] = hi[i * Mpad + j];
        }
    return jc;
}

uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
float bf16_val(uint16_t u) { return __bfloat162float(__ushort_as_bfloat16(u)); }
uint16_t f16_bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
float f16_val(uint16_t u) { return __half2float(__ushort_as_half(u)); }

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
    std::vector<uint16_t> jb((size_t)Mpad * Mpad, 0), jl((size_t)Mpad * Mpad, 0);
    bool exact = true;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            const float v = (i == j) ? 0.f : J[(size_t)i * N + j];
            const uint16_t b = bf16_bits(v);
            const float r = v - bf16_val(b);
            exact = exact && r == 0.f;
            jb[(size_t)i * Mpad + j] = b;
            jl[(size_t)i * Mpad + j] = bf16_bits(r);
        }
    if (!get_encode()) return HQA_OK;
    ctx->Mpad = Mpad;
    hqa_status s = upload16(jb, Mpad, Mpad, false, &ctx->d_Jbf, &ctx->tmJ);
    if (s != HQA_OK) return s;
    if (!exact) {
        s = upload16(concat3(jb, jl, Mpad), Mpad, (uint64_t)3 * Mpad, false, &ctx->d_Jcat, &ctx->tmJ3);
        if (s != HQA_OK) return s;
    }
    ctx->dense_exact = exact;
    ctx->dense_tc = true;
    return HQA_OK;
}

// FP16 operands, built on first use from the context's host copy of J: J
// scaled by 2^10 and rounded to FP16 (exact for +-1 couplings) and, when that
// rounding is not exact, the split [J_hi | J_lo | J_hi] (about 22 significant
// bits of J).
static hqa_status dense_setup_f16(hqa_ctx* ctx)
{
    if (ctx->dense_f16) return HQA_OK;
    if (!ctx->dense_tc) return HQA_ERR_UNSUPPORTED;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    const int N = ctx->N;
    const size_t Mpad = (size_t)ctx->Mpad;
    std::vector<uint16_t> jh(Mpad * Mpad, 0), jl(Mpad * Mpad, 0);
    bool exact = true;
    for (int i = 0; i < N; ++i)
        for (int64_t k = ctx->row_ptr[i]; k < ctx->row_ptr[i + 1]; ++k) {
            const float v = ctx->val[k] * hqa_dense::kF16JScale;
            const uint16_t b = f16_bits(v);
            const float r = v - f16_val(b);
            exact = exact && r == 0.f;
            jh[(size_t)i * Mpad + ctx->col[k]] = b;
            jl[(size_t)i * Mpad + ctx->col[k]] = f16_bits(r);
        }
    ++ctx->generation;
    hqa_status s = upload16(jh, Mpad, Mpad, true, &ctx->d_Jh, &ctx->tmJh);
    if (s != HQA_OK) return s;
    if (!exact) {
        s = upload16(concat3(jh, jl, Mpad), Mpad, 3 * Mpad, true, &ctx->d_Jhcat, &ctx->tmJh3);
        if (s != HQA_OK) return s;
    }
    ctx->dense_exact16 = exact;
    ctx->dense_f16 = true;
    return HQA_OK;
}

bool hqa_tc_precision(int prec)
{
    return prec == HQA_PREC_BF16 || prec == HQA_PREC_BF16X2 || prec == HQA_PREC_FP16 ||
           prec == HQA_PREC_FP16X2;
}

static bool is_f16(int prec) { return prec == HQA_PREC_FP16 || prec == HQA_PREC_FP16X2; }
static bool is_split(int prec) { return prec == HQA_PREC_BF16X2 || prec == HQA_PREC_FP16X2; }

hqa_status hqa_dense_prepare(hqa_ctx* ctx, int prec)
{
    if (!ctx->dense_tc || !hqa_tc_precision(prec)) return HQA_ERR_UNSUPPORTED;
    return is_f16(prec) ? dense_setup_f16(ctx) : HQA_OK;
}

hqa_status hqa_dense_field(hqa_ctx* ctx, int32_t R, const float* phi, float* L, int prec,
                           cudaStream_t st)
{
    if (prec != HQA_PREC_BF16 && prec != HQA_PREC_FP16) return HQA_ERR_UNSUPPORTED;
    hqa_status s = hqa_dense_prepare(ctx, prec);
    if (s != HQA_OK) return s;
    const bool f16 = prec == HQA_PREC_FP16;
    const int Kpad = ctx->Mpad;
    const int Rpad = (R + kFieldBN - 1) / kFieldBN * kFieldBN;
    const size_t bytes = (size_t)Rpad * Kpad * sizeof(uint16_t);
    s = hqa_reserve(ctx, &ctx->d_ws, &ctx->ws_cap, bytes);
    if (s != HQA_OK) return s;
    uint16_t* phib = static_cast<uint16_t*>(ctx->d_ws);
    const int g = (int)std::min<size_t>(4096, (bytes / 2 + 255) / 256);
    if (f16)
        k_phi_to_16<true><<<g, 256, 0, st>>>(phi, R, ctx->N, Rpad, Kpad, hqa_dense::kF16PhiScale, phib);
    else
        k_phi_to_16<false><<<g, 256, 0, st>>>(phi, R, ctx->N, Rpad, Kpad, 1.f, phib);
    CUtensorMap tmB;
    if (!make_tmap16(&tmB, phib, Rpad, Kpad, kFieldBN, f16)) return HQA_ERR_CUDA;
    FieldArgs a{};
    a.L = L;
    a.phi = phi;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.status = ctx->d_status;
    a.lscale = f16 ? hqa_dense::kF16LScale : 1.f;
    a.N = ctx->N;
    a.R = R;
    a.KT = Kpad / BK;
    const size_t smem = field_smem<kFieldBN, kFieldStages>();
    const void* fn = f16 ? (const void*)k_dense_field<kFieldBN, kFieldStages, true>
                         : (const void*)k_dense_field<kFieldBN, kFieldStages, false>;
    if (hqa_smem_attr(fn, smem) != cudaSuccess) return HQA_ERR_CUDA;
    const dim3 grid(ctx->Mpad / BM, Rpad / kFieldBN);
    if (f16)
        k_dense_field<kFieldBN, kFieldStages, true><<<grid, 192, smem, st>>>(ctx->tmJh, tmB, a);
    else
        k_dense_field<kFieldBN, kFieldStages, false><<<grid, 192, smem, st>>>(ctx->tmJ, tmB, a);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

bool hqa_dense_md_possible(const hqa_ctx* ctx, int32_t R)
{
    if (!ctx->dense_tc || R < 1) return false;
    return hqa_dense::pick_nh(ctx->Mpad / BM, 1, ctx->sm_count) > 0;   // larger R runs in chunks
}

namespace {

// K segments of the tensor-core product: 1 (one 16-bit operand), 2 (split Phi
// against a J exact in the format, J reused), 3 (split Phi against a split J).
int kseg_of(const hqa_ctx* ctx, int prec)
{
    if (!is_split(prec)) return 1;
    const bool exact = is_f16(prec) ? ctx->dense_exact16 : ctx->dense_exact;
    return exact ? 2 : 3;
}

// Bytes one step touches for R replicas: FP32 phi and p, the two 16-bit
// operand buffers (kseg segments each) and the coupling operand.
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
// costs its MMA columns (NH per half, times the K segments) plus a fixed part
// worth ~150 columns (streaming its 128-row coupling tile through shared
// memory, the column-group barrier, pipeline fill), measured on K2000; a chunk
// whose step touches more than ~70% of L2 streams its state from HBM every
// step, which about doubles the step.  C minimises the sum over chunks.
int dense_chunks(const hqa_ctx* ctx, int32_t R, int prec)
{
    const int kseg = kseg_of(ctx, prec);
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
    const int h = hqa_dense::pick_nh(Mt, R, ctx->sm_count);
    if (h == 0) return 0;
    const int nc = (R + 2 * h - 1) / (2 * h);
    *nh = h;
    *grid = Mt * nc;
    return 1;
}

static hqa_status dense_md_chunk(hqa_ctx* ctx, const StepCoef* d_sched, int64_t S, int32_t W,
                                 int32_t R, int32_t rep0, uint64_t seed, int init,
                                 const float* phi0, const float* p0, int M, float* phi_out,
                                 float* p_out, float* phibar_out, int prec, cudaStream_t st)
{
    int NH = 0, grid = 0;
    if (!hqa_dense_md_geometry(ctx, R, &NH, &grid)) return HQA_ERR_TOO_LARGE;
    const bool f16 = is_f16(prec);
    const int Mt = ctx->Mpad / BM;
    const int Nc = grid / Mt;
    const int Rpad = Nc * 2 * NH;
    const int Npad = ctx->Mpad;
    const size_t n = (size_t)Rpad * Npad;
    const int kseg = kseg_of(ctx, prec);
    const size_t nb = (size_t)kseg * n;   // operand elements per buffer
    // state: phi, p, w (FP32), two 16-bit operand buffers, 2 Nc counters
    const size_t off_p = n * 4, off_w = 2 * n * 4, off_b = 3 * n * 4, off_g = off_b + 2 * nb * 2;
    const size_t need = off_g + (size_t)2 * Nc * sizeof(unsigned int);
    hqa_status s = hqa_reserve(ctx, &ctx->d_state, &ctx->state_cap, need);
    if (s != HQA_OK) return s;
    char* b = static_cast<char*>(ctx->d_state);
    DenseMDArgs a{};
    a.phi = reinterpret_cast<float*>(b);
    a.p = reinterpret_cast<float*>(b + off_p);
    a.w = reinterpret_cast<float*>(b + off_w);
    a.phib = reinterpret_cast<uint16_t*>(b + off_b);
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
    a.oscale = f16 ? hqa_dense::kF16PhiScale : 1.f;
    a.lscale = f16 ? hqa_dense::kF16LScale : 1.f;
    if (ctx->wait_flag) {   // one-shot: the first chunk of the next launch
        a.wait_flag = static_cast<const unsigned int*>(ctx->wait_flag);
        a.wait_step = ctx->wait_step;
        a.wait_ns = ctx->wait_ns;
        ctx->wait_flag = nullptr;
    }
    CUtensorMap tmB;
    // a CTA of a pair stages half of each NH-replica phi tile
    const uint32_t box_rows = hqa_dense::use_pair(NH, Mt) ? NH / 2 : NH;
    if (!make_tmap16(&tmB, a.phib, (uint64_t)2 * Rpad, (uint64_t)kseg * Npad, box_rows, f16))
        return HQA_ERR_CUDA;
    // the epilogue's operand stores: 128 spins x 16 replicas per box, unswizzled
    CUtensorMap tmS;
    if (!make_tmap16_box(&tmS, a.phib, (uint64_t)2 * Rpad, (uint64_t)kseg * Npad, 128, 16, false, f16))
        return HQA_ERR_CUDA;
    const CUtensorMap& tmA = f16 ? (kseg == 3 ? ctx->tmJh3 : ctx->tmJh)
                                 : (kseg == 3 ? ctx->tmJ3 : ctx->tmJ);
    const int g = (int)std::min<size_t>(8192, (n + 255) / 256);
    if (f16) hqa_dense::k_dense_init<true><<<g, 256, 0, st>>>(a, seed, init, phi0, p0, kseg);
    else hqa_dense::k_dense_init<false><<<g, 256, 0, st>>>(a, seed, init, phi0, p0, kseg);
    if (cudaMemsetAsync(a.gbar, 0, (size_t)2 * Nc * sizeof(unsigned int), st) != cudaSuccess)
        return HQA_ERR_CUDA;
    s = f16 ? hqa_dense::dense_md_dispatch<true>(ctx, a, NH, kseg, grid, st, tmA, tmB, tmS)
            : hqa_dense::dense_md_dispatch<false>(ctx, a, NH, kseg, grid, st, tmA, tmB, tmS);
    if (s != HQA_OK) return s;
    const int64_t nwin = S < W ? S : W;
    hqa_dense::k_dense_out<<<std::min<size_t>(8192, ((size_t)R * ctx->N + 255) / 256), 256, 0, st>>>(
        a, 1.0f / (float)nwin, phi_out, p_out, phibar_out);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

int hqa_dense_md_chunks(const hqa_ctx* ctx, int32_t R, int prec)
{
    return dense_chunks(ctx, R, prec);
}

hqa_status hqa_dense_launch_md(hqa_ctx* ctx, const StepCoef* d_sched, int64_t S, int32_t W,
                               int32_t R, uint64_t seed, int init, const float* phi0,
                               const float* p0, int M, float* phi_out, float* p_out,
                               float* phibar_out, int prec, cudaStream_t st)
{
    hqa_status s = hqa_dense_prepare(ctx, prec);
    if (s != HQA_OK) return s;
    const int C = dense_chunks(ctx, R, prec);
    const int Rc = (R + C - 1) / C;
    const size_t N = (size_t)ctx->N;
    for (int r0 = 0; r0 < R; r0 += Rc) {
        const int Rk = std::min(Rc, R - r0);
        const size_t o = (size_t)r0 * N;
        s = dense_md_chunk(ctx, d_sched, S, W, Rk, r0, seed, init, phi0 ? phi0 + o : nullptr,
                           p0 ? p0 + o : nullptr, M, phi_out ? phi_out + o : nullptr,
                           p_out ? p_out + o : nullptr, phibar_out ? phibar_out + o : nullptr,
                           prec, st);
        if (s != HQA_OK) return s;
    }
    return HQA_OK;
}

template hqa_status hqa_dense::dense_md_dispatch<false>(hqa_ctx*, const DenseMDArgs&, int, int, int,
                                                        cudaStream_t, const CUtensorMap&,
                                                        const CUtensorMap&, const CUtensorMap&);

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
