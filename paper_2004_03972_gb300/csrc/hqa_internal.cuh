// hqa_internal.cuh -- context layout, status bits and launch helpers shared by
// the library's translation units (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <vector>

#include "../../include/hqa.h"

// Device-side status bits, OR-ed into ctx->d_status by kernels.
enum : uint32_t {
    HQA_DEV_NONFINITE = 1u << 0,
    HQA_DEV_BAD_SUBPROBLEM = 1u << 1,
    HQA_DEV_TIMEOUT = 1u << 2,
};

#define HQA_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            (void)cudaGetLastError();                        \
            return _e == cudaErrorMemoryAllocation ? HQA_ERR_OOM : HQA_ERR_CUDA; \
        }                                                    \
    } while (0)

// The potential's force term phi^(M-1) = phi (phi^2)^((M-2)/2), for the even
// M in [2, 12] that hqa_create_schedule accepts: at most kMaxMHalf squarings,
// written as a fixed sequence of predicated multiplications.  A loop with a
// data-dependent trip count inside an unrolled per-element update keeps the
// compiler from interleaving the independent elements; this form performs
// the same multiplications in the same order (bitwise identical results).
constexpr int kMaxMHalf = 5;

__device__ __forceinline__ float pot_pow(float phi, float phi2, int mhalf)
{
    float pw = phi;
#pragma unroll
    for (int q = 0; q < kMaxMHalf; ++q)
        if (q < mhalf) pw = __fmul_rn(pw, phi2);
    return pw;
}

// One step of the kick/drift coefficient table (see hqa_run).
struct StepCoef {
    float kA;  // c_j h alpha(j dt) M       multiplies phi^(M-1)
    float kB;  // c_j h beta(j dt)          multiplies the local field
    float dA;  // h alpha((j + 1/2) dt)     multiplies p in the drift
    float pad;
};

// Resident sparse plan for one (replicas-per-block, operand precision).
// Rows are grouped into "tuples" of G = 32 / RB rows; one warp evaluates a
// tuple with lane = (row slot g, replica r).  Each tuple's neighbour lists
// are padded to a common length, split into an all-positive and an
// all-negative section, and packed as chunks of 4 byte offsets per lane.
struct SparsePlan {
    int RB = 0, G = 0, T = 0, Npad = 0, prec = 0;
    int64_t chunks = 0;
    uint4* d_entries = nullptr;   // [chunk][G] uint4: byte offsets of phi rows in one buffer
    int4* d_tuples = nullptr;     // [T] {first chunk, positive chunks, negative chunks, 0}
    int* d_tuple_rows = nullptr;  // [T][G] row index or -1
    double pad_ratio = 0.0;       // stored positions / nnz
    double conflict_ratio = 0.0;  // bank wavefronts / conflict-free wavefronts (host model)
    // vectorised variant (sparse_md_vec.cu): 16-byte gathers, entries staged in shared memory
    bool vec = false;
    int NW = 0;                   // warps per CTA
    int P = 0;                    // rows per bank phase
    size_t ent_bytes = 0;         // packed u16 neighbour offsets (bytes)
    int* d_slot_of_row = nullptr; // [N] shared-memory slot of each row (vectorised plan)
    int* d_warp_off = nullptr;    // [NW + 1] offsets into d_tuple_list
    int* d_tuple_list = nullptr;  // tuples in per-warp order
    double balance = 0.0;         // mean warp load / max warp load
    int max_wt = 0;               // most tuples any warp owns (register-resident state if <= 4)
};

// Orders one section of G neighbour lists into K positions so that rows read
// at one position fall in distinct bank groups (row j -> group j mod P, the
// lists split into G / P phases of P rows) where possible; empty slots read
// zero rows N .. N+P-1.  Adds the modelled wavefront count to `wavefronts`.
void hqa_schedule_bank_section(const std::vector<std::vector<int>>& lists, int P, int N, int K,
                               std::vector<int>& out /* [K][G] */, int64_t& wavefronts);

// Per-instance table of a batch context (device copy used by batch kernels).
struct BatchInst {
    const int32_t* row_ptr;
    const int32_t* col;
    const int8_t* val_i8;
    const int32_t* h_i32;
    int64_t sumJ;
    int64_t off;   // spins of the instances before this one
    int32_t N;
    int32_t pad;
};

struct hqa_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    struct Dep {
        hqa_ctx* ctx;
        uint64_t uid;          // the context's unique id (addresses can be reused)
        uint64_t generation;   // its generation at capture
    };
    std::vector<Dep> deps;
};

struct hqa_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    size_t l2_bytes = 0;
    int32_t N = 0;
    int64_t nnz = 0;            // stored off-diagonal entries (both triangles)
    bool dense_input = false;
    bool integer = false;       // all J and h integral with |J| <= 127, |h| <= 2^20
    bool unit = false;          // all J in {-1, 0, +1}
    bool has_h = false;

    // host copies of the symmetric CSR (diagonal dropped), used to build plans
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<float> val;
    std::vector<float> h;

    // device copies
    int32_t* d_row_ptr = nullptr;  // N+1 (int32: nnz < 2^31 enforced)
    int32_t* d_col = nullptr;
    float* d_val = nullptr;
    int8_t* d_val_i8 = nullptr;    // integer path
    float* d_h = nullptr;          // N or null
    int32_t* d_h_i32 = nullptr;    // integer path
    int64_t sum_J_all = 0;         // sum of all stored entries (integer path)

    std::map<int, SparsePlan> plans;   // key = RB * 16 + prec

    // schedule table cache
    std::vector<StepCoef> sched_host;
    StepCoef* d_sched = nullptr;
    size_t sched_cap = 0;

    // grow-only workspaces: run temporaries, MD state spilled from shared
    // memory, sub-solve scratch
    void* d_ws = nullptr;
    size_t ws_cap = 0;
    void* d_state = nullptr;
    size_t state_cap = 0;
    void* d_sub = nullptr;
    size_t sub_cap = 0;
    void* d_feat = nullptr;         // surrogate features / readout scratch
    size_t feat_cap = 0;
    void* d_diag = nullptr;         // H_MD diagnostic: local field
    size_t diag_cap = 0;
    void* d_efx = nullptr;          // fixed-point energy: spin masks and partial sums
    size_t efx_cap = 0;
    int fx_shift = -1;              // its grid 2^-fx_shift (computed on first use)
    void* d_tune = nullptr;         // autotuner probe outputs
    size_t tune_cap = 0;
    // autotuned (kernel, replicas per block) per (replicas, precision); used by
    // hqa_run when the options leave both to the library
    std::map<std::pair<int, int>, std::pair<int, int>> tuned;
    uint32_t* d_status = nullptr;

    // batch contexts: member contexts (not owned), spin offsets, device tables
    bool is_batch = false;
    std::vector<hqa_ctx*> members;
    std::vector<int64_t> member_off;
    int64_t total_spins = 0;
    BatchInst* d_binst = nullptr;
    void* d_bwork = nullptr;        // per-run instance arguments, work items, queue counter
    size_t bwork_cap = 0;
    std::vector<char> bwork_host;   // what d_bwork holds (tables are uploaded only on change)
    // low-degree batch kernel: eligibility (0 unknown, 1 yes, -1 no), the members'
    // compact lists (built once) and per-run tables
    mutable int ld_state = 0;
    void* d_ld = nullptr;
    size_t ld_cap = 0;
    std::vector<int64_t> ld_off;
    void* d_ldwork = nullptr;
    size_t ldwork_cap = 0;
    std::vector<char> ldwork_host;
    // bumped whenever a device buffer of the context is reallocated or a device
    // table (schedule, batch work tables) is re-uploaded: captured graphs check it
    uint64_t generation = 0;
    uint64_t uid = 0;               // unique per created context

    // dense contexts whose couplings are exact in BF16: tensor-core operand
    bool dense_tc = false;
    void* d_Jbf = nullptr;         // [Mpad][Mpad] BF16, zero padded
    int Mpad = 0;
    CUtensorMap tmJ;               // TMA map of d_Jbf, 128 x 64 boxes
    // J exactly representable in BF16 (e.g. +-1); otherwise d_Jbf holds J rounded
    // to BF16 and d_Jcat the three-segment operand [J_hi | J_lo | J_hi] of the
    // split product J_hi Phi_hi + J_lo Phi_hi + J_hi Phi_lo
    bool dense_exact = false;
    // hqa_arm_wait_check: consumed by the next dense MD launch
    const void* wait_flag = nullptr;
    int64_t wait_step = 0;
    uint64_t wait_ns = 0;
    void* d_Jcat = nullptr;        // [Mpad][3 Mpad] BF16 (non-exact J only)
    CUtensorMap tmJ3;
    // FP16 tensor-core operands (built on first use): J scaled by 2^10 and rounded
    // to FP16, and the split [J_hi | J_lo | J_hi] when that rounding is not exact
    bool dense_f16 = false;
    bool dense_exact16 = false;
    void* d_Jh = nullptr;          // [Mpad][Mpad] FP16
    void* d_Jhcat = nullptr;       // [Mpad][3 Mpad] FP16 (J not exact in FP16 only)
    CUtensorMap tmJh;
    CUtensorMap tmJh3;
    // plain FP32 dense path (CUDA cores): J in FP32, [Npad32][Npad32], built on first use
    float* d_Jf32 = nullptr;
    int Npad32 = 0;
    // bit-mask integer energy (readout.cu): word-major nonzero and negative masks, degrees
    void* d_ebits = nullptr;
};

// Ensures *p holds at least `bytes` device bytes (frees and reallocates;
// cudaFree synchronises the device, so in-flight users are finished).
// During a capture a needed reallocation fails with HQA_ERR_UNSUPPORTED.
hqa_status hqa_reserve(hqa_ctx* ctx, void** p, size_t* cap, size_t bytes);

// Stream capture (hqa_capture_begin/end) of the calling thread: while it is
// open, anything that would allocate, upload from the host or synchronise
// returns HQA_ERR_UNSUPPORTED, and the first failure of a capturing call is
// kept for hqa_capture_end.
bool hqa_capturing();
// Records that the capture uses `ctx`'s device buffers: the graph refuses to
// replay once the context has reallocated or re-uploaded any of them.
void hqa_capture_touch(hqa_ctx* ctx);
double hqa_sched_alpha(const hqa_schedule* s, double tau);
double hqa_sched_beta(const hqa_schedule* s, double tau);
hqa_status hqa_capture_note(hqa_status s);

// Raises a kernel's dynamic shared-memory limit once (not per launch, so
// that captured launches make no attribute calls).
cudaError_t hqa_smem_attr(const void* kernel, size_t smem);

// sparse_md_vec.cu
bool hqa_vec_supported(const hqa_ctx* ctx, int RB, int prec);
size_t hqa_vec_smem_bytes(const hqa_ctx* ctx, int RB, int prec, size_t ent_bytes);
hqa_status hqa_vec_plan(hqa_ctx* ctx, int RB, int prec, const SparsePlan** out);
hqa_status hqa_vec_launch_md(hqa_ctx* ctx, const SparsePlan* plan, const StepCoef* d_sched,
                             int64_t S, int32_t W, int32_t R, uint64_t seed, int init,
                             const float* phi0, const float* p0, int M, float* phi_out,
                             float* p_out, float* phibar_out, cudaStream_t st);
hqa_status hqa_vec_launch_field(hqa_ctx* ctx, const SparsePlan* plan, int32_t R,
                                const float* phi, float* L, cudaStream_t st);

// sparse_stream.cu: operand and state in global memory, grid barrier per step
bool hqa_stream_supported(const hqa_ctx* ctx, int prec);
hqa_status hqa_stream_launch_md(hqa_ctx* ctx, int prec, const StepCoef* d_sched, int64_t S,
                                int32_t W, int32_t R, uint64_t seed, int init, const float* phi0,
                                const float* p0, int M, float* phi_out, float* p_out,
                                float* phibar_out, cudaStream_t st);
hqa_status hqa_stream_field(hqa_ctx* ctx, int prec, int32_t R, const float* phi, float* L,
                            cudaStream_t st);

// sparse_md.cu
hqa_status hqa_sparse_plan(hqa_ctx* ctx, int RB, int prec, const SparsePlan** out);
hqa_status hqa_batch_launch_md(hqa_ctx* batch, int RB, int prec, const StepCoef* d_sched,
                               int64_t S, int32_t W, int32_t R, uint64_t seed, int init,
                               const float* phi0, const float* p0, int M, float* phi_out,
                               float* p_out, float* phibar_out, cudaStream_t st);
int hqa_sparse_pick_rb(const hqa_ctx* ctx, int32_t R, int prec);
// batch_lowdeg.cu
bool hqa_lowdeg_eligible(const hqa_ctx* batch);
size_t hqa_lowdeg_smem_bytes(const hqa_ctx* batch, int RB, int prec);
int hqa_lowdeg_pick_rb(const hqa_ctx* batch, int32_t R, int prec);
hqa_status hqa_lowdeg_launch_md(hqa_ctx* batch, int RB, int prec, const StepCoef* d_sched,
                                int64_t S, int32_t W, int32_t R, uint64_t seed, int init,
                                const float* phi0, const float* p0, int M, float* phi_out,
                                float* p_out, float* phibar_out, cudaStream_t st);
size_t hqa_sparse_smem_bytes(const hqa_ctx* ctx, int RB, int prec);
hqa_status hqa_sparse_launch_md(hqa_ctx* ctx, const SparsePlan* plan, const StepCoef* d_sched,
                                int64_t S, int32_t W, int32_t R, uint64_t seed, int init,
                                const float* phi0, const float* p0, int M, float* phi_out,
                                float* p_out, float* phibar_out, cudaStream_t st);
hqa_status hqa_sparse_launch_field(hqa_ctx* ctx, const SparsePlan* plan, int32_t R,
                                   const float* phi, float* L, cudaStream_t st);

// dense_md.cu
hqa_status hqa_dense_setup(hqa_ctx* ctx, const float* J);
hqa_status hqa_dense_field(hqa_ctx* ctx, int32_t R, const float* phi, float* L, int prec,
                           cudaStream_t st);
bool hqa_dense_md_possible(const hqa_ctx* ctx, int32_t R);
int hqa_dense_md_geometry(const hqa_ctx* ctx, int32_t R, int* nh, int* grid);
int hqa_dense_md_chunks(const hqa_ctx* ctx, int32_t R, int prec);
// precision: HQA_PREC_BF16, _BF16X2, _FP16 or _FP16X2
bool hqa_tc_precision(int prec);
hqa_status hqa_dense_prepare(hqa_ctx* ctx, int prec);
hqa_status hqa_dense_launch_md(hqa_ctx* ctx, const StepCoef* d_sched, int64_t S, int32_t W,
                               int32_t R, uint64_t seed, int init, const float* phi0,
                               const float* p0, int M, float* phi_out, float* p_out,
                               float* phibar_out, int prec, cudaStream_t st);
// dense_simt.cu: the plain FP32 dense path on the CUDA cores
bool hqa_simt_possible(const hqa_ctx* ctx);
hqa_status hqa_simt_prepare(hqa_ctx* ctx);
hqa_status hqa_simt_field(hqa_ctx* ctx, int32_t R, const float* phi, float* L, cudaStream_t st);
hqa_status hqa_simt_launch_md(hqa_ctx* ctx, const StepCoef* d_sched, int64_t S, int32_t W,
                              int32_t R, uint64_t seed, int init, const float* phi0,
                              const float* p0, int M, float* phi_out, float* p_out,
                              float* phibar_out, cudaStream_t st);

// readout.cu
hqa_status hqa_launch_readout_batch(hqa_ctx* batch, int32_t R, const float* phibar, int32_t n,
                                    int8_t* spins, uint8_t* frozen, int32_t* tally, cudaStream_t st);
hqa_status hqa_launch_energy_batch(hqa_ctx* batch, int32_t R, const int8_t* spins, int64_t* energy,
                                   int64_t* cut, cudaStream_t st);
hqa_status hqa_launch_readout(hqa_ctx* ctx, int32_t R, const float* phibar, int32_t n,
                              int8_t* spins, uint8_t* frozen, int32_t* tally, cudaStream_t st);
hqa_status hqa_launch_energy(hqa_ctx* ctx, int32_t R, const int8_t* spins, int64_t* energy,
                             int64_t* cut, cudaStream_t st);
// may_allocate = false: never allocates (the bit-mask tables are used only when
// an earlier call built them; otherwise the per-coupling kernel runs)
hqa_status hqa_launch_energy_ex(hqa_ctx* ctx, int32_t R, const int8_t* spins, int64_t* energy,
                                int64_t* cut, cudaStream_t st, bool may_allocate);

// subsolve.cu
hqa_status hqa_launch_subsolve(hqa_ctx* ctx, int32_t R, const int8_t* spins,
                               const uint8_t* frozen, int32_t n, int8_t* out_spins,
                               int64_t* out_energy, cudaStream_t st);
