// sparse_stream.cu -- streaming sparse MD kernel for instances whose flux
// operand does not fit in one SM's shared memory (large N, many replicas).
//
// The state lives in global memory, spin-major and replica-contiguous:
//   op[2]  [N][Rpad] flux operand (FP32, or BF16 with an FP32 master copy),
//          double-buffered across steps; L2-resident at the sizes it serves
//          (N = 20000, 256 replicas: 10 MB in BF16)
//   phi    [N][Rpad] FP32 master (BF16 operand only)
//   p, w   [N][Rpad] FP32 momenta and window sums
// A "cell" is one spin i and one 16-byte vector of V replicas (V = 8 in BF16,
// 4 in FP32).  Cells are dealt to the threads of a persistent cooperative
// grid in row-major order, so the lanes of a warp cover consecutive vectors
// of a row: the gather of neighbour j's vectors is one coalesced read of
// row j (512 bytes for 256 replicas in BF16), and the lanes of a row share
// its neighbour list (broadcast loads of the CSR column and sign).  Each step
// (Methods, "Leapfrog algorithm"):
//   L = sum_k J_ik op[cur][col_k][v] + 2 h_i |phi_i|,
//   p <- p - (kA phi^(M-1) + kB L),  phi <- phi + dA p,
// writes op[nxt], and ends with a grid-wide barrier: an arrival counter
// (release by __threadfence, acquire by ld.acquire) whose wait gives up after
// 2 s, latches HQA_ERR_TIMEOUT and makes every CTA leave.  Operand reads of
// other SMs' writes bypass L1 (ld.global.cg); each thread's own p, phi and w
// are private to it across steps.
#include <cuda_bf16.h>

#include <algorithm>

#include "hqa_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kGatherBatch = 4;   // neighbour gathers issued together
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s bound on the grid barrier

struct StreamArgs {
    const int32_t* row_ptr;
    const int32_t* col;
    const int8_t* val;
    const float* h;        // [N] or null
    const StepCoef* sched;
    void* op0;             // [N][Rpad] operand buffers (FP32 or BF16)
    void* op1;
    float* phi;            // [N][Rpad] FP32 master (BF16 operand only)
    float* p;
    float* w;
    unsigned int* bar;     // grid barrier arrival counter
    uint32_t* status;
    int64_t S;
    int W, N, Rpad, M;
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier on a monotonic counter: every CTA arrives once per step;
// returns false (on every thread of the CTA) when the wait timed out here or
// another CTA latched a timeout.
__device__ bool grid_sync(unsigned int* bar, unsigned int target, uint32_t* status)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        const uint64_t t0 = globaltimer();
        uint32_t spins = 0;
        while (ld_acquire(bar) < target) {
            if ((++spins & 63u) == 0) {
                if (*(volatile uint32_t*)status & HQA_DEV_TIMEOUT) { ok = 0; break; }
                if (globaltimer() - t0 > kWaitNs) {
                    atomicOr(status, HQA_DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <bool BF16>
struct Vec;
template <>
struct Vec<false> {   // 4 FP32 replicas
    static constexpr int V = 4;
    __device__ static void load(const void* base, size_t e, float (&x)[4])
    {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(static_cast<const float*>(base) + e));
        x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
    }
    __device__ static void store(void* base, size_t e, const float (&x)[4])
    {
        *reinterpret_cast<float4*>(static_cast<float*>(base) + e) = make_float4(x[0], x[1], x[2], x[3]);
    }
};
template <>
struct Vec<true> {    // 8 BF16 replicas
    static constexpr int V = 8;
    __device__ static void load(const void* base, size_t e, float (&x)[8])
    {
        const uint4 q = __ldcg(reinterpret_cast<const uint4*>(
            static_cast<const __nv_bfloat16*>(base) + e));
        const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x[2 * k] = __uint_as_float(u[k] << 16);
            x[2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
        }
    }
    __device__ static void store(void* base, size_t e, const float (&x)[8])
    {
        uint32_t u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(x[2 * k]));
            const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(x[2 * k + 1]));
            u[k] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(base) + e) =
            make_uint4(u[0], u[1], u[2], u[3]);
    }
};

// Field of one cell (row i, replica vector starting at column c) from operand `op`.
template <bool BF16>
__device__ __forceinline__ void cell_field(const StreamArgs& a, const void* op, int i, int c,
                                           float (&L)[Vec<BF16>::V])
{
    constexpr int V = Vec<BF16>::V;
#pragma unroll
    for (int e = 0; e < V; ++e) L[e] = 0.f;
    const int k0 = __ldg(a.row_ptr + i), k1 = __ldg(a.row_ptr + i + 1);
    int k = k0;
    // four neighbours' gathers in flight at once (the same accumulation order)
    for (; k + kGatherBatch <= k1; k += kGatherBatch) {
        int j[kGatherBatch];
        float s[kGatherBatch], x[kGatherBatch][V];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            j[u] = __ldg(a.col + k + u);
            s[u] = (float)__ldg(a.val + k + u);
        }
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) Vec<BF16>::load(op, (size_t)j[u] * a.Rpad + c, x[u]);
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u)
#pragma unroll
            for (int e = 0; e < V; ++e) L[e] = fmaf(s[u], x[u][e], L[e]);
    }
    for (; k < k1; ++k) {
        const int j = __ldg(a.col + k);
        const float s = (float)__ldg(a.val + k);
        float x[V];
        Vec<BF16>::load(op, (size_t)j * a.Rpad + c, x);
#pragma unroll
        for (int e = 0; e < V; ++e) L[e] = fmaf(s, x[e], L[e]);
    }
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads) k_sparse_stream(const StreamArgs a)
{
    constexpr int V = Vec<BF16>::V;
    const int nv = a.Rpad / V;
    const int64_t cells = (int64_t)a.N * nv;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t win0 = a.S - (int64_t)a.W;
    const int mhalf = (a.M - 2) / 2;
    for (int64_t m = 0; m < a.S; ++m) {
        const float4 cf = __ldg(reinterpret_cast<const float4*>(a.sched) + m);
        const void* cur = (m & 1) ? a.op1 : a.op0;
        void* nxt = (m & 1) ? a.op0 : a.op1;
        const bool in_win = m >= win0;
        for (int64_t cell = t0; cell < cells; cell += T) {
            const int i = (int)(cell / nv), c = (int)(cell % nv) * V;
            float L[V];
            cell_field<BF16>(a, cur, i, c, L);
            const size_t o = (size_t)i * a.Rpad + c;
            float ph[V], pp[V];
            if constexpr (BF16) {
#pragma unroll
                for (int e = 0; e < V; e += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(a.phi + o + e);
                    ph[e] = q.x; ph[e + 1] = q.y; ph[e + 2] = q.z; ph[e + 3] = q.w;
                }
            } else {
                Vec<false>::load(cur, o, ph);
            }
#pragma unroll
            for (int e = 0; e < V; e += 4) {
                const float4 q = *reinterpret_cast<const float4*>(a.p + o + e);
                pp[e] = q.x; pp[e + 1] = q.y; pp[e + 2] = q.z; pp[e + 3] = q.w;
            }
            const float hr = a.h ? 2.f * __ldg(a.h + i) : 0.f;
            float fn[V];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const float Le = hr != 0.f ? L[e] + hr * fabsf(ph[e]) : L[e];
                const float phi2 = ph[e] * ph[e];
                const float pw = pot_pow(ph[e], phi2, mhalf);
                pp[e] = pp[e] - fmaf(cf.x, pw, cf.y * Le);
                fn[e] = fmaf(cf.z, pp[e], ph[e]);
            }
#pragma unroll
            for (int e = 0; e < V; e += 4) {
                *reinterpret_cast<float4*>(a.p + o + e) = make_float4(pp[e], pp[e + 1], pp[e + 2], pp[e + 3]);
                if constexpr (BF16)
                    *reinterpret_cast<float4*>(a.phi + o + e) =
                        make_float4(fn[e], fn[e + 1], fn[e + 2], fn[e + 3]);
                if (in_win) {
                    float4 q = *reinterpret_cast<float4*>(a.w + o + e);
                    q.x += fn[e]; q.y += fn[e + 1]; q.z += fn[e + 2]; q.w += fn[e + 3];
                    *reinterpret_cast<float4*>(a.w + o + e) = q;
                }
            }
            Vec<BF16>::store(nxt, o, fn);
        }
        if (!grid_sync(a.bar, (unsigned int)(gridDim.x * (m + 1)), a.status)) return;
    }
}

// Field only: L[r][i] = sum_k J_ik phi[r][col_k] + 2 h_i |phi[r][i]| from an
// operand already in the streaming layout.
template <bool BF16>
__global__ void __launch_bounds__(kThreads) k_sparse_stream_field(const StreamArgs a, int R,
                                                                  const float* phi_in, float* L_out)
{
    constexpr int V = Vec<BF16>::V;
    const int nv = a.Rpad / V;
    const int64_t cells = (int64_t)a.N * nv;
    for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < cells;
         cell += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(cell / nv), c = (int)(cell % nv) * V;
        float L[V];
        cell_field<BF16>(a, a.op0, i, c, L);
        const float hr = a.h ? 2.f * __ldg(a.h + i) : 0.f;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int r = c + e;
            if (r >= R) continue;
            float v = L[e];
            if (hr != 0.f) v += hr * fabsf(phi_in[(size_t)r * a.N + i]);
            L_out[(size_t)r * a.N + i] = v;
        }
    }
}

// phi(0), p(0) (SplitMix64 or the caller's [R][N] arrays) into the streaming
// layout; window sums and padding replicas zero.
template <bool BF16>
__global__ void k_stream_init(StreamArgs a, int R, uint64_t seed, int init, const float* phi0,
                              const float* p0)
{
    const size_t total = (size_t)a.N * a.Rpad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / a.Rpad), r = (int)(idx % a.Rpad);
        float f = 0.f, q = 0.f;
        if (r < R) {
            const uint64_t c = ((uint64_t)r << 32) | (uint64_t)i;
            if (init == HQA_INIT_GIVEN) {
                f = phi0[(size_t)r * a.N + i];
                q = p0[(size_t)r * a.N + i];
            } else {
                uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;  // SplitMix64
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                z ^= z >> 31;
                q = (z >> 63) ? -1.f : 1.f;
                if (init == HQA_INIT_RANDOM_FLUX) {
                    uint64_t y = seed + ((c | (1ull << 62)) + 1ull) * 0x9E3779B97F4A7C15ull;
                    y = (y ^ (y >> 30)) * 0xBF58476D1CE4E5B9ull;
                    y = (y ^ (y >> 27)) * 0x94D049BB133111EBull;
                    y ^= y >> 31;
                    f = (float)((int64_t)(y >> 40) - (1 << 23)) * 0x1p-26f;
                }
            }
        }
        if constexpr (BF16) {
            static_cast<__nv_bfloat16*>(a.op0)[idx] = __float2bfloat16_rn(f);
            a.phi[idx] = f;
        } else {
            static_cast<float*>(a.op0)[idx] = f;
        }
        a.p[idx] = q;
        a.w[idx] = 0.f;
    }
}

// [R][N] operand from the caller's phi (field only).
template <bool BF16>
__global__ void k_stream_load(StreamArgs a, int R, const float* phi)
{
    const size_t total = (size_t)a.N * a.Rpad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / a.Rpad), r = (int)(idx % a.Rpad);
        const float f = r < R ? phi[(size_t)r * a.N + i] : 0.f;
        if constexpr (BF16) static_cast<__nv_bfloat16*>(a.op0)[idx] = __float2bfloat16_rn(f);
        else static_cast<float*>(a.op0)[idx] = f;
    }
}

template <bool BF16>
__global__ void k_stream_out(StreamArgs a, int R, const void* fin, float inv_w, float* phi_out,
                             float* p_out, float* phibar_out)
{
    const size_t total = (size_t)R * a.N;
    bool bad = false;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / a.N), i = (int)(idx % a.N);
        const size_t o = (size_t)i * a.Rpad + r;
        const float f = BF16 ? a.phi[o] : static_cast<const float*>(fin)[o];
        const float q = a.p[o];
        if (phi_out) phi_out[idx] = f;
        if (p_out) p_out[idx] = q;
        if (phibar_out) phibar_out[idx] = a.w[o] * inv_w;
        bad |= !(isfinite(f) && isfinite(q));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, HQA_DEV_NONFINITE);
}

int grid_1d(size_t n) { return (int)std::min<size_t>(8192, (n + 255) / 256); }

// Workspace: operand buffers, FP32 master (BF16), p, w, barrier counter.
hqa_status stream_args(hqa_ctx* ctx, int32_t R, bool bf16, StreamArgs* a)
{
    const int V = bf16 ? 8 : 4;
    const int Rpad = (R + V - 1) / V * V;
    const size_t n = (size_t)ctx->N * Rpad;
    const size_t es = bf16 ? 2 : 4;
    const auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t off_op1 = up(n * es), off_phi = off_op1 + up(n * es);
    const size_t off_p = off_phi + (bf16 ? up(n * 4) : 0), off_w = off_p + up(n * 4);
    const size_t off_bar = off_w + up(n * 4), need = off_bar + 256;
    hqa_status s = hqa_reserve(ctx, &ctx->d_state, &ctx->state_cap, need);
    if (s != HQA_OK) return s;
    char* b = static_cast<char*>(ctx->d_state);
    *a = StreamArgs{};
    a->row_ptr = ctx->d_row_ptr;
    a->col = ctx->d_col;
    a->val = ctx->d_val_i8;
    a->h = ctx->has_h ? ctx->d_h : nullptr;
    a->op0 = b;
    a->op1 = b + off_op1;
    a->phi = bf16 ? reinterpret_cast<float*>(b + off_phi) : nullptr;
    a->p = reinterpret_cast<float*>(b + off_p);
    a->w = reinterpret_cast<float*>(b + off_w);
    a->bar = reinterpret_cast<unsigned int*>(b + off_bar);
    a->status = ctx->d_status;
    a->N = ctx->N;
    a->Rpad = Rpad;
    return HQA_OK;
}

}  // namespace

bool hqa_stream_supported(const hqa_ctx* ctx, int prec)
{
    return !ctx->is_batch && ctx->unit && ctx->integer && ctx->d_val_i8 &&
           (prec == HQA_PREC_FP32 || prec == HQA_PREC_BF16);
}

hqa_status hqa_stream_launch_md(hqa_ctx* ctx, int prec, const StepCoef* d_sched, int64_t S,
                                int32_t W, int32_t R, uint64_t seed, int init, const float* phi0,
                                const float* p0, int M, float* phi_out, float* p_out,
                                float* phibar_out, cudaStream_t st)
{
    if (!hqa_stream_supported(ctx, prec)) return HQA_ERR_UNSUPPORTED;
    const bool bf16 = prec == HQA_PREC_BF16;
    StreamArgs a;
    hqa_status s = stream_args(ctx, R, bf16, &a);
    if (s != HQA_OK) return s;
    a.sched = d_sched;
    a.S = S;
    a.W = W;
    a.M = M;
    const size_t n = (size_t)ctx->N * a.Rpad;
    if (bf16) k_stream_init<true><<<grid_1d(n), 256, 0, st>>>(a, R, seed, init, phi0, p0);
    else k_stream_init<false><<<grid_1d(n), 256, 0, st>>>(a, R, seed, init, phi0, p0);
    if (cudaMemsetAsync(a.bar, 0, sizeof(unsigned int), st) != cudaSuccess) return HQA_ERR_CUDA;
    // persistent grid: every CTA co-resident (the per-step barrier waits on all of them)
    const void* fn = bf16 ? (const void*)k_sparse_stream<true> : (const void*)k_sparse_stream<false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        return HQA_ERR_CUDA;
    }
    const int64_t cells = (int64_t)ctx->N * (a.Rpad / (bf16 ? 8 : 4));
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)per_sm * ctx->sm_count, (cells + kThreads - 1) / kThreads));
    void* args[] = {&a};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return hqa_capture_note(hqa_capturing() ? HQA_ERR_UNSUPPORTED : HQA_ERR_CUDA);
    }
    const int64_t nwin = S < W ? S : W;
    const void* fin = (S & 1) ? a.op1 : a.op0;
    if (bf16)
        k_stream_out<true><<<grid_1d((size_t)R * ctx->N), 256, 0, st>>>(
            a, R, fin, 1.0f / (float)nwin, phi_out, p_out, phibar_out);
    else
        k_stream_out<false><<<grid_1d((size_t)R * ctx->N), 256, 0, st>>>(
            a, R, fin, 1.0f / (float)nwin, phi_out, p_out, phibar_out);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_stream_field(hqa_ctx* ctx, int prec, int32_t R, const float* phi, float* L,
                            cudaStream_t st)
{
    if (!hqa_stream_supported(ctx, prec)) return HQA_ERR_UNSUPPORTED;
    const bool bf16 = prec == HQA_PREC_BF16;
    StreamArgs a;
    hqa_status s = stream_args(ctx, R, bf16, &a);
    if (s != HQA_OK) return s;
    const size_t n = (size_t)ctx->N * a.Rpad;
    const int64_t cells = (int64_t)ctx->N * (a.Rpad / (bf16 ? 8 : 4));
    const int g = (int)std::min<int64_t>(8192, (cells + kThreads - 1) / kThreads);
    if (bf16) {
        k_stream_load<true><<<grid_1d(n), 256, 0, st>>>(a, R, phi);
        k_sparse_stream_field<true><<<g, kThreads, 0, st>>>(a, R, phi, L);
    } else {
        k_stream_load<false><<<grid_1d(n), 256, 0, st>>>(a, R, phi);
        k_sparse_stream_field<false><<<g, kThreads, 0, st>>>(a, R, phi, L);
    }
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}
