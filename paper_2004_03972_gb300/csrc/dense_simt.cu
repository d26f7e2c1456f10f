// dense_simt.cu -- the plain FP32 dense local field and MD step on the CUDA
// cores (no tensor cores, no reduced precision).
//
// It is the FP32 reference form of the dense path: the field of all replicas
// is the product L = J Phi (Methods, "Leapfrog algorithm"), evaluated with
// FP32 fused multiply-adds, and each leapfrog step is one launch of a tiled
// SGEMM whose epilogue applies the kick and drift to its tile.
//
// Layout: the state is spin-major, [Npad][Rpad] (replicas contiguous), so
// that both GEMM operands load as contiguous rows: the coupling tile
// As[k][i] = J[k][i0 + i] is row k of J (J is symmetric, J[i][k] = J[k][i])
// and the flux tile Bs[k][r] = phi[k][r0 + r] is row k of the state.  A CTA
// owns a 128-spin x 128-replica output tile; 256 threads each accumulate an
// 8 x 8 sub-tile (spins {4ty..4ty+3, 64+4ty..}, replicas {4tx..4tx+3,
// 64+4tx..}) over K in steps of 8, with the next k-slice loaded into
// registers while the current one is multiplied out of shared memory.
#include <algorithm>
#include <vector>

#include "hqa_internal.cuh"

namespace {

constexpr int TM = 128, TN = 128, TK = 8, kThreads = 256;

struct SimtArgs {
    const float* J;      // [Npad][Npad], zero padded, zero diagonal
    const float* phi;    // [Npad][Rpad] phi^(m) (operand and master)
    float* phi_next;     // [Npad][Rpad] phi^(m+1)
    float* p;            // [Npad][Rpad]
    float* w;            // [Npad][Rpad] window sums
    float* L;            // field mode: [R][N] output
    const float* h;      // [N] or null
    const StepCoef* sched;
    int64_t m;           // absolute index into sched
    int in_win;
    int N, Npad, Rpad, R, M;
};

// MODE 0: L = J phi + 2 h |phi| written to a.L ([R][N]).
// MODE 1: one leapfrog step (kick with sched[m], drift) of the tile.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_dense_simt(const SimtArgs a)
{
    __shared__ __align__(16) float As[2][TK][TM];
    __shared__ __align__(16) float Bs[2][TK][TN];
    const int t = threadIdx.x;
    const int ty = t / 16, tx = t % 16;
    const int i0 = blockIdx.y * TM, r0 = blockIdx.x * TN;
    // loader: k-row lk, 4 consecutive columns at 4 * lc
    const int lk = t / 32, lc = (t % 32) * 4;
    const float* Ag = a.J + (size_t)lk * a.Npad + i0 + lc;
    const float* Bg = a.phi + (size_t)lk * a.Rpad + r0 + lc;
    const size_t Astep = (size_t)TK * a.Npad, Bstep = (size_t)TK * a.Rpad;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra = *reinterpret_cast<const float4*>(Ag);
    float4 rb = *reinterpret_cast<const float4*>(Bg);
    *reinterpret_cast<float4*>(&As[0][lk][lc]) = ra;
    *reinterpret_cast<float4*>(&Bs[0][lk][lc]) = rb;
    __syncthreads();
    const int KT = a.Npad / TK;
    for (int kt = 0; kt < KT; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < KT) {
            ra = *reinterpret_cast<const float4*>(Ag + (size_t)(kt + 1) * Astep);
            rb = *reinterpret_cast<const float4*>(Bg + (size_t)(kt + 1) * Bstep);
        }
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + 4 * tx]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < KT) {
            *reinterpret_cast<float4*>(&As[cur ^ 1][lk][lc]) = ra;
            *reinterpret_cast<float4*>(&Bs[cur ^ 1][lk][lc]) = rb;
        }
        __syncthreads();
    }

    float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE == 1) cf = __ldg(reinterpret_cast<const float4*>(a.sched) + a.m);
    const int mhalf = (a.M - 2) / 2;
#pragma unroll
    for (int ih = 0; ih < 2; ++ih)
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
            const int i = i0 + 64 * ih + 4 * ty + ii;
            if (i >= a.N) continue;
            const float hr = a.h ? 2.f * a.h[i] : 0.f;
#pragma unroll
            for (int jh = 0; jh < 2; ++jh) {
                const int rc = r0 + 64 * jh + 4 * tx;
                const size_t o = (size_t)i * a.Rpad + rc;
                const float4 ph = *reinterpret_cast<const float4*>(a.phi + o);
                const float phv[4] = {ph.x, ph.y, ph.z, ph.w};
                float Lv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    Lv[j] = acc[4 * ih + ii][4 * jh + j];
                    if (hr != 0.f) Lv[j] += hr * fabsf(phv[j]);
                }
                if (MODE == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (rc + j < a.R) a.L[(size_t)(rc + j) * a.N + i] = Lv[j];
                } else {
                    const float4 pp = *reinterpret_cast<const float4*>(a.p + o);
                    const float ppv[4] = {pp.x, pp.y, pp.z, pp.w};
                    float pn[4], fn[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float phi2 = phv[j] * phv[j];
                        const float pw = pot_pow(phv[j], phi2, mhalf);
                        pn[j] = ppv[j] - fmaf(cf.x, pw, cf.y * Lv[j]);
                        fn[j] = fmaf(cf.z, pn[j], phv[j]);
                    }
                    *reinterpret_cast<float4*>(a.p + o) = make_float4(pn[0], pn[1], pn[2], pn[3]);
                    *reinterpret_cast<float4*>(a.phi_next + o) = make_float4(fn[0], fn[1], fn[2], fn[3]);
                    if (a.in_win) {
                        float4 wv = *reinterpret_cast<float4*>(a.w + o);
                        wv.x += fn[0];
                        wv.y += fn[1];
                        wv.z += fn[2];
                        wv.w += fn[3];
                        *reinterpret_cast<float4*>(a.w + o) = wv;
                    }
                }
            }
        }
}

// State set-up in the spin-major layout: phi(0), p(0) (SplitMix64 or the
// caller's [R][N] arrays), window sums 0; padding rows and replicas zero.
__global__ void k_simt_init(float* phi, float* phi_next, float* p, float* w, int N, int Npad,
                            int R, int Rpad, uint64_t seed, int init, const float* phi0,
                            const float* p0)
{
    const size_t total = (size_t)Npad * Rpad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / Rpad), r = (int)(idx % Rpad);
        float f = 0.f, q = 0.f;
        if (r < R && i < N) {
            if (init == HQA_INIT_GIVEN) {
                f = phi0[(size_t)r * N + i];
                q = p0[(size_t)r * N + i];
            } else {
                const uint64_t c = ((uint64_t)r << 32) | (uint64_t)i;
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
        phi[idx] = f;
        phi_next[idx] = 0.f;   // padding rows of the second buffer are never written later
        p[idx] = q;
        w[idx] = 0.f;
    }
}

// Final state in the [R][N] layout; flags a non-finite state.
__global__ void k_simt_out(const float* phi, const float* p, const float* w, int N, int Rpad,
                           int R, float inv_w, float* phi_out, float* p_out, float* phibar_out,
                           uint32_t* status)
{
    const size_t total = (size_t)R * N;
    bool bad = false;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / N), i = (int)(idx % N);
        const size_t o = (size_t)i * Rpad + r;
        const float f = phi[o], q = p[o];
        if (phi_out) phi_out[idx] = f;
        if (p_out) p_out[idx] = q;
        if (phibar_out) phibar_out[idx] = w[o] * inv_w;
        bad |= !(isfinite(f) && isfinite(q));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, HQA_DEV_NONFINITE);
}

__global__ void k_simt_transpose_in(const float* src, int R, int N, int Rpad, int Npad, float* dst)
{
    const size_t total = (size_t)Npad * Rpad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / Rpad), r = (int)(idx % Rpad);
        dst[idx] = (r < R && i < N) ? src[(size_t)r * N + i] : 0.f;
    }
}

int grid_1d(size_t n) { return (int)std::min<size_t>(8192, (n + 255) / 256); }

}  // namespace

// FP32 copy of J, [Npad][Npad] with Npad a multiple of 128, built on first use.
hqa_status hqa_simt_prepare(hqa_ctx* ctx)
{
    if (ctx->d_Jf32) return HQA_OK;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    const int N = ctx->N;
    const int Npad = (N + TM - 1) / TM * TM;
    std::vector<float> jf((size_t)Npad * Npad, 0.f);
    for (int i = 0; i < N; ++i)
        for (int64_t k = ctx->row_ptr[i]; k < ctx->row_ptr[i + 1]; ++k)
            jf[(size_t)i * Npad + ctx->col[k]] = ctx->val[k];
    void* d = nullptr;
    HQA_CUDA_TRY(cudaMalloc(&d, jf.size() * sizeof(float)));
    if (cudaMemcpy(d, jf.data(), jf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        (void)cudaGetLastError();
        return HQA_ERR_CUDA;
    }
    ctx->d_Jf32 = static_cast<float*>(d);
    ctx->Npad32 = Npad;
    ++ctx->generation;
    return HQA_OK;
}

bool hqa_simt_possible(const hqa_ctx* ctx)
{
    return !ctx->is_batch && ctx->dense_input;
}


hqa_status hqa_simt_field(hqa_ctx* ctx, int32_t R, const float* phi, float* L, cudaStream_t st)
{
    hqa_status s = hqa_simt_prepare(ctx);
    if (s != HQA_OK) return s;
    const int Npad = ctx->Npad32;
    const int Rpad = (R + TN - 1) / TN * TN;
    const size_t n = (size_t)Npad * Rpad;
    s = hqa_reserve(ctx, &ctx->d_ws, &ctx->ws_cap, n * sizeof(float));
    if (s != HQA_OK) return s;
    float* phit = static_cast<float*>(ctx->d_ws);
    k_simt_transpose_in<<<grid_1d(n), 256, 0, st>>>(phi, R, ctx->N, Rpad, Npad, phit);
    SimtArgs a{};
    a.J = ctx->d_Jf32;
    a.phi = phit;
    a.L = L;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.N = ctx->N;
    a.Npad = Npad;
    a.Rpad = Rpad;
    a.R = R;
    a.M = 6;
    k_dense_simt<0><<<dim3(Rpad / TN, Npad / TM), kThreads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}

hqa_status hqa_simt_launch_md(hqa_ctx* ctx, const StepCoef* d_sched, int64_t S, int32_t W,
                              int32_t R, uint64_t seed, int init, const float* phi0,
                              const float* p0, int M, float* phi_out, float* p_out,
                              float* phibar_out, cudaStream_t st)
{
    hqa_status s = hqa_simt_prepare(ctx);
    if (s != HQA_OK) return s;
    const int Npad = ctx->Npad32;
    const int Rpad = (R + TN - 1) / TN * TN;
    const size_t n = (size_t)Npad * Rpad;
    // phi (two step buffers), p, window sums
    s = hqa_reserve(ctx, &ctx->d_state, &ctx->state_cap, 4 * n * sizeof(float));
    if (s != HQA_OK) return s;
    float* base = static_cast<float*>(ctx->d_state);
    float* phib[2] = {base, base + n};
    float* p = base + 2 * n;
    float* w = base + 3 * n;
    k_simt_init<<<grid_1d(n), 256, 0, st>>>(phib[0], phib[1], p, w, ctx->N, Npad, R, Rpad, seed,
                                            init, phi0, p0);
    SimtArgs a{};
    a.J = ctx->d_Jf32;
    a.p = p;
    a.w = w;
    a.h = ctx->has_h ? ctx->d_h : nullptr;
    a.sched = d_sched;
    a.N = ctx->N;
    a.Npad = Npad;
    a.Rpad = Rpad;
    a.R = R;
    a.M = M;
    const dim3 grid(Rpad / TN, Npad / TM);
    const int64_t win0 = S - (int64_t)W;
    for (int64_t m = 0; m < S; ++m) {
        a.phi = phib[m & 1];
        a.phi_next = phib[(m + 1) & 1];
        a.m = m;
        a.in_win = m >= win0 ? 1 : 0;
        k_dense_simt<1><<<grid, kThreads, 0, st>>>(a);
    }
    const int64_t nwin = S < W ? S : W;
    k_simt_out<<<grid_1d((size_t)R * ctx->N), 256, 0, st>>>(phib[S & 1], p, w, ctx->N, Rpad, R,
                                                            1.0f / (float)nwin, phi_out, p_out,
                                                            phibar_out, ctx->d_status);
    return cudaGetLastError() == cudaSuccess ? HQA_OK : HQA_ERR_CUDA;
}
