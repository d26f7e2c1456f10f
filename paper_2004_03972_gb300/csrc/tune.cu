// tune.cu -- the autotuner: times every launch shape hqa_run could use for a
// (context, replica count, precision) and records the fastest, which hqa_run
// then takes whenever its options leave kernel and replica blocking open.
//
// Candidates: the scalar sparse kernel at 1..32 replicas per block, the
// vectorised sparse kernel at the blockings that fill a 16-byte vector, the
// persistent batch kernels (list-streaming at 1..32 replicas per block, the
// low-degree one at 1, 2, 4 where every member allows it), and the dense
// GEMM kernels (dense contexts: tcgen05 for the 16-bit precisions, the FP32
// CUDA-core GEMM for FP32).  Each one
// runs a short probe anneal (probe_steps leapfrog steps, dt = 1/probe_steps,
// init PAPER) once untimed (plan build, caches) and then three times between
// CUDA events on the caller's stream; the figure kept is the mean time per
// step.  A candidate that the library rejects (shared memory, alignment of
// the blocking, precision) is listed with ms_per_step = -1.
#include <vector>

#include "hqa_internal.cuh"

namespace {

struct Cand {
    int kernel;
    int rb;
};

std::vector<Cand> candidates(const hqa_ctx* ctx, int prec)
{
    std::vector<Cand> c;
    const int rbs[6] = {1, 2, 4, 8, 16, 32};
    if (!ctx->is_batch && ctx->dense_tc && hqa_tc_precision(prec)) {
        c.push_back({HQA_KERNEL_DENSE, 0});
        return c;
    }
    // FP32 on a dense context: the CUDA-core GEMM, and the sparse kernels
    // when the couplings are all +-1
    if (prec == HQA_PREC_FP32 && hqa_simt_possible(ctx)) c.push_back({HQA_KERNEL_DENSE, 0});
    if (!ctx->unit || (prec != HQA_PREC_FP32 && prec != HQA_PREC_BF16)) return c;
    for (int rb : rbs) c.push_back({HQA_KERNEL_SCALAR, rb});
    if (ctx->is_batch && hqa_lowdeg_eligible(ctx))
        for (int rb : {1, 2, 4}) c.push_back({HQA_KERNEL_LOWDEG, rb});
    if (!ctx->is_batch) {
        const int V = prec == HQA_PREC_BF16 ? 8 : 4;
        for (int rb : rbs)
            if (rb >= V) c.push_back({HQA_KERNEL_VECTOR, rb});
        if (hqa_stream_supported(ctx, prec)) c.push_back({HQA_KERNEL_STREAM, 0});
    }
    return c;
}

}  // namespace

extern "C" hqa_status hqa_autotune(hqa_ctx* ctx, const hqa_schedule* sched, int32_t replicas,
                                   const hqa_run_opts* opts, int32_t probe_steps,
                                   hqa_run_opts* best, hqa_tune_entry* table, int32_t table_cap,
                                   int32_t* table_len, void* stream)
{
    if (!ctx || !sched || !best || replicas < 1 || probe_steps < 1 || probe_steps > 100000)
        return HQA_ERR_INVALID_ARG;
    if (table_cap < 0 || (table_cap > 0 && !table)) return HQA_ERR_INVALID_ARG;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    hqa_run_opts o;
    if (opts) o = *opts;
    else hqa_run_opts_default(&o);
    if (o.precision < HQA_PREC_FP32 || o.precision > HQA_PREC_FP16X2) return HQA_ERR_INVALID_ARG;
    o.init = HQA_INIT_PAPER;
    o.phi0 = nullptr;
    o.p0 = nullptr;
    o.start_step = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // spin-indexed outputs: [R][N], or the members' [R][N_k] blocks of a batch
    const size_t spins = ctx->is_batch ? (size_t)ctx->total_spins : (size_t)ctx->N;
    const size_t RN = (size_t)replicas * spins;
    hqa_status s = hqa_reserve(ctx, &ctx->d_tune, &ctx->tune_cap, 2 * RN * sizeof(float));
    if (s != HQA_OK) return s;
    hqa_result res{};
    res.phi = static_cast<float*>(ctx->d_tune);
    res.p = res.phi + RN;
    const std::vector<Cand> cands = candidates(ctx, o.precision);
    cudaEvent_t e0, e1;
    HQA_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        (void)cudaGetLastError();
        return HQA_ERR_CUDA;
    }
    const double dt = 1.0 / (double)probe_steps;
    const int reps = 3;
    int best_i = -1;
    double best_ms = 0.0;
    std::vector<double> ms(cands.size(), -1.0);
    hqa_status fail = HQA_OK;
    // the tuned table must not steer the probes themselves
    auto saved = ctx->tuned.find({replicas, o.precision});
    const bool had = saved != ctx->tuned.end();
    const std::pair<int, int> old = had ? saved->second : std::pair<int, int>{0, 0};
    ctx->tuned.erase({replicas, o.precision});
    for (size_t i = 0; i < cands.size() && fail == HQA_OK; ++i) {
        hqa_run_opts c = o;
        c.kernel = cands[i].kernel;
        c.replicas_per_block = cands[i].rb;
        s = hqa_run(ctx, sched, dt, probe_steps, replicas, 0, &c, &res, stream);
        if (s == HQA_ERR_CUDA || s == HQA_ERR_OOM) fail = s;
        if (s != HQA_OK) continue;
        if (cudaEventRecord(e0, st) != cudaSuccess) fail = HQA_ERR_CUDA;
        for (int r = 0; r < reps && fail == HQA_OK; ++r) {
            s = hqa_run(ctx, sched, dt, probe_steps, replicas, 0, &c, &res, stream);
            if (s != HQA_OK) fail = s;
        }
        if (fail != HQA_OK) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            fail = HQA_ERR_CUDA;
            break;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            fail = HQA_ERR_CUDA;
            break;
        }
        ms[i] = (double)t / (double)(reps * (int64_t)probe_steps);
        if (best_i < 0 || ms[i] < best_ms) {
            best_i = (int)i;
            best_ms = ms[i];
        }
    }
    (void)cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (fail == HQA_OK) {
        // a probe that went non-finite or timed out does not count
        const hqa_status latched = hqa_sync(ctx, stream);
        if (latched != HQA_OK) fail = latched;
    }
    if (fail != HQA_OK || best_i < 0) {
        if (had) ctx->tuned[{replicas, o.precision}] = old;
        return fail != HQA_OK ? fail : HQA_ERR_UNSUPPORTED;
    }
    ctx->tuned[{replicas, o.precision}] = {cands[best_i].kernel, cands[best_i].rb};
    *best = o;
    best->kernel = cands[best_i].kernel;
    best->replicas_per_block = cands[best_i].rb;
    for (int i = 0; i < (int)cands.size() && i < table_cap; ++i) {
        table[i].kernel = cands[i].kernel;
        table[i].replicas_per_block = cands[i].rb;
        table[i].ms_per_step = ms[i];
    }
    if (table_len) *table_len = (int32_t)cands.size();
    return HQA_OK;
}
