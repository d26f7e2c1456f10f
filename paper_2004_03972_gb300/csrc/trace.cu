// trace.cu -- strided snapshots of the time-averaged flux along one anneal,
// the data behind the frozen / ambivalent separation as tau grows (Results,
// "Sorting frozen and ambivalent variables", Fig. 4): the trajectory runs as
// consecutive resumed segments of `stride` steps (bitwise the same trajectory
// as one run), and after segment t the window mean of its last
// min(W, segment length) steps is written to snapshot t.
#include "hqa_internal.cuh"

extern "C" hqa_status hqa_run_trace(hqa_ctx* ctx, const hqa_schedule* sched, double dt,
                                    int64_t steps, int64_t stride, int32_t replicas,
                                    uint64_t seed, const hqa_run_opts* opts, float* phibar_trace,
                                    float* phi, float* p, void* stream)
{
    if (!ctx || ctx->is_batch || !sched || !phibar_trace || !phi || !p || replicas < 1)
        return HQA_ERR_INVALID_ARG;
    if (steps < 1 || stride < 1) return HQA_ERR_INVALID_ARG;
    hqa_run_opts o;
    if (opts) o = *opts;
    else hqa_run_opts_default(&o);
    if (o.start_step != 0) return HQA_ERR_INVALID_ARG;
    hqa_capture_touch(ctx);
    const size_t RN = (size_t)replicas * ctx->N;
    int64_t m0 = 0;
    for (int64_t t = 0; m0 < steps; ++t) {
        const int64_t len = std::min(stride, steps - m0);
        hqa_run_opts so = o;
        if (t > 0) {
            so.init = HQA_INIT_GIVEN;
            so.phi0 = phi;
            so.p0 = p;
            so.start_step = m0;
        }
        hqa_result res{};
        res.phi = phi;
        res.p = p;
        res.phibar = phibar_trace + (size_t)t * RN;
        hqa_status s = hqa_run(ctx, sched, dt, len, replicas, seed, &so, &res, stream);
        if (s != HQA_OK) return s;
        m0 += len;
    }
    return HQA_OK;
}
