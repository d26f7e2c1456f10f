// api.cu -- the C ABI (include/hqa.h): argument checks, context set-up, the
// schedule table and the stream-ordered sequence of kernels behind hqa_run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "hqa_internal.cuh"

// Schedules (Methods, "Leapfrog algorithm"; Results, Eq. (3)-(4)):
//   alpha(tau) = alpha_f (tau + rho1 (1 - tau) + rho2 tau (tau - 1)),
//   beta(tau)  = beta_f (tau + kappa1 (1 - tau) + kappa2 tau (tau - 1)),
// or alpha(tau) = gamma0 (1 - tau) for the linear transverse-field schedule.
double hqa_sched_alpha(const hqa_schedule* s, double tau)
{
    if (s->kind == HQA_SCHED_LINEAR_GAMMA) return s->gamma0 * (1.0 - tau);
    return s->alpha_f * (tau + s->rho1 * (1.0 - tau) + s->rho2 * tau * (tau - 1.0));
}

double hqa_sched_beta(const hqa_schedule* s, double tau)
{
    return s->beta_f * (tau + s->kappa1 * (1.0 - tau) + s->kappa2 * tau * (tau - 1.0));
}

namespace {
thread_local bool t_capturing = false;
thread_local hqa_status t_capture_status = HQA_OK;
}  // namespace

bool hqa_capturing() { return t_capturing; }

hqa_status hqa_capture_note(hqa_status s)
{
    if (t_capturing && s != HQA_OK && t_capture_status == HQA_OK) t_capture_status = s;
    return s;
}

cudaError_t hqa_smem_attr(const void* kernel, size_t smem)
{
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(kernel);
    if (it != done.end() && it->second >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done[kernel] = smem;
    return e;
}

namespace {
// live contexts, so that a graph can tell a destroyed context from a live one
std::mutex g_live_mu;
std::map<const hqa_ctx*, uint64_t> g_live;   // context -> unique id (no reuse)
uint64_t g_next_uid = 1;
thread_local std::vector<hqa_ctx*> t_touched;
}  // namespace

void hqa_capture_touch(hqa_ctx* ctx)
{
    if (t_capturing && ctx) t_touched.push_back(ctx);
}

hqa_status hqa_reserve(hqa_ctx* ctx, void** p, size_t* cap, size_t bytes)
{
    if (bytes <= *cap && *p) return HQA_OK;
    if (t_capturing) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    ++ctx->generation;
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? HQA_ERR_OOM : HQA_ERR_CUDA;
    }
    *cap = want;
    return HQA_OK;
}

namespace {

void free_ctx_device(hqa_ctx* c)
{
    for (auto& kv : c->plans) {
        cudaFree(kv.second.d_entries);
        cudaFree(kv.second.d_tuples);
        cudaFree(kv.second.d_tuple_rows);
        if (kv.second.d_warp_off) cudaFree(kv.second.d_warp_off);
        if (kv.second.d_slot_of_row) cudaFree(kv.second.d_slot_of_row);
        if (kv.second.d_tuple_list) cudaFree(kv.second.d_tuple_list);
    }
    c->plans.clear();
    void* ptrs[] = {c->d_row_ptr, c->d_col,   c->d_val,    c->d_val_i8, c->d_h,
                    c->d_h_i32,   c->d_sched, c->d_ws,     c->d_state,  c->d_sub,
                    c->d_status,  c->d_Jbf,   c->d_binst,  c->d_bwork, c->d_feat,
                    c->d_tune,    c->d_diag,   c->d_Jcat,  c->d_efx,   c->d_ld,
                    c->d_ldwork,  c->d_Jh,     c->d_Jhcat, c->d_Jf32,  c->d_ebits};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// Builds a context from a validated symmetric CSR without diagonal or zero entries.
hqa_status finish_create(hqa_ctx* c, hqa_ctx** out)
{
    HQA_CUDA_TRY(cudaGetDevice(&c->device));
    HQA_CUDA_TRY(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    int optin = 0;
    HQA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    c->smem_optin = (size_t)optin;
    int l2 = 0;
    HQA_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device));
    c->l2_bytes = (size_t)l2;
    const int N = c->N;
    c->nnz = (int64_t)c->col.size();
    if (c->nnz >= (int64_t)1 << 31) return HQA_ERR_TOO_LARGE;
    // coupling classes
    bool integer = true, unit = true;
    int64_t sum = 0;
    for (float v : c->val) {
        if (v != std::nearbyint(v) || std::fabs(v) > 127.f) integer = false;
        if (std::fabs(v) != 1.f) unit = false;
        if (integer) sum += (int64_t)v;
    }
    c->has_h = false;
    for (float v : c->h) {
        if (v != 0.f) c->has_h = true;
        if (v != std::nearbyint(v) || std::fabs(v) > 1048576.f) integer = false;
    }
    if (!c->has_h) c->h.clear();
    c->integer = integer;
    c->unit = unit;
    c->sum_J_all = integer ? sum : 0;

    std::vector<int32_t> rp32(N + 1);
    for (int i = 0; i <= N; ++i) rp32[i] = (int32_t)c->row_ptr[i];
    const size_t nz = std::max<size_t>(c->col.size(), 1);
    HQA_CUDA_TRY(cudaMalloc(&c->d_row_ptr, (N + 1) * sizeof(int32_t)));
    HQA_CUDA_TRY(cudaMalloc(&c->d_col, nz * sizeof(int32_t)));
    HQA_CUDA_TRY(cudaMalloc(&c->d_val, nz * sizeof(float)));
    HQA_CUDA_TRY(cudaMemcpy(c->d_row_ptr, rp32.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!c->col.empty()) {
        HQA_CUDA_TRY(cudaMemcpy(c->d_col, c->col.data(), c->col.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        HQA_CUDA_TRY(cudaMemcpy(c->d_val, c->val.data(), c->val.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (integer) {
        std::vector<int8_t> v8(nz, 0);
        for (size_t k = 0; k < c->val.size(); ++k) v8[k] = (int8_t)c->val[k];
        HQA_CUDA_TRY(cudaMalloc(&c->d_val_i8, nz));
        HQA_CUDA_TRY(cudaMemcpy(c->d_val_i8, v8.data(), nz, cudaMemcpyHostToDevice));
    }
    if (c->has_h) {
        HQA_CUDA_TRY(cudaMalloc(&c->d_h, N * sizeof(float)));
        HQA_CUDA_TRY(cudaMemcpy(c->d_h, c->h.data(), N * sizeof(float), cudaMemcpyHostToDevice));
        if (integer) {
            std::vector<int32_t> hi(N);
            for (int i = 0; i < N; ++i) hi[i] = (int32_t)c->h[i];
            HQA_CUDA_TRY(cudaMalloc(&c->d_h_i32, N * sizeof(int32_t)));
            HQA_CUDA_TRY(cudaMemcpy(c->d_h_i32, hi.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
    }
    HQA_CUDA_TRY(cudaMalloc(&c->d_status, sizeof(uint32_t)));
    HQA_CUDA_TRY(cudaMemset(c->d_status, 0, sizeof(uint32_t)));
    {
        std::lock_guard<std::mutex> lock(g_live_mu);
        c->uid = g_next_uid++;
        g_live[c] = c->uid;
    }
    *out = c;
    return HQA_OK;
}

hqa_status create_guarded(hqa_ctx* c, hqa_ctx** out)
{
    hqa_status s = finish_create(c, out);
    if (s != HQA_OK) {
        free_ctx_device(c);
        delete c;
        *out = nullptr;
    }
    return s;
}

bool misaligned(const void* p, size_t a) { return p && ((uintptr_t)p % a) != 0; }

bool finite_all(const float* p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

double sched_alpha(const hqa_schedule* s, double tau) { return hqa_sched_alpha(s, tau); }
double sched_beta(const hqa_schedule* s, double tau) { return hqa_sched_beta(s, tau); }

hqa_status check_schedule(const hqa_schedule* s, double dt, int64_t steps)
{
    if (!s) return HQA_ERR_INVALID_ARG;
    if (s->kind < HQA_SCHED_PAPER || s->kind > HQA_SCHED_TABLE) return HQA_ERR_INVALID_ARG;
    if (s->M < 2 || s->M > 12 || (s->M & 1)) return HQA_ERR_INVALID_ARG;
    if (!(s->hstep > 0.0) || !std::isfinite(s->hstep)) return HQA_ERR_INVALID_ARG;
    if (s->window < 1) return HQA_ERR_INVALID_ARG;
    if (!std::isfinite(dt) || steps < 1) return HQA_ERR_INVALID_ARG;
    if (s->kind == HQA_SCHED_TABLE && (!s->table_alpha || !s->table_beta)) return HQA_ERR_INVALID_ARG;
    return HQA_OK;
}

// Kick/drift coefficients per step (Methods, "Leapfrog algorithm"):
//   kA_j = c_j h alpha(j dt) M, kB_j = c_j h beta(j dt), dA_j = h alpha((j+1/2) dt),
// c_0 = 1/2 (initial half step), c_j = 1 after.  Computed in FP64, stored FP32.
hqa_status upload_schedule(hqa_ctx* c, const hqa_schedule* s, double dt, int64_t S, int64_t m0 = 0)
{
    std::vector<StepCoef> t((size_t)S);
    for (int64_t jj = 0; jj < S; ++jj) {
        const int64_t j = m0 + jj;   // absolute step index
        double a, b, ah;
        if (s->kind == HQA_SCHED_TABLE) {
            a = s->table_alpha[2 * j];
            ah = s->table_alpha[2 * j + 1];
            b = s->table_beta[j];
        } else {
            a = sched_alpha(s, (double)j * dt);
            ah = sched_alpha(s, ((double)j + 0.5) * dt);
            b = sched_beta(s, (double)j * dt);
        }
        if (!std::isfinite(a) || !std::isfinite(ah) || !std::isfinite(b)) return HQA_ERR_INVALID_ARG;
        const double cj = j == 0 ? 0.5 : 1.0;
        t[jj].kA = (float)(cj * s->hstep * a * (double)s->M);
        t[jj].kB = (float)(cj * s->hstep * b);
        t[jj].dA = (float)(s->hstep * ah);
        t[jj].pad = 0.f;
    }
    const size_t bytes = t.size() * sizeof(StepCoef);
    if (c->sched_host.size() == t.size() && c->d_sched &&
        std::memcmp(c->sched_host.data(), t.data(), bytes) == 0)
        return HQA_OK;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    if (bytes > c->sched_cap) {
        if (c->d_sched) cudaFree(c->d_sched);
        c->d_sched = nullptr;
        c->sched_cap = 0;
        HQA_CUDA_TRY(cudaMalloc(&c->d_sched, bytes));
        c->sched_cap = bytes;
    }
    ++c->generation;
    // synchronous copy: the device may still read the previous table
    HQA_CUDA_TRY(cudaDeviceSynchronize());
    HQA_CUDA_TRY(cudaMemcpy(c->d_sched, t.data(), bytes, cudaMemcpyHostToDevice));
    c->sched_host.swap(t);
    return HQA_OK;
}

// Operand precisions the sparse (CSR) kernels implement.
bool sparse_precision(int prec) { return prec == HQA_PREC_FP32 || prec == HQA_PREC_BF16; }

hqa_status check_opts(const hqa_run_opts& o)
{
    if (o.precision < HQA_PREC_FP32 || o.precision > HQA_PREC_FP16X2) return HQA_ERR_INVALID_ARG;
    const int rbq = o.replicas_per_block;
    if (rbq != 0 && rbq != 1 && rbq != 2 && rbq != 4 && rbq != 8 && rbq != 16 && rbq != 32)
        return HQA_ERR_INVALID_ARG;
    if (o.kernel < HQA_KERNEL_AUTO || o.kernel > HQA_KERNEL_STREAM) return HQA_ERR_INVALID_ARG;
    return HQA_OK;
}

// Replica blocking and kernel variant: the vectorised kernel when the
// blocking allows it and its shared-memory image fits, else the scalar one.
hqa_status choose_plan(hqa_ctx* ctx, int32_t R, const hqa_run_opts& opts, const SparsePlan** plan)
{
    if (opts.kernel == HQA_KERNEL_LOWDEG) return HQA_ERR_UNSUPPORTED;   // batch contexts only
    hqa_run_opts o = opts;
    if (o.kernel == HQA_KERNEL_AUTO && o.replicas_per_block == 0) {
        const auto it = ctx->tuned.find({R, o.precision});
        if (it != ctx->tuned.end()) {
            o.kernel = it->second.first;
            o.replicas_per_block = it->second.second;
        }
    }
    int RB = o.replicas_per_block;
    int rb_scalar = RB;   // the scalar kernel's blocking if the vectorised one is not used
    if (RB == 0) {
        RB = rb_scalar = hqa_sparse_pick_rb(ctx, R, o.precision);
        // the vectorised kernel needs a full 16-byte vector of replicas per lane
        const int V = o.precision == HQA_PREC_BF16 ? 8 : 4;
        if (o.kernel != HQA_KERNEL_SCALAR && RB < V && RB > 0 && R >= V) RB = V;
    }
    if (RB == 0) return HQA_ERR_TOO_LARGE;
    if (o.kernel != HQA_KERNEL_SCALAR && hqa_vec_supported(ctx, RB, o.precision)) {
        const SparsePlan* vp = nullptr;
        hqa_status s = hqa_vec_plan(ctx, RB, o.precision, &vp);
        if (s != HQA_OK) return s;
        if (hqa_vec_smem_bytes(ctx, RB, o.precision, vp->ent_bytes) <= ctx->smem_optin) {
            *plan = vp;
            return HQA_OK;
        }
    }
    if (o.kernel == HQA_KERNEL_VECTOR) return HQA_ERR_UNSUPPORTED;
    if (rb_scalar > 0) RB = rb_scalar;   // the vector width was only for the vectorised kernel
    if (hqa_sparse_smem_bytes(ctx, RB, o.precision) > ctx->smem_optin) return HQA_ERR_TOO_LARGE;
    return hqa_sparse_plan(ctx, RB, o.precision, plan);
}

// Which dense path a single-context run or field takes: 0 none (the sparse
// kernels), 1 the tcgen05 GEMM (16-bit precisions), 2 the FP32 CUDA-core GEMM.
// HQA_KERNEL_DENSE asks for the dense path; AUTO takes it for 16-bit
// precisions on a dense context, for FP32 only when the couplings are not all
// +-1 (the sparse kernels need them) or the autotuner chose it.
hqa_status pick_dense(hqa_ctx* ctx, int32_t R, const hqa_run_opts& o, int* which)
{
    const bool tc_prec = hqa_tc_precision(o.precision);
    bool want = o.kernel == HQA_KERNEL_DENSE;
    if (o.kernel == HQA_KERNEL_AUTO) {
        if (tc_prec) want = hqa_dense_md_possible(ctx, R);
        else if (o.precision == HQA_PREC_FP32 && hqa_simt_possible(ctx)) {
            const auto it = ctx->tuned.find({R, o.precision});
            want = !ctx->unit ||
                   (o.replicas_per_block == 0 && it != ctx->tuned.end() &&
                    it->second.first == HQA_KERNEL_DENSE);
        }
    }
    *which = 0;
    if (want) {
        if (tc_prec) {
            if (!ctx->dense_tc) return HQA_ERR_UNSUPPORTED;
            *which = 1;
        } else if (o.precision == HQA_PREC_FP32) {
            if (!hqa_simt_possible(ctx)) return HQA_ERR_UNSUPPORTED;
            *which = 2;
        } else {
            return HQA_ERR_UNSUPPORTED;
        }
        return HQA_OK;
    }
    if (!ctx->unit || !sparse_precision(o.precision)) return HQA_ERR_UNSUPPORTED;
    return HQA_OK;
}

// Sparse launch for a single context: the streaming kernel when asked for,
// when the autotuner chose it, or (AUTO) when no resident plan fits; else the
// resident plan (*plan).
hqa_status pick_sparse(hqa_ctx* ctx, int32_t R, const hqa_run_opts& o, const SparsePlan** plan,
                       bool* stream)
{
    *stream = false;
    *plan = nullptr;
    bool want = o.kernel == HQA_KERNEL_STREAM;
    if (o.kernel == HQA_KERNEL_AUTO && o.replicas_per_block == 0) {
        const auto it = ctx->tuned.find({R, o.precision});
        want = it != ctx->tuned.end() && it->second.first == HQA_KERNEL_STREAM;
    }
    if (!want) {
        hqa_status s = choose_plan(ctx, R, o, plan);
        if (s != HQA_ERR_TOO_LARGE || o.kernel != HQA_KERNEL_AUTO ||
            !hqa_stream_supported(ctx, o.precision))
            return s;
    }
    if (!hqa_stream_supported(ctx, o.precision)) return HQA_ERR_UNSUPPORTED;
    *plan = nullptr;
    *stream = true;
    return HQA_OK;
}

// Batch run: one persistent launch over (member, replica block) items, then
// batched readout and energy.  Kernel: the low-degree one when every member
// allows it (lists on chip), else the list-streaming one.  Replica blocking:
// the largest RB whose shared-memory image fits every member and that leaves
// at least two items per SM.
hqa_status run_batch(hqa_ctx* ctx, const hqa_schedule* sched, double dt, int64_t steps,
                     int32_t replicas, uint64_t seed, const hqa_run_opts* opts,
                     const hqa_result* out, void* stream)
{
    hqa_run_opts o;
    if (opts) o = *opts;
    else hqa_run_opts_default(&o);
    hqa_status s = check_opts(o);
    if (s != HQA_OK) return s;
    if (o.kernel == HQA_KERNEL_DENSE || o.kernel == HQA_KERNEL_VECTOR ||
        o.kernel == HQA_KERNEL_STREAM || !sparse_precision(o.precision))
        return HQA_ERR_UNSUPPORTED;
    // kernel and blocking: the caller's, else the autotuned pair, else the
    // low-degree kernel when every member allows it, else the list-streaming one
    int kern = o.kernel;
    int RB = o.replicas_per_block;
    if (kern == HQA_KERNEL_AUTO && RB == 0) {
        const auto it = ctx->tuned.find({replicas, o.precision});
        if (it != ctx->tuned.end()) {
            kern = it->second.first;
            RB = it->second.second;
        }
    }
    if (kern == HQA_KERNEL_AUTO) kern = hqa_lowdeg_eligible(ctx) ? HQA_KERNEL_LOWDEG : HQA_KERNEL_SCALAR;
    if (kern == HQA_KERNEL_LOWDEG) {
        if (!hqa_lowdeg_eligible(ctx)) return HQA_ERR_UNSUPPORTED;
        if (RB == 0) RB = hqa_lowdeg_pick_rb(ctx, replicas, o.precision);
        if (RB == 0) return HQA_ERR_TOO_LARGE;
    }
    if (o.init < HQA_INIT_PAPER || o.init > HQA_INIT_GIVEN) return HQA_ERR_INVALID_ARG;
    if (o.init == HQA_INIT_GIVEN && (!o.phi0 || !o.p0)) return HQA_ERR_INVALID_ARG;
    if (o.start_step < 0 || (o.start_step > 0 && o.init != HQA_INIT_GIVEN)) return HQA_ERR_INVALID_ARG;
    if (misaligned(out->phi, 4) || misaligned(out->p, 4) || misaligned(out->phibar, 4) ||
        misaligned(out->energy, 8) || misaligned(out->cut, 8) || misaligned(out->tally, 4) ||
        misaligned(o.phi0, 4) || misaligned(o.p0, 4))
        return HQA_ERR_INVALID_ARG;
    const bool want_readout = out->spins || out->frozen || out->tally || out->energy || out->cut;
    const bool want_energy = out->energy || out->cut;
    if (want_energy && !ctx->integer) return HQA_ERR_UNSUPPORTED;
    if (RB == 0) {
        const int cands[6] = {32, 16, 8, 4, 2, 1};
        for (int rb : cands) {
            bool fits = true;
            for (hqa_ctx* m : ctx->members)
                fits = fits && hqa_sparse_smem_bytes(m, rb, o.precision) <= ctx->smem_optin;
            const int64_t items = (int64_t)ctx->members.size() * ((replicas + rb - 1) / rb);
            if (fits && items >= 2 * (int64_t)ctx->sm_count) { RB = rb; break; }
            if (fits) RB = rb;  // remember the smallest fitting so far (more items)
        }
        if (RB == 0) return HQA_ERR_TOO_LARGE;
    }
    s = upload_schedule(ctx, sched, dt, steps, o.start_step);
    if (s != HQA_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t RN = (size_t)replicas * (size_t)ctx->total_spins;
    const bool tmp_phibar = want_readout && !out->phibar;
    const bool tmp_spins = want_energy && !out->spins;
    size_t need = (tmp_phibar ? RN * sizeof(float) : 0) + (tmp_spins ? RN : 0);
    if (need) {
        s = hqa_reserve(ctx, &ctx->d_ws, &ctx->ws_cap, need);
        if (s != HQA_OK) return s;
    }
    char* ws = static_cast<char*>(ctx->d_ws);
    float* phibar = out->phibar;
    if (tmp_phibar) {
        phibar = reinterpret_cast<float*>(ws);
        ws += RN * sizeof(float);
    }
    int8_t* spins = out->spins;
    if (tmp_spins) spins = reinterpret_cast<int8_t*>(ws);
    const float* phi0 = o.init == HQA_INIT_GIVEN ? o.phi0 : nullptr;
    const float* p0 = o.init == HQA_INIT_GIVEN ? o.p0 : nullptr;
    if (kern == HQA_KERNEL_LOWDEG)
        s = hqa_lowdeg_launch_md(ctx, RB, o.precision, ctx->d_sched, steps, sched->window, replicas,
                                 seed, o.init, phi0, p0, sched->M, out->phi, out->p, phibar, st);
    else
        s = hqa_batch_launch_md(ctx, RB, o.precision, ctx->d_sched, steps, sched->window, replicas,
                                seed, o.init, phi0, p0, sched->M, out->phi, out->p, phibar, st);
    if (s != HQA_OK) return s;
    if (want_readout) {
        s = hqa_launch_readout_batch(ctx, replicas, phibar, sched->n_ambivalent, spins, out->frozen,
                                     out->tally, st);
        if (s != HQA_OK) return s;
    }
    if (want_energy) return hqa_launch_energy_batch(ctx, replicas, spins, out->energy, out->cut, st);
    return HQA_OK;
}

}  // namespace

extern "C" {

void hqa_schedule_default(hqa_schedule* s)
{
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
    s->kind = HQA_SCHED_PAPER;
    s->alpha_f = 0.008;
    s->rho1 = 4.0;
    s->rho2 = 3.0;
    s->beta_f = 0.12;
    s->kappa1 = 0.05;
    s->kappa2 = 1.0;
    s->gamma0 = 0.032;
    s->M = 6;
    s->hstep = 1.0;
    s->window = 100;
    s->n_ambivalent = 0;
}

void hqa_run_opts_default(hqa_run_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = HQA_PREC_FP32;
    o->init = HQA_INIT_PAPER;
}

hqa_status hqa_create_csr(int32_t N, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                          const float* val, const float* h, uint32_t flags, hqa_ctx** out)
{
    if (!out) return HQA_ERR_INVALID_ARG;
    *out = nullptr;
    if (N < 1 || N > 65536 || nnz < 0 || !row_ptr || flags != 0) return HQA_ERR_INVALID_ARG;
    if (nnz > 0 && (!col || !val)) return HQA_ERR_INVALID_ARG;
    if (row_ptr[0] != 0 || row_ptr[N] != nnz) return HQA_ERR_INVALID_ARG;
    for (int i = 0; i < N; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return HQA_ERR_INVALID_ARG;
    for (int64_t k = 0; k < nnz; ++k)
        if (col[k] < 0 || col[k] >= N) return HQA_ERR_INVALID_ARG;
    if (nnz > 0 && !finite_all(val, (size_t)nnz)) return HQA_ERR_NONFINITE_INPUT;
    if (h && !finite_all(h, (size_t)N)) return HQA_ERR_NONFINITE_INPUT;

    hqa_ctx* c = new (std::nothrow) hqa_ctx();
    if (!c) return HQA_ERR_OOM;
    c->N = N;
    // sorted rows, diagonal and explicit zeros dropped
    c->row_ptr.assign(N + 1, 0);
    std::vector<std::pair<int32_t, float>> rowbuf;
    for (int i = 0; i < N; ++i) {
        rowbuf.clear();
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (col[k] != i && val[k] != 0.f) rowbuf.emplace_back(col[k], val[k]);
        std::sort(rowbuf.begin(), rowbuf.end(),
                  [](const std::pair<int32_t, float>& a, const std::pair<int32_t, float>& b) {
                      return a.first < b.first;
                  });
        for (size_t k = 1; k < rowbuf.size(); ++k)
            if (rowbuf[k].first == rowbuf[k - 1].first) {
                delete c;
                return HQA_ERR_INVALID_ARG;  // duplicate entry
            }
        for (auto& e : rowbuf) {
            c->col.push_back(e.first);
            c->val.push_back(e.second);
        }
        c->row_ptr[i + 1] = (int64_t)c->col.size();
    }
    // symmetry: (i, j, v) present iff (j, i, v) present
    for (int i = 0; i < N; ++i) {
        for (int64_t k = c->row_ptr[i]; k < c->row_ptr[i + 1]; ++k) {
            const int j = c->col[k];
            auto b = c->col.begin() + c->row_ptr[j], e = c->col.begin() + c->row_ptr[j + 1];
            auto it = std::lower_bound(b, e, i);
            if (it == e || *it != i || c->val[it - c->col.begin()] != c->val[k]) {
                delete c;
                return HQA_ERR_ASYMMETRIC;
            }
        }
    }
    if (h) c->h.assign(h, h + N);
    return create_guarded(c, out);
}

hqa_status hqa_create_dense(int32_t N, const float* J, const float* h, uint32_t flags,
                            hqa_ctx** out)
{
    if (!out) return HQA_ERR_INVALID_ARG;
    *out = nullptr;
    if (N < 1 || N > 65536 || !J) return HQA_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)(HQA_J_BF16 | HQA_J_FP16 | HQA_J_FP32 | HQA_J_FP8))
        return HQA_ERR_INVALID_ARG;
    if (flags & HQA_J_FP8) return HQA_ERR_UNSUPPORTED;
    const size_t NN = (size_t)N * N;
    if (!finite_all(J, NN)) return HQA_ERR_NONFINITE_INPUT;
    if (h && !finite_all(h, (size_t)N)) return HQA_ERR_NONFINITE_INPUT;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j)
            if (J[(size_t)i * N + j] != J[(size_t)j * N + i]) return HQA_ERR_ASYMMETRIC;
    hqa_ctx* c = new (std::nothrow) hqa_ctx();
    if (!c) return HQA_ERR_OOM;
    c->N = N;
    c->dense_input = true;
    c->row_ptr.assign(N + 1, 0);
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < N; ++j) {
            const float v = J[(size_t)i * N + j];
            if (j != i && v != 0.f) {
                c->col.push_back(j);
                c->val.push_back(v);
            }
        }
        c->row_ptr[i + 1] = (int64_t)c->col.size();
    }
    if (h) c->h.assign(h, h + N);
    hqa_status s = create_guarded(c, out);
    if (s != HQA_OK) return s;
    s = hqa_dense_setup(c, J);
    if (s == HQA_OK && (flags & HQA_J_FP16)) s = hqa_dense_prepare(c, HQA_PREC_FP16);
    if (s == HQA_OK && (flags & HQA_J_FP32)) s = hqa_simt_prepare(c);
    if (s != HQA_OK) {
        hqa_destroy(c);
        *out = nullptr;
    }
    return s;
}

hqa_status hqa_create_batch(int32_t count, hqa_ctx* const* instances, hqa_ctx** out)
{
    if (!out) return HQA_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || !instances) return HQA_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k) {
        const hqa_ctx* m = instances[k];
        if (!m || m->is_batch) return HQA_ERR_INVALID_ARG;
        if (!m->unit) return HQA_ERR_UNSUPPORTED;
        if (m->device != instances[0]->device) return HQA_ERR_INVALID_ARG;
    }
    hqa_ctx* c = new (std::nothrow) hqa_ctx();
    if (!c) return HQA_ERR_OOM;
    c->is_batch = true;
    c->device = instances[0]->device;
    c->sm_count = instances[0]->sm_count;
    c->smem_optin = instances[0]->smem_optin;
    c->l2_bytes = instances[0]->l2_bytes;
    c->integer = true;
    c->unit = true;
    std::vector<BatchInst> tab(count);
    int64_t off = 0;
    for (int k = 0; k < count; ++k) {
        hqa_ctx* m = instances[k];
        c->members.push_back(m);
        c->member_off.push_back(off);
        c->N = std::max(c->N, m->N);
        c->nnz += m->nnz;
        c->integer = c->integer && m->integer;
        c->has_h = c->has_h || m->has_h;
        tab[k] = BatchInst{m->d_row_ptr, m->d_col, m->d_val_i8, m->has_h ? m->d_h_i32 : nullptr,
                           m->sum_J_all, off, m->N, 0};
        off += m->N;
    }
    c->total_spins = off;
    auto fail = [&](hqa_status s) {
        free_ctx_device(c);
        delete c;
        return s;
    };
    if (cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess) return fail(HQA_ERR_OOM);
    if (cudaMemset(c->d_status, 0, sizeof(uint32_t)) != cudaSuccess) return fail(HQA_ERR_CUDA);
    if (cudaMalloc(&c->d_binst, tab.size() * sizeof(BatchInst)) != cudaSuccess) return fail(HQA_ERR_OOM);
    if (cudaMemcpy(c->d_binst, tab.data(), tab.size() * sizeof(BatchInst), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return fail(HQA_ERR_CUDA);
    {
        std::lock_guard<std::mutex> lock(g_live_mu);
        c->uid = g_next_uid++;
        g_live[c] = c->uid;
    }
    *out = c;
    return HQA_OK;
}

hqa_status hqa_ctx_info(const hqa_ctx* ctx, int32_t* N, int64_t* nnz, int32_t* integer_couplings)
{
    if (!ctx) return HQA_ERR_INVALID_ARG;
    if (N) *N = ctx->N;
    if (nnz) *nnz = ctx->nnz;
    if (integer_couplings) *integer_couplings = ctx->integer ? 1 : 0;
    return HQA_OK;
}

static hqa_status run_impl(hqa_ctx* ctx, const hqa_schedule* sched, double dt, int64_t steps,
                   int32_t replicas, uint64_t seed, const hqa_run_opts* opts,
                   const hqa_result* out, void* stream)
{
    if (!ctx || !out || replicas < 1) return HQA_ERR_INVALID_ARG;
    hqa_status s = check_schedule(sched, dt, steps);
    if (s != HQA_OK) return s;
    if (ctx->is_batch) return run_batch(ctx, sched, dt, steps, replicas, seed, opts, out, stream);
    hqa_run_opts o;
    if (opts) o = *opts;
    else hqa_run_opts_default(&o);
    s = check_opts(o);
    if (s != HQA_OK) return s;
    if (o.init < HQA_INIT_PAPER || o.init > HQA_INIT_GIVEN) return HQA_ERR_INVALID_ARG;
    if (o.init == HQA_INIT_GIVEN && (!o.phi0 || !o.p0)) return HQA_ERR_INVALID_ARG;
    if (o.start_step < 0 || (o.start_step > 0 && o.init != HQA_INIT_GIVEN)) return HQA_ERR_INVALID_ARG;
    if (misaligned(out->phi, 4) || misaligned(out->p, 4) || misaligned(out->phibar, 4) ||
        misaligned(out->energy, 8) || misaligned(out->cut, 8) || misaligned(out->tally, 4) ||
        misaligned(o.phi0, 4) || misaligned(o.p0, 4))
        return HQA_ERR_INVALID_ARG;
    const bool want_readout = out->spins || out->frozen || out->tally || out->energy || out->cut;
    const bool want_energy = out->energy || out->cut;
    if (want_energy && !ctx->integer) return HQA_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (o.kernel == HQA_KERNEL_LOWDEG) return HQA_ERR_UNSUPPORTED;   // batch contexts only
    int dense = 0;   // 1: tcgen05 GEMM, 2: FP32 CUDA-core GEMM
    s = pick_dense(ctx, replicas, o, &dense);
    if (s != HQA_OK) return s;

    const SparsePlan* plan = nullptr;
    bool streaming = false;
    if (!dense) {
        s = pick_sparse(ctx, replicas, o, &plan, &streaming);
        if (s != HQA_OK) return s;
    }
    s = upload_schedule(ctx, sched, dt, steps, o.start_step);
    if (s != HQA_OK) return s;

    // temporaries for outputs the caller skipped but later stages need
    const size_t RN = (size_t)replicas * ctx->N;
    size_t need = 0;
    const bool tmp_phibar = want_readout && !out->phibar;
    const bool tmp_spins = want_energy && !out->spins;
    if (tmp_phibar) need += RN * sizeof(float);
    if (tmp_spins) need += RN;
    if (need) {
        s = hqa_reserve(ctx, &ctx->d_ws, &ctx->ws_cap, need);
        if (s != HQA_OK) return s;
    }
    char* ws = static_cast<char*>(ctx->d_ws);
    float* phibar = out->phibar;
    if (tmp_phibar) {
        phibar = reinterpret_cast<float*>(ws);
        ws += RN * sizeof(float);
    }
    int8_t* spins = out->spins;
    if (tmp_spins) spins = reinterpret_cast<int8_t*>(ws);

    if (dense == 1)
        s = hqa_dense_launch_md(ctx, ctx->d_sched, steps, sched->window, replicas, seed, o.init,
                                o.phi0, o.p0, sched->M, out->phi, out->p, phibar, o.precision, st);
    else if (dense == 2)
        s = hqa_simt_launch_md(ctx, ctx->d_sched, steps, sched->window, replicas, seed, o.init,
                               o.phi0, o.p0, sched->M, out->phi, out->p, phibar, st);
    else if (streaming)
        s = hqa_stream_launch_md(ctx, o.precision, ctx->d_sched, steps, sched->window, replicas,
                                 seed, o.init, o.phi0, o.p0, sched->M, out->phi, out->p, phibar,
                                 st);
    else if (plan->vec)
        s = hqa_vec_launch_md(ctx, plan, ctx->d_sched, steps, sched->window, replicas, seed, o.init,
                              o.phi0, o.p0, sched->M, out->phi, out->p, phibar, st);
    else
        s = hqa_sparse_launch_md(ctx, plan, ctx->d_sched, steps, sched->window, replicas, seed,
                                 o.init, o.phi0, o.p0, sched->M, out->phi, out->p, phibar, st);
    if (s != HQA_OK) return s;
    if (want_readout) {
        s = hqa_launch_readout(ctx, replicas, phibar, sched->n_ambivalent, spins, out->frozen,
                               out->tally, st);
        if (s != HQA_OK) return s;
    }
    if (want_energy) {
        s = hqa_launch_energy(ctx, replicas, spins, out->energy, out->cut, st);
        if (s != HQA_OK) return s;
    }
    return HQA_OK;
}

hqa_status hqa_run(hqa_ctx* ctx, const hqa_schedule* sched, double dt, int64_t steps,
                   int32_t replicas, uint64_t seed, const hqa_run_opts* opts,
                   const hqa_result* out, void* stream)
{
    hqa_capture_touch(ctx);
    return hqa_capture_note(run_impl(ctx, sched, dt, steps, replicas, seed, opts, out, stream));
}

static hqa_status local_field_impl(hqa_ctx* ctx, int32_t replicas, const float* phi, float* L,
                           const hqa_run_opts* opts, void* stream)
{
    if (ctx && ctx->is_batch) return HQA_ERR_UNSUPPORTED;
    if (!ctx || replicas < 1 || !phi || !L || misaligned(phi, 4) || misaligned(L, 4))
        return HQA_ERR_INVALID_ARG;
    hqa_run_opts o;
    if (opts) o = *opts;
    else hqa_run_opts_default(&o);
    hqa_status s = check_opts(o);
    if (s != HQA_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dense = 0;
    s = pick_dense(ctx, replicas, o, &dense);
    if (s != HQA_OK) return s;
    if (dense == 1) return hqa_dense_field(ctx, replicas, phi, L, o.precision, st);
    if (dense == 2) return hqa_simt_field(ctx, replicas, phi, L, st);
    const SparsePlan* plan = nullptr;
    bool streaming = false;
    s = pick_sparse(ctx, replicas, o, &plan, &streaming);
    if (s != HQA_OK) return s;
    if (streaming) return hqa_stream_field(ctx, o.precision, replicas, phi, L, st);
    if (plan->vec) return hqa_vec_launch_field(ctx, plan, replicas, phi, L, st);
    return hqa_sparse_launch_field(ctx, plan, replicas, phi, L, st);
}

hqa_status hqa_local_field(hqa_ctx* ctx, int32_t replicas, const float* phi, float* L,
                           const hqa_run_opts* opts, void* stream)
{
    hqa_capture_touch(ctx);
    return hqa_capture_note(local_field_impl(ctx, replicas, phi, L, opts, stream));
}

static hqa_status readout_impl(hqa_ctx* ctx, int32_t replicas, const float* phibar, int32_t n,
                       int8_t* spins, uint8_t* frozen, int32_t* tally, void* stream)
{
    if (!ctx || replicas < 1 || !phibar || (!spins && !frozen && !tally)) return HQA_ERR_INVALID_ARG;
    if (misaligned(phibar, 4) || misaligned(tally, 4)) return HQA_ERR_INVALID_ARG;
    if (ctx->is_batch)
        return hqa_launch_readout_batch(ctx, replicas, phibar, n, spins, frozen, tally,
                                        static_cast<cudaStream_t>(stream));
    return hqa_launch_readout(ctx, replicas, phibar, n, spins, frozen, tally,
                              static_cast<cudaStream_t>(stream));
}

hqa_status hqa_readout(hqa_ctx* ctx, int32_t replicas, const float* phibar, int32_t n,
                       int8_t* spins, uint8_t* frozen, int32_t* tally, void* stream)
{
    hqa_capture_touch(ctx);
    return hqa_capture_note(readout_impl(ctx, replicas, phibar, n, spins, frozen, tally, stream));
}

static hqa_status energy_impl(hqa_ctx* ctx, int32_t replicas, const int8_t* spins, int64_t* energy,
                      int64_t* cut, void* stream)
{
    if (!ctx || replicas < 1 || !spins || (!energy && !cut)) return HQA_ERR_INVALID_ARG;
    if (misaligned(energy, 8) || misaligned(cut, 8)) return HQA_ERR_INVALID_ARG;
    if (ctx->is_batch)
        return hqa_launch_energy_batch(ctx, replicas, spins, energy, cut,
                                       static_cast<cudaStream_t>(stream));
    return hqa_launch_energy(ctx, replicas, spins, energy, cut, static_cast<cudaStream_t>(stream));
}

hqa_status hqa_energy(hqa_ctx* ctx, int32_t replicas, const int8_t* spins, int64_t* energy,
                      int64_t* cut, void* stream)
{
    hqa_capture_touch(ctx);
    return hqa_capture_note(energy_impl(ctx, replicas, spins, energy, cut, stream));
}

static hqa_status solve_sub_impl(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                         const uint8_t* frozen, int32_t n, int8_t* out_spins,
                         int64_t* out_energy, void* stream)
{
    if (ctx && ctx->is_batch) return HQA_ERR_UNSUPPORTED;
    if (!ctx || replicas < 1 || !spins || !frozen || !out_spins) return HQA_ERR_INVALID_ARG;
    if (n < 0 || misaligned(out_energy, 8)) return HQA_ERR_INVALID_ARG;
    return hqa_launch_subsolve(ctx, replicas, spins, frozen, n, out_spins, out_energy,
                               static_cast<cudaStream_t>(stream));
}

hqa_status hqa_solve_sub(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                         const uint8_t* frozen, int32_t n, int8_t* out_spins,
                         int64_t* out_energy, void* stream)
{
    hqa_capture_touch(ctx);
    return hqa_capture_note(solve_sub_impl(ctx, replicas, spins, frozen, n, out_spins, out_energy, stream));
}

hqa_status hqa_plan_query(hqa_ctx* ctx, int32_t replicas, const hqa_run_opts* opts,
                          hqa_plan_info* out)
{
    if (ctx && ctx->is_batch) return HQA_ERR_UNSUPPORTED;
    if (!ctx || replicas < 1 || !out) return HQA_ERR_INVALID_ARG;
    hqa_run_opts o;
    if (opts) o = *opts;
    else hqa_run_opts_default(&o);
    hqa_status s = check_opts(o);
    if (s != HQA_OK) return s;
    int dense = 0;
    s = pick_dense(ctx, replicas, o, &dense);
    if (s != HQA_OK) return s;
    if (dense == 2) {
        out->kernel = HQA_KERNEL_DENSE;
        out->replicas_per_block = 128;
        out->blocks = ((replicas + 127) / 128) * ((ctx->N + 127) / 128);
        out->threads = 256;
        out->smem_bytes = 0;
        out->chunks = 1;
        out->pad_ratio = (double)out->blocks * 128 * 128 / ((double)ctx->N * replicas);
        out->conflict_ratio = 1.0;
        out->balance = 1.0;
        return HQA_OK;
    }
    if (dense == 1) {
        int nh = 0, grid = 0;
        const int C = hqa_dense_md_chunks(ctx, replicas, o.precision);
        const int Rc = (replicas + C - 1) / C;
        if (!hqa_dense_md_geometry(ctx, Rc, &nh, &grid)) return HQA_ERR_UNSUPPORTED;
        out->kernel = HQA_KERNEL_DENSE;
        out->replicas_per_block = 2 * nh;
        out->blocks = grid;
        out->threads = 448;         // TMA warp, MMA warp, 12 epilogue warps
        out->smem_bytes = 0;
        out->chunks = C;
        out->pad_ratio = (double)C * grid * 128 * 2 * nh / ((double)ctx->N * replicas);
        out->conflict_ratio = 1.0;
        out->balance = 1.0;
        return HQA_OK;
    }
    const SparsePlan* plan = nullptr;
    bool stream = false;
    s = pick_sparse(ctx, replicas, o, &plan, &stream);
    if (s != HQA_OK) return s;
    if (stream) {
        const int V = o.precision == HQA_PREC_BF16 ? 8 : 4;
        out->kernel = HQA_KERNEL_STREAM;
        out->replicas_per_block = V;
        out->blocks = 0;            // persistent: as many CTAs as are co-resident
        out->threads = 256;
        out->smem_bytes = 0;
        out->chunks = 1;
        out->pad_ratio = (double)((replicas + V - 1) / V * V) / replicas;
        out->conflict_ratio = 1.0;
        out->balance = 1.0;
        return HQA_OK;
    }
    out->kernel = plan->vec ? HQA_KERNEL_VECTOR : HQA_KERNEL_SCALAR;
    out->chunks = 1;
    out->replicas_per_block = plan->RB;
    out->blocks = (replicas + plan->RB - 1) / plan->RB;
    if (plan->vec) {
        out->threads = plan->NW * 32;
        out->smem_bytes = (int64_t)hqa_vec_smem_bytes(ctx, plan->RB, plan->prec, plan->ent_bytes);
    } else {
        out->threads = std::min(32, std::max(1, plan->T)) * 32;
        out->smem_bytes = (int64_t)hqa_sparse_smem_bytes(ctx, plan->RB, plan->prec);
    }
    out->pad_ratio = plan->pad_ratio;
    out->conflict_ratio = plan->conflict_ratio;
    out->balance = plan->vec ? plan->balance : 0.0;
    return HQA_OK;
}

hqa_status hqa_sync(hqa_ctx* ctx, void* stream)
{
    if (!ctx) return HQA_ERR_INVALID_ARG;
    if (hqa_capturing()) return hqa_capture_note(HQA_ERR_UNSUPPORTED);
    HQA_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    uint32_t bits = 0;
    HQA_CUDA_TRY(cudaMemcpy(&bits, ctx->d_status, sizeof(bits), cudaMemcpyDeviceToHost));
    if (bits) HQA_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(uint32_t)));
    if (bits & HQA_DEV_NONFINITE) return HQA_ERR_NONFINITE;
    if (bits & HQA_DEV_TIMEOUT) return HQA_ERR_TIMEOUT;
    if (bits & HQA_DEV_BAD_SUBPROBLEM) return HQA_ERR_INVALID_ARG;
    return HQA_OK;
}

const char* hqa_status_string(hqa_status s)
{
    switch (s) {
    case HQA_OK: return "ok";
    case HQA_ERR_INVALID_ARG: return "invalid argument";
    case HQA_ERR_ASYMMETRIC: return "coupling matrix is not symmetric";
    case HQA_ERR_NONFINITE_INPUT: return "non-finite coupling or field";
    case HQA_ERR_OOM: return "device out of memory";
    case HQA_ERR_CUDA: return "CUDA runtime error";
    case HQA_ERR_UNSUPPORTED: return "unsupported by this build";
    case HQA_ERR_NONFINITE: return "trajectory became non-finite";
    case HQA_ERR_TIMEOUT: return "device-side wait timed out";
    case HQA_ERR_TOO_LARGE: return "size beyond a documented limit";
    }
    return "unknown status";
}

hqa_status hqa_capture_begin(void* stream)
{
    // the legacy default stream cannot be captured
    if (!stream || t_capturing) return HQA_ERR_INVALID_ARG;
    HQA_CUDA_TRY(cudaStreamBeginCapture(static_cast<cudaStream_t>(stream),
                                        cudaStreamCaptureModeThreadLocal));
    t_capturing = true;
    t_capture_status = HQA_OK;
    t_touched.clear();
    return HQA_OK;
}

hqa_status hqa_capture_end(void* stream, hqa_graph** out)
{
    if (!stream || !out || !t_capturing) return HQA_ERR_INVALID_ARG;
    *out = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &g);
    t_capturing = false;
    const hqa_status first = t_capture_status;
    t_capture_status = HQA_OK;
    if (e != cudaSuccess || first != HQA_OK || !g) {
        (void)cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        t_touched.clear();
        return first != HQA_OK ? first : HQA_ERR_CUDA;
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaGraphDestroy(g);
        t_touched.clear();
        return HQA_ERR_CUDA;
    }
    hqa_graph* h = new (std::nothrow) hqa_graph;
    if (!h) {
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        return HQA_ERR_OOM;
    }
    h->graph = g;
    h->exec = x;
    for (hqa_ctx* c : t_touched) {
        bool seen = false;
        for (const auto& d : h->deps) seen = seen || d.ctx == c;
        if (!seen) h->deps.push_back({c, c->uid, c->generation});
    }
    t_touched.clear();
    *out = h;
    return HQA_OK;
}

hqa_status hqa_graph_launch(hqa_graph* g, void* stream)
{
    if (!g || t_capturing) return HQA_ERR_INVALID_ARG;
    {
        // every context the graph uses must be alive, with the buffers and tables
        // it had at capture (a reallocation would leave the graph a dangling pointer)
        std::lock_guard<std::mutex> lock(g_live_mu);
        for (const auto& d : g->deps) {
            const auto it = g_live.find(d.ctx);
            if (it == g_live.end() || it->second != d.uid || d.ctx->generation != d.generation)
                return HQA_ERR_INVALID_ARG;
        }
    }
    HQA_CUDA_TRY(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
    return HQA_OK;
}

void hqa_graph_destroy(hqa_graph* g)
{
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}

void hqa_destroy(hqa_ctx* ctx)
{
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> lock(g_live_mu);
        g_live.erase(ctx);
    }
    cudaDeviceSynchronize();
    free_ctx_device(ctx);
    delete ctx;
}

}  // extern "C"
