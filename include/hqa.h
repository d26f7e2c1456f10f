/*
 * hqa.h -- C ABI of the GB300 HQA-MD library (libhqa.so).
 *
 * HQA-MD is the hybrid quantum annealing scheme of arXiv:2004.03972: a
 * classical molecular dynamics of continuous flux variables phi_i with
 * momenta p_i, one per Ising spin, integrated by leapfrog under annealing
 * schedules alpha(tau), beta(tau); the time-averaged fluxes are read out as
 * spins, the |phibar| ranking splits frozen from ambivalent spins, and the
 * small problem on the ambivalent spins is solved exactly.
 *
 * Conventions
 *  - Every call returns hqa_status; nothing throws across the ABI.
 *  - Host pointers are only read during the call (the caller keeps them).
 *  - "device" pointers are CUDA global-memory pointers on the device that
 *    was current when the context was created; the caller owns them.
 *  - Work is enqueued on the caller's `stream` (a cudaStream_t, passed as
 *    void* so this header needs no CUDA include; NULL = legacy stream) and
 *    runs asynchronously.  Errors found on the device (non-finite state,
 *    bad sub-problem sizes) are latched in the context and reported by
 *    hqa_sync().
 *  - Arrays indexed by replica and spin use the layout [R][N] (row-major,
 *    replica-major): element (r, i) is at r * N + i.
 *  - Contexts are not thread-safe; use one context per host thread, or
 *    serialise calls.
 */
#ifndef HQA_H
#define HQA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HQA_OK = 0,
    HQA_ERR_INVALID_ARG = 1,     /* null pointer, bad size or flag */
    HQA_ERR_ASYMMETRIC = 2,      /* J_ij != J_ji */
    HQA_ERR_NONFINITE_INPUT = 3, /* NaN/Inf in J or h */
    HQA_ERR_OOM = 4,             /* device allocation failed */
    HQA_ERR_CUDA = 5,            /* a CUDA runtime call failed */
    HQA_ERR_UNSUPPORTED = 6,     /* valid request this build does not implement */
    HQA_ERR_NONFINITE = 7,       /* a trajectory became NaN/Inf on the device */
    HQA_ERR_TIMEOUT = 8,         /* a bounded device-side wait expired */
    HQA_ERR_TOO_LARGE = 9        /* size beyond a documented limit */
} hqa_status;

typedef struct hqa_ctx hqa_ctx;

/* Schedule kinds. */
enum {
    /* Methods, "Scheduling functions for MD":
     *   alpha(tau) = alpha_f (tau + rho1 (1 - tau) + rho2 tau (tau - 1))
     *   beta(tau)  = beta_f  (tau + kappa1 (1 - tau) + kappa2 tau (tau - 1)) */
    HQA_SCHED_PAPER = 0,
    /* alpha(tau) = gamma0 (1 - tau) (a linearly vanishing transverse-field
     * analogue; not in the paper), beta(tau) as in HQA_SCHED_PAPER. */
    HQA_SCHED_LINEAR_GAMMA = 1,
    /* caller tables: table_alpha[k] = alpha at tau = k dt / 2 (k = 0..2S),
     * table_beta[m] = beta at tau = m dt (m = 0..S). */
    HQA_SCHED_TABLE = 2
};

/* Annealing schedule and run constants (Methods; Results Eqs. (3)-(5)). */
typedef struct {
    int32_t kind;                 /* HQA_SCHED_* */
    double alpha_f, rho1, rho2;   /* paper: 0.008, 4, 3 */
    double beta_f, kappa1, kappa2;/* paper: 0.12, 0.05, 1 */
    double gamma0;                /* HQA_SCHED_LINEAR_GAMMA only; default 0.032 = alpha(0) */
    int32_t M;                    /* V(phi) = phi^M, even, 2..12; paper: 6 */
    double hstep;                 /* h = dtau / g multiplying each kick and drift; paper: 1 */
    int32_t window;               /* W: phibar averages phi^(m), m = S-W+1..S; paper: 100 */
    int32_t n_ambivalent;         /* n: the n smallest |phibar| are ambivalent */
    const double* table_alpha;    /* host, HQA_SCHED_TABLE only, 2*(start_step+steps)+1 values */
    const double* table_beta;     /* host, HQA_SCHED_TABLE only, start_step+steps+1 values */
} hqa_schedule;

/* Initial conditions. */
enum {
    HQA_INIT_PAPER = 0,       /* phi_i(0) = 0, p_i(0) = +-1 (Results, after Eq. (4)) */
    HQA_INIT_RANDOM_FLUX = 1, /* phi_i(0) uniform on [-1/8, 1/8), p_i(0) = +-1 */
    HQA_INIT_GIVEN = 2        /* phi0 / p0 supplied by the caller */
};

/* Arithmetic of the local-field operand.  phi and p stay FP32 in every case. */
enum {
    HQA_PREC_FP32 = 0,   /* phi operand FP32, FP32 accumulate (sparse kernels; dense
                            contexts with HQA_KERNEL_DENSE: an FP32 GEMM on the CUDA cores) */
    HQA_PREC_BF16 = 1,   /* phi operand rounded to BF16 (8 significant bits), FP32
                            accumulate; dense: J rounded to BF16 too (exact for +-1) */
    HQA_PREC_BF16X2 = 2, /* dense tensor-core path only: phi = hi + lo, both BF16 (about 16
                            significant bits), two K segments, FP32 accumulate */
    HQA_PREC_FP16 = 3,   /* dense tensor-core path only: phi * 2^6 and J * 2^10 rounded to
                            FP16 (11 significant bits; exact for +-1 J), FP32 accumulate,
                            scaled back by 2^-16 */
    HQA_PREC_FP16X2 = 4  /* dense tensor-core path only: phi * 2^6 = hi + lo, both FP16
                            (about 22 significant bits), and J split the same way when it
                            is not exact in FP16; two (exact J) or three K segments */
};

/* Sparse kernel variants (all compute the same sums, in different orders). */
enum {
    HQA_KERNEL_AUTO = 0,   /* vectorised when the blocking allows, else scalar */
    HQA_KERNEL_SCALAR = 1, /* one replica per lane, neighbour lists streamed from L1/L2 */
    HQA_KERNEL_VECTOR = 2, /* 16-byte gathers per lane, lists in shared memory; needs
                              replicas_per_block >= 4 (FP32) or >= 8 (BF16) */
    HQA_KERNEL_DENSE = 3,  /* dense contexts: the field as a GEMM of J and the replicas'
                              fluxes -- on the tcgen05 tensor cores for the 16-bit
                              precisions (BF16, BF16X2, FP16, FP16X2), on the CUDA cores
                              for FP32 */
    HQA_KERNEL_LOWDEG = 4, /* batch contexts whose members have at most 4 couplings per
                              spin and fewer than 2^15 spins: compact lists, operand and
                              state of a work item all in shared memory; replicas_per_block
                              1, 2 or 4.  AUTO picks it for such batches */
    HQA_KERNEL_STREAM = 5  /* single contexts with couplings in {-1, 0, +1}, FP32 or BF16:
                              the operand and state in global memory (L2-resident at the
                              sizes it serves), one persistent cooperative grid with a
                              bounded-wait barrier per step.  For instances whose operand
                              does not fit in one SM's shared memory; AUTO takes it when
                              the resident kernels cannot run (HQA_ERR_TOO_LARGE) or the
                              autotuner chose it */
};

typedef struct {
    int32_t precision;          /* HQA_PREC_*; default FP32 */
    int32_t init;               /* HQA_INIT_*; default PAPER */
    const float* phi0;          /* device [R][N] (a batch: its array layout); HQA_INIT_GIVEN only */
    const float* p0;            /* device [R][N] (a batch: its array layout); HQA_INIT_GIVEN only */
    int32_t replicas_per_block; /* 0 = chosen by the library; else 1,2,4,8,16,32 */
    int32_t kernel;             /* HQA_KERNEL_*; default AUTO */
    int64_t start_step;         /* resume: first step index m0 (default 0).  With m0 > 0 the
                                   run continues a trajectory: init must be HQA_INIT_GIVEN
                                   with phi0 = phi^(m0) and p0 = p^(m0 - 1/2) as returned by
                                   the previous call, every kick is a full kick and step j
                                   evaluates the schedule at tau = (m0 + j) dt.  Splitting a
                                   run this way reproduces phi and p bitwise; phibar
                                   averages the last W steps of this call. */
} hqa_run_opts;

/* Caller-owned device outputs of hqa_run ([R][N] unless noted).  Any
 * pointer may be NULL to skip that output, except that spins/frozen/tally
 * need the readout and energy/cut need spins internally (the library then
 * uses its own workspace). */
typedef struct {
    float* phi;      /* phi^(S) */
    float* p;        /* p^(S - 1/2) (leapfrog momenta are staggered) */
    float* phibar;   /* window mean of phi (Eq. (5)) */
    int8_t* spins;   /* s_i = sgn(phibar_i), sgn(0) = +1 */
    uint8_t* frozen; /* 1 = frozen, 0 = ambivalent */
    int64_t* energy; /* [R] H_Ising(s), Eq. (1); integer couplings only */
    int64_t* cut;    /* [R] C(s) = 1/2 sum_{i<j, J_ij != 0} J_ij (1 - s_i s_j); integer couplings, h = 0 */
    int32_t* tally;  /* [R][2] (frozen count, ambivalent count) */
} hqa_result;

/* Fills `s` with the paper's constants (Methods): alpha_f = 0.008, rho1 = 4,
 * rho2 = 3, beta_f = 0.12, kappa1 = 0.05, kappa2 = 1, M = 6, hstep = 1,
 * window = 100 (delta = 100 dtau, Results "Sorting ..."), n_ambivalent = 0,
 * gamma0 = 0.032, kind = HQA_SCHED_PAPER. */
void hqa_schedule_default(hqa_schedule* s);

/* Fills `o` with defaults: FP32, HQA_INIT_PAPER, library-chosen blocking. */
void hqa_run_opts_default(hqa_run_opts* o);

/* Storage of the coupling operands of a dense context (flags of
 * hqa_create_dense).  Each copy is also built on first use when absent; a
 * flag builds it at create instead (so that no later call allocates or
 * uploads, e.g. before a stream capture).  Couplings of +-1 are exact in
 * every format. */
enum {
    HQA_J_BF16 = 1u << 0, /* BF16 tensor-core operand (always built for the tcgen05 path) */
    HQA_J_FP16 = 1u << 1, /* FP16 tensor-core operand, J * 2^10 (HQA_PREC_FP16 / FP16X2) */
    HQA_J_FP32 = 1u << 2, /* FP32 operand of the CUDA-core dense GEMM (HQA_PREC_FP32) */
    HQA_J_FP8 = 1u << 3   /* FP8 E4M3: not provided (HQA_ERR_UNSUPPORTED).  The kind::f16
                             MMA needs both operands in the same 16-bit format, and an
                             FP8 MMA would need phi in FP8 (3 significant bits); widening
                             an FP8 tile in shared memory would cost more shared-memory
                             traffic than the L2-resident 16-bit J it replaces */
};

/* Creates a context from dense couplings (Results Eq. (1)).
 *   N      number of spins, 1..65536
 *   J      host, N*N row-major float; must be symmetric; the diagonal is
 *          ignored (all sums in Eqs. (1), (3) run over j != i)
 *   h      host, N floats, or NULL for h = 0
 *   flags  0 or an OR of HQA_J_BF16, HQA_J_FP16, HQA_J_FP32
 * The couplings are copied; `*out` owns device copies, among them the
 * tensor-core operand of J.  Precisions on a dense context (hqa_run with
 * HQA_KERNEL_DENSE, or AUTO with a 16-bit precision): BF16 / FP16 multiply J
 * and phi rounded to that format (J exact for +-1 couplings); BF16X2 /
 * FP16X2 split phi into hi + lo and, when J is not exact in the format
 * (real-valued couplings), J as well: J_hi phi_hi + J_lo phi_hi +
 * J_hi phi_lo, about 16 (BF16) or 22 (FP16) significant bits of each.  FP32
 * with HQA_KERNEL_DENSE is an FP32 GEMM on the CUDA cores (any real J); FP32
 * with the sparse kernels needs couplings in {-1, 0, +1}.
 * Errors: INVALID_ARG (N out of range, null J/out, unknown flag), ASYMMETRIC,
 * NONFINITE_INPUT, UNSUPPORTED (HQA_J_FP8), OOM, CUDA. */
hqa_status hqa_create_dense(int32_t N, const float* J, const float* h, uint32_t flags,
                            hqa_ctx** out);

/* Creates a context from CSR couplings (host arrays): the Ising problem of
 * Results Eq. (1) with sparse symmetric J, e.g. the weighted graphs of the
 * MAX-CUT mapping (Methods, "MAX-CUT and Ising spin-glass": J_ij = w_ij, h = 0).
 *   row_ptr  N+1 int64, row_ptr[0] = 0, non-decreasing, row_ptr[N] = nnz
 *   col      nnz int32 in [0, N); duplicates within a row are rejected
 *   val      nnz float
 *   h        N floats or NULL
 * The pattern and values must be symmetric (entry (i, j) present iff
 * (j, i) present, equal values).  Diagonal entries are dropped.
 *   flags  0: the sparse kernels store no coupling values for +-1 couplings
 *          (a coupling picks the +phi or -phi copy of the operand), so there
 *          is no storage format to choose.
 * Errors: as hqa_create_dense, plus INVALID_ARG for a malformed CSR or a
 * nonzero flags. */
hqa_status hqa_create_csr(int32_t N, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                          const float* val, const float* h, uint32_t flags, hqa_ctx** out);

/* Creates a batch context over `count` existing contexts (instances of
 * uneven size).  The paper runs ensembles of random instances, each its own
 * problem of Results Eq. (1) (Results, "HQA for MAX-CUT": 100 random K2000
 * instances; "HQA for Ising spin-glass"); a batch runs many such instances
 * in one launch, which the paper does not do.  The members
 * are not copied: they must outlive the batch and not be destroyed first.
 * hqa_run on a batch runs `replicas` replicas of every member in one
 * persistent launch (work items = member x replica block, longest first):
 * HQA_KERNEL_LOWDEG when every member has at most 4 couplings per spin,
 * else the list-streaming kernel (HQA_KERNEL_SCALAR).
 * Batch array layout: member k's [R][N_k] block starts at R * (N_0 + ... +
 * N_{k-1}); per-replica results (energy, cut, tally) are [count][R].  Member
 * k draws its momenta from the stream seed + (k + 1) * 0x632BE59BD9B4E019
 * (HQA_INIT_PAPER / RANDOM_FLUX) or takes phi0 / p0 in the same layout
 * (HQA_INIT_GIVEN, which also resumes a batch with start_step).
 * Members need couplings in {-1, 0, +1}; hqa_readout and hqa_energy accept a
 * batch with the same layout; other calls return HQA_ERR_UNSUPPORTED.
 * Errors: INVALID_ARG (count < 1, null or batch member), UNSUPPORTED, OOM, CUDA. */
hqa_status hqa_create_batch(int32_t count, hqa_ctx* const* instances, hqa_ctx** out);

/* Queries: number of spins, stored off-diagonal entries, and whether all
 * couplings and fields are integers (the int64 energy path). */
hqa_status hqa_ctx_info(const hqa_ctx* ctx, int32_t* N, int64_t* nnz, int32_t* integer_couplings);

/* Runs the HQA-MD leapfrog (Methods, "Leapfrog algorithm") for `steps`
 * steps on `replicas` independent replicas, then reads out spins, the
 * frozen/ambivalent split and the integer energy and cut.
 *   sched     schedule and constants (hqa_schedule_default for the paper's)
 *   dt        dtau: step m evaluates the schedule at tau = m dt; the paper
 *             uses dt = 1 / steps
 *   steps     S >= 1: S kicks and S drifts, producing phi^(S), p^(S-1/2)
 *   replicas  R >= 1
 *   seed      initial momenta p_i(0) = +-1 come from SplitMix64 (Steele,
 *             Lea, Flood 2014): z = mix64(seed + (c + 1) * 0x9E3779B97F4A7C15)
 *             with counter c = (r << 32) | i, p = -1 if bit 63 of z is set,
 *             else +1.  HQA_INIT_RANDOM_FLUX draws phi_i(0) from counter
 *             c' = 2^62 | c: phi = ((z >> 40) - 2^23) * 2^-26.
 *   opts      NULL for defaults
 *   out       caller-owned device buffers
 *   stream    cudaStream_t
 * Step j (0-based) of replica r:
 *   p   <- p - c_j h [ alpha(j dt) M phi^(M-1) + beta(j dt) (sum_k J_ik phi_k + 2 h_i |phi_i|) ]
 *   phi <- phi + h alpha((j + 1/2) dt) p
 * with c_0 = 1/2 (the initial half step) and c_j = 1 otherwise.
 * Errors: INVALID_ARG, TOO_LARGE (N x replicas-per-block exceeds on-chip
 * capacity), UNSUPPORTED, OOM, CUDA; NONFINITE is latched if a state
 * becomes non-finite. */
hqa_status hqa_run(hqa_ctx* ctx, const hqa_schedule* sched, double dt, int64_t steps,
                   int32_t replicas, uint64_t seed, const hqa_run_opts* opts,
                   const hqa_result* out, void* stream);

/* Local field of the paper's kick (Methods, "Leapfrog algorithm"):
 *   L_i = sum_{j != i} J_ij phi_j + 2 h_i |phi_i|
 * for R replicas.  phi, L: device [R][N] float.  The sum is evaluated by
 * the same device code hqa_run would use with the same `opts` (precision,
 * replicas_per_block, kernel; NULL = defaults; init fields are ignored). */
hqa_status hqa_local_field(hqa_ctx* ctx, int32_t replicas, const float* phi, float* L,
                           const hqa_run_opts* opts, void* stream);

/* Readout (Results, "Sorting frozen and ambivalent variables"; HQA
 * section): s_i = sgn(phibar_i), sgn(0) = +1; spins ordered by
 * (|phibar_i|, i) ascending, the first n are ambivalent (frozen = 0).
 * n is clamped to [0, N].  phibar: device [R][N] float; spins [R][N] int8;
 * frozen [R][N] uint8; tally [R][2] int32 (may be NULL). */
hqa_status hqa_readout(hqa_ctx* ctx, int32_t replicas, const float* phibar, int32_t n,
                       int8_t* spins, uint8_t* frozen, int32_t* tally, void* stream);

/* Integer Ising energy (Results Eq. (1)) and MAX-CUT value (Methods,
 * "MAX-CUT and Ising spin-glass") of R spin configurations, exact in int64.
 * spins: device [R][N] int8 (+-1); energy, cut: device [R] int64 (either
 * may be NULL; cut ignores h).  Requires integer couplings and fields
 * (UNSUPPORTED otherwise). */
hqa_status hqa_energy(hqa_ctx* ctx, int32_t replicas, const int8_t* spins, int64_t* energy,
                      int64_t* cut, void* stream);

/* Ising energy (Results Eq. (1)) for any real couplings and field:
 *   E = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i
 * with J, h as given at create (FP32).  J and h are rounded once onto a grid
 * 2^-s chosen per context (max_i (sum_j |J_ij| + 2|h_i|) 2^s <= 2^61; each
 * value moves by at most 2^-(s+1)); the sum on that grid is exact (64-bit row
 * sums, a 128-bit total) and rounded to double once.  So the same inputs give
 * the same bits under any schedule, and integer J, h give exactly the int64
 * energy.  spins: device [R][N] int8; energy: device [R] double, 8-byte
 * aligned.  Workspace owned by the context (INVALID_ARG for bad pointers,
 * TOO_LARGE beyond 2^21 replicas per call, UNSUPPORTED for batch contexts
 * or row sums of |J| beyond 2^61). */
hqa_status hqa_energy_f64(hqa_ctx* ctx, int32_t replicas, const int8_t* spins, double* energy,
                          void* stream);

/* Exact solution of the reduced Ising problem on the ambivalent spins (HQA
 * section, Eqs. (6)-(7)).  For each replica the frozen spins keep their
 * value; the ambivalent ones (frozen == 0), taken in ascending spin index
 * a_0 < a_1 < ..., are set to the minimiser over all 2^n assignments of
 *   H'(s) = sum_{a<b} J_ab s_a s_b + sum_a h_eff_a s_a,
 *   h_eff_a = h_a + sum_{k frozen} J_ak s_k,
 * with x = sum_k [s_{a_k} = -1] 2^k and ties going to the smallest x.
 *   spins      device [R][N] int8 (+-1)
 *   frozen     device [R][N] uint8
 *   n          upper bound on the ambivalent count of every replica, 0..30
 *   out_spins  device [R][N] int8: the assembled configuration
 *   out_energy device [R] int64: its full energy (Eq. (1)); may be NULL
 * Requires integer couplings in {-1, 0, +1} and integer h (UNSUPPORTED
 * otherwise); a replica with more than n ambivalent spins latches
 * INVALID_ARG.  Uses workspace owned by the context. */
hqa_status hqa_solve_sub(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                         const uint8_t* frozen, int32_t n, int8_t* out_spins,
                         int64_t* out_energy, void* stream);

/* Tabu search on the reduced problem (HQA section, Eqs. (6)-(7)) for
 * ambivalent sets too large to enumerate (up to 1024 spins; the paper's
 * HQA(TS1000) hands such sets to a tabu search).  Deterministic: with
 *   f_a = h_a + sum_{j != a} J_aj s_j and d_a = -2 s_a f_a,
 * iteration it = 1..iters flips, among ambivalent spins that are not tabu
 * (tabu until iteration it' < it) or would give a new best energy, the one
 * with the smallest (d_a, a) -- even uphill -- and makes it tabu until
 * it + tenure; the best assignment met (the input if none is lower) is
 * written to out_spins and its full energy (Eq. (1)) to out_energy (may be
 * NULL).  spins, frozen, out_spins: device [R][N]; out_energy device [R]
 * int64.  The ambivalent count of each replica must be <= n <= 1024 (else
 * the input is copied and hqa_sync reports INVALID_ARG).  Integer couplings
 * in {-1, 0, +1} and integer h (UNSUPPORTED otherwise); iters, tenure in
 * [0, 2^30].  Not a guarantee of the optimum: hqa_solve_sub is the exact
 * solver for n <= 30. */
hqa_status hqa_solve_sub_tabu(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                              const uint8_t* frozen, int32_t n, int32_t iters, int32_t tenure,
                              int8_t* out_spins, int64_t* out_energy, void* stream);

/* hqa_solve_sub without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot let the library call
 * cudaMalloc -- a process whose device memory is already reserved by
 * another allocator or arena, or a latency-sensitive caller that cannot
 * accept cudaMalloc's implicit device-wide synchronisation.  Same arguments
 * and results as hqa_solve_sub, and its errors checked in the same order;
 * after them come the two of this variant: replicas > 2048 returns
 * HQA_ERR_TOO_LARGE and a current device other than the context's returns
 * HQA_ERR_INVALID_ARG.  The caller still provides every input and output
 * buffer.  Every replica takes the scalar Gray-code walk: hqa_solve_sub's
 * faster packed 16-bit walk keeps per-thread minima whose size grows with the
 * enumeration and does not fit the fixed scratch.  The results are the same.
 * Scratch: a fixed array compiled into the library (about 1.1 MB, enough for
 * 2048 replicas), present on every GPU that loads the library until the
 * process exits.
 * The first call on a device looks up that array's device address (once per
 * device, with the context's device current); make that first call before
 * any stream capture.  The current device must be the context's device
 * (HQA_ERR_INVALID_ARG otherwise).
 * Every call shares the one array and leaves its contents behind; each call
 * rewrites what it reads before reading it.  Calls whose work overlaps on
 * the GPU (for example on two streams) race: serialise them. */
hqa_status hqa_solve_sub_noalloc(hqa_ctx* ctx, int32_t replicas, const int8_t* spins,
                                 const uint8_t* frozen, int32_t n, int8_t* out_spins,
                                 int64_t* out_energy, void* stream);

/* Launch plan hqa_run / hqa_local_field would use for `replicas` replicas
 * with `opts` (NULL = defaults); builds and caches it if needed.  The
 * modelled figures describe the neighbour-list layout: stored positions per
 * coupling entry (padding), shared-memory wavefronts per conflict-free
 * wavefront (bank conflicts), and mean/max warp load (balance). */
typedef struct {
    int32_t kernel;              /* HQA_KERNEL_SCALAR, _VECTOR or _DENSE */
    int32_t replicas_per_block;
    int32_t blocks;              /* CTAs per launch */
    int32_t threads;             /* threads per CTA */
    int64_t smem_bytes;          /* dynamic shared memory per CTA */
    double pad_ratio;
    double conflict_ratio;
    double balance;
    int32_t chunks;              /* sequential launches over replica chunks (dense: each
                                    chunk's per-step data fits in L2), else 1 */
} hqa_plan_info;

hqa_status hqa_plan_query(hqa_ctx* ctx, int32_t replicas, const hqa_run_opts* opts,
                          hqa_plan_info* out);

/* ---------------------------------------------------------------------
 * Surrogate gate (an addition to the method: the paper has no learned
 * component).  A per-spin MLP, 6 inputs -> 64 ReLU -> 64 ReLU -> 2 logits,
 * predicts from features of the first part of a trajectory whether a spin
 * ends frozen (logit 0) and whether it ends at s = +1 (logit 1).  Trained
 * with the mean binary cross-entropy of the two sigmoid outputs.
 * Parameter vector (HQA_MLP_PARAMS FP32 values, in this order):
 *   W1[64][6], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
 * precision: HQA_PREC_FP32, or HQA_PREC_BF16 (weights, inputs and hidden
 * activations rounded to BF16, FP32 accumulation).
 * --------------------------------------------------------------------- */
enum { HQA_MLP_IN = 6, HQA_MLP_HIDDEN = 64, HQA_MLP_OUT = 2, HQA_MLP_PARAMS = 4738 };

typedef struct hqa_mlp hqa_mlp;

/* Creates a network on the current device from host parameters (copied);
 * AdamW moments start at zero. */
hqa_status hqa_mlp_create(const float* params, hqa_mlp** out);
/* Copies the current FP32 master parameters to host memory. */
hqa_status hqa_mlp_params(const hqa_mlp* mlp, float* params);
/* logits [n][2] for inputs x [n][6] (device arrays). */
hqa_status hqa_mlp_forward(hqa_mlp* mlp, int64_t n, const float* x, float* logits,
                           int32_t precision, void* stream);
/* Gradient of the mean loss over n samples x [n][6], labels y [n][2] in
 * {0, 1} (device), into grad [HQA_MLP_PARAMS] and loss [1] (device; loss
 * may be NULL). */
hqa_status hqa_mlp_grad(hqa_mlp* mlp, int64_t n, const float* x, const float* y, float* grad,
                        float* loss, int32_t precision, void* stream);
/* One AdamW step (decoupled weight decay) with device gradient `grad`. */
hqa_status hqa_mlp_adamw(hqa_mlp* mlp, const float* grad, float lr, float beta1, float beta2,
                         float eps, float weight_decay, void* stream);
void hqa_mlp_destroy(hqa_mlp* mlp);

/* Features of the first `steps` leapfrog steps of a trajectory (same
 * schedule, dt, seed and opts as the full run), computed by running those
 * steps as `segments` consecutive resumed runs and sampling phi and the
 * local field L at every segment end.  features: device [R][N][6], per spin
 *   (phi, p, mean L, variance L, window mean of phi, fraction of sign
 *   changes of phi between consecutive samples),
 * each z-scored over the N spins of its replica.  phi, p: device [R][N],
 * the state after `steps` (phi^(S), p^(S-1/2)) from which the full run can
 * resume (start_step = steps).  1 <= segments <= steps; opts->start_step
 * must be 0. */
hqa_status hqa_run_features(hqa_ctx* ctx, const hqa_schedule* sched, double dt, int64_t steps,
                            int32_t segments, int32_t replicas, uint64_t seed,
                            const hqa_run_opts* opts, float* features, float* phi, float* p,
                            void* stream);

/* Readout driven by the network's logits ([R][N][2], device: z_f frozen,
 * z_s spin +1): s = sgn(z_s); the n spins of least confidence
 * c = sigmoid(z_f) |2 sigmoid(z_s) - 1| are ambivalent (ties by index);
 * accept[r] = 1 when the expected number of wrong frozen signs,
 * E_r = sum_frozen (1 - |2 sigmoid(z_s) - 1|) / 2, is <= max_expected_errors.
 * spins, frozen: device [R][N]; accept (uint8), expected_errors (float):
 * device [R], either may be NULL. */
hqa_status hqa_surrogate_readout(hqa_ctx* ctx, int32_t replicas, const float* logits, int32_t n,
                                 float max_expected_errors, int8_t* spins, uint8_t* frozen,
                                 uint8_t* accept, float* expected_errors, void* stream);

/* Strided snapshots of the window mean along one anneal (Results, "Sorting
 * frozen and ambivalent variables", Fig. 4: how spins separate into frozen
 * and ambivalent as tau grows).  The `steps` steps run as consecutive
 * resumed segments of `stride` steps (the last may be shorter), bitwise the
 * trajectory of one hqa_run with the same arguments; snapshot t is the
 * window mean of segment t's last min(W, segment length) steps, so with
 * stride >= W it equals the phibar of a run stopped after that segment.
 * phibar_trace: device [T][R][N] float, T = ceil(steps / stride); phi, p:
 * device [R][N], the final state (phi^(S), p^(S-1/2)).  opts->start_step
 * must be 0.  Errors as hqa_run. */
hqa_status hqa_run_trace(hqa_ctx* ctx, const hqa_schedule* sched, double dt, int64_t steps,
                         int64_t stride, int32_t replicas, uint64_t seed, const hqa_run_opts* opts,
                         float* phibar_trace, float* phi, float* p, void* stream);

/* MD Hamiltonian (Results, Eq. (3)) of R states as a diagnostic:
 *   H_MD = alpha(tau) sum_i (p_i^2/2 + phi_i^M)
 *        + beta(tau) (1/2 sum_ij J_ij phi_i phi_j + sum_i h_i |phi_i| phi_i),
 * alpha, beta from `sched` at tau (PAPER or LINEAR_GAMMA kinds; a TABLE
 * schedule has no value between its samples: UNSUPPORTED).  With half_kick
 * != 0 the momenta are first completed to the integer step,
 * p - (h/2) dH_MD/dphi (h = sched->hstep), so that hqa_run's p^(S-1/2)
 * gives H_MD at step S.  phi, p: device [R][N] float; out: device [R]
 * double.  The local field is the library's (opts: precision, kernel; NULL =
 * defaults); the per-spin terms and their sum are FP64.  Not for batch
 * contexts (UNSUPPORTED). */
hqa_status hqa_hmd(hqa_ctx* ctx, const hqa_schedule* sched, double tau, int32_t replicas,
                   const float* phi, const float* p, int32_t half_kick, double* out,
                   const hqa_run_opts* opts, void* stream);

/* Autotuner: times each launch shape hqa_run can use for `replicas`
 * replicas at opts->precision (NULL = defaults) -- the scalar sparse kernel
 * at 1, 2, 4, ..., 32 replicas per block, the vectorised one at the
 * blockings that fill a 16-byte vector, the persistent batch kernels
 * (batch contexts: list-streaming at 1..32, HQA_KERNEL_LOWDEG at 1, 2, 4
 * when every member allows it), the dense tensor-core kernel (dense BF16/BF16X2)
 * -- on a probe anneal of probe_steps steps (1..100000; dt = 1/probe_steps,
 * init PAPER), one untimed run then three between CUDA events on `stream`.
 * The fastest is written to *best (the other fields from opts) and kept in
 * the context: later hqa_run calls for the same replica count and precision
 * whose opts leave kernel (AUTO) and replicas_per_block (0) open use it.
 * table (may be NULL when table_cap = 0) receives up to table_cap entries,
 * *table_len (may be NULL) the number of candidates; a candidate the
 * library rejects has ms_per_step = -1.  Synchronises `stream`; the probe
 * outputs go to a context workspace.  Errors: INVALID_ARG, UNSUPPORTED (no
 * candidate runs, or called during a capture), OOM, CUDA, and a status a
 * probe latched (NONFINITE, TIMEOUT). */
typedef struct {
    int32_t kernel;               /* HQA_KERNEL_SCALAR, _VECTOR or _DENSE */
    int32_t replicas_per_block;   /* 0 for the dense kernel */
    double ms_per_step;           /* mean over the timed probes; -1 = rejected */
} hqa_tune_entry;
hqa_status hqa_autotune(hqa_ctx* ctx, const hqa_schedule* sched, int32_t replicas,
                        const hqa_run_opts* opts, int32_t probe_steps, hqa_run_opts* best,
                        hqa_tune_entry* table, int32_t table_cap, int32_t* table_len,
                        void* stream);

/* CUDA-graph capture of a sequence of library calls made by this thread on
 * `stream` (a created stream: the legacy default stream, NULL, cannot be
 * captured).  Every call between begin and end must find what it needs
 * already prepared by an identical earlier call without capture: launch
 * plans, the schedule table, workspaces and batch work tables.  A call that
 * would have to allocate, upload from the host or synchronise returns
 * HQA_ERR_UNSUPPORTED instead (the dense tensor-core MD is recorded as a
 * cooperative kernel node, or as a kernel node with a 2-CTA cluster shape
 * when its row tiles run as CTA pairs);
 * hqa_capture_end then returns the first failure of the capture and no
 * graph.  hqa_capture_end must follow every successful hqa_capture_begin.
 * The graph replays the same launches with the same pointers and
 * arguments: the caller keeps those buffers alive and may change their
 * contents between replays.  The graph also reads device buffers and tables
 * its contexts own (schedule table, workspaces, batch work tables): once a
 * later call has reallocated or re-uploaded any of them (another step
 * count, dt, seed of a batch run, a larger workspace), or a context is
 * destroyed, hqa_graph_launch refuses the graph with HQA_ERR_INVALID_ARG.
 * hqa_sync is not capturable. */
typedef struct hqa_graph hqa_graph;
hqa_status hqa_capture_begin(void* stream);
hqa_status hqa_capture_end(void* stream, hqa_graph** out);
hqa_status hqa_graph_launch(hqa_graph* graph, void* stream);
void hqa_graph_destroy(hqa_graph* graph);

/* Exercises the dense kernel's bounded waits (every spin of the persistent
 * tensor-core MD kernel gives up after a time limit, latches
 * HQA_ERR_TIMEOUT and leaves, so a lost arrival never hangs the GPU).
 * Arms a one-shot check for the next dense MD launch on `ctx`: before step
 * `step` every CTA's producer waits until the device word `flag` is
 * nonzero, for at most limit_ns (1 ns .. 10 s).  With a flag that nothing
 * sets the wait runs out, the launch stops early and hqa_sync returns
 * HQA_ERR_TIMEOUT; the context stays usable.  With a set flag the launch
 * is unchanged.  Dense contexts only (UNSUPPORTED otherwise). */
hqa_status hqa_arm_wait_check(hqa_ctx* ctx, const uint32_t* flag, int64_t step, int64_t limit_ns);

/* Shared-memory bandwidth of the current device in GB/s (no counterpart in the
 * paper: the measured peak for the roofline of the sparse and batch MD
 * kernels, whose neighbour gathers are shared-memory loads).  Two CTAs of 1024
 * threads per SM stream conflict-free 128-bit ld.shared loads over 32 KB;
 * the best of three timed launches (CUDA events on `stream`, after one
 * warm-up) is returned in *gbps.  Synchronises `stream`; allocates a small
 * result buffer.  Errors: INVALID_ARG (null gbps), UNSUPPORTED (during a
 * capture), CUDA, OOM. */
hqa_status hqa_probe_smem_bandwidth(double* gbps, void* stream);

/* L2 read bandwidth of the current device in GB/s (no counterpart in the
 * paper: the measured peak for the roofline of the streaming sparse kernel,
 * whose gathers are L2 reads).  Two CTAs of 1024 threads per SM read a buffer
 * of half the L2 size with 16-byte ld.global.cg loads, 40 grid-stride passes
 * per launch; the best of three timed launches (CUDA events on `stream`, after
 * one warm-up) is returned in *gbps.  Synchronises `stream`; allocates and
 * frees the buffer.  Errors: INVALID_ARG, UNSUPPORTED (during a capture),
 * CUDA, OOM. */
hqa_status hqa_probe_l2_bandwidth(double* gbps, void* stream);

/* Waits for the context's work on `stream` and returns (and clears) the
 * latched device-side status. */
hqa_status hqa_sync(hqa_ctx* ctx, void* stream);

/* Static description of a status code. */
const char* hqa_status_string(hqa_status s);

/* Frees the context and its device memory (synchronises the device). */
void hqa_destroy(hqa_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HQA_H */
