/*
 * hqa_oracle.c -- plain FP64 CPU oracle for HQA-MD (arXiv:2004.03972).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header or constant table with the CUDA
 * path under paper_2004_03972_gb300/csrc/.
 *
 * Every function follows the paper's definitions in the paper's order, with
 * no blocking, fusion or reordering:
 *   - Ising energy ................ Results, Eq. (1) (eq:Ising)
 *   - MD Hamiltonian .............. Results, Eq. (3) (Eq-MD-Hamiltonian), V = phi^M
 *   - scheduling functions ........ Methods, "Scheduling functions for MD"
 *   - leapfrog + initial half step  Methods, "Leapfrog algorithm"
 *   - time-averaged flux .......... Results, "Sorting frozen and ambivalent variables" (Eq. 5)
 *   - sorting / projection ........ same section; HQA section (projection s = sgn(phibar))
 *   - reduced Ising problem ....... HQA section, Eqs. (6)-(7) (J_eff, h_eff)
 *   - MAX-CUT <-> Ising ........... Methods, "MAX-CUT and Ising spin-glass"
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), written here from that
 * published definition.
 *
 * Readings where the paper is silent:
 *   h = dtau/g is a free step factor, 1 in the paper (g = dtau identification).
 *   Window: rectangle rule over the last W integer-step samples phi^(m),
 *           m in [max(1, S-W+1), S].
 *   sgn(0) = +1.  Rank ties broken by spin index.
 *   Sub-solve: configurations x over the ambivalent set in ascending spin
 *           index, bit k = 1 <=> s = -1; minimum energy, ties -> smallest x.
 *
 * Parity status: every function here is pinned by a CPU test (see
 * tests/test_oracle_*.py) except where noted "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Schedules (Methods, "Scheduling functions for MD").                 */
/* prm = {alpha_f, rho1, rho2, beta_f, kappa1, kappa2, gamma0}          */
/* kind 0: the paper's polynomials.                                    */
/* kind 1: alpha(tau) = gamma0 (1 - tau) (a linear transverse-field     */
/*         analogue), beta(tau) = the paper's polynomial.               */
/* ------------------------------------------------------------------ */
void or_schedule(int kind, const double* prm, double tau, double* alpha, double* beta)
{
    double alpha_f = prm[0], rho1 = prm[1], rho2 = prm[2];
    double beta_f = prm[3], kappa1 = prm[4], kappa2 = prm[5];
    double gamma0 = prm[6];
    double b = beta_f * (tau + kappa1 * (1.0 - tau) + kappa2 * tau * (tau - 1.0));
    double a;
    if (kind == 1)
        a = gamma0 * (1.0 - tau);
    else
        a = alpha_f * (tau + rho1 * (1.0 - tau) + rho2 * tau * (tau - 1.0));
    *alpha = a;
    *beta = b;
}

/* ------------------------------------------------------------------ */
/* SplitMix64: state advances by the golden gamma, output is the        */
/* published 64-bit finaliser.  or_splitmix64_at returns output number  */
/* (counter + 1) of the stream seeded with `seed`.                      */
/* ------------------------------------------------------------------ */
uint64_t or_splitmix64_at(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Initial momenta p_i(0) = +-1 (Results, after Eq. (4)): the sign is the
 * top bit of output (replica << 32 | i) of the stream. */
void or_initial_momenta(uint64_t seed, int64_t replica, int32_t N, double* p0)
{
    for (int32_t i = 0; i < N; ++i) {
        uint64_t z = or_splitmix64_at(seed, ((uint64_t)replica << 32) | (uint64_t)i);
        p0[i] = (z >> 63) ? -1.0 : 1.0;
    }
}

/* Random initial flux (an optional start, not the paper's phi(0) = 0):
 * phi_i = (k - 2^23) * 2^-26 with k the top 24 bits of output
 * (2^62 | replica << 32 | i); uniform on [-1/8, 1/8) and exact in FP32. */
void or_initial_flux_random(uint64_t seed, int64_t replica, int32_t N, double* phi0)
{
    for (int32_t i = 0; i < N; ++i) {
        uint64_t c = (1ull << 62) | ((uint64_t)replica << 32) | (uint64_t)i;
        uint64_t z = or_splitmix64_at(seed, c);
        int64_t k = (int64_t)(z >> 40);
        phi0[i] = (double)(k - (1 << 23)) * ldexp(1.0, -26);
    }
}

/* ------------------------------------------------------------------ */
/* Couplings.  Either dense (J != NULL, N*N row-major) or CSR           */
/* (row_ptr[N+1], col[nnz], val[nnz]).  Diagonal entries are ignored:   */
/* every sum in Eqs. (1) and (3) runs over j != i.                       */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t N;
    const double* J;
    const int64_t* row_ptr;
    const int32_t* col;
    const double* val;
    const double* h; /* may be NULL (h = 0) */
} or_problem;

static double coupling_sum(const or_problem* pr, const double* x, int32_t i)
{
    double s = 0.0;
    if (pr->J) {
        for (int32_t j = 0; j < pr->N; ++j)
            if (j != i) s += pr->J[(int64_t)i * pr->N + j] * x[j];
    } else {
        for (int64_t k = pr->row_ptr[i]; k < pr->row_ptr[i + 1]; ++k)
            if (pr->col[k] != i) s += pr->val[k] * x[pr->col[k]];
    }
    return s;
}

/* The part of dH_MD/dphi_i proportional to beta (Eq. (3)):
 *   sum_{j != i} J_ij phi_j + 2 h_i |phi_i|. */
void or_beta_field(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                   const double* val, const double* h, const double* phi, double* out)
{
    or_problem pr = {N, J, row_ptr, col, val, h};
    for (int32_t i = 0; i < N; ++i) {
        double L = coupling_sum(&pr, phi, i);
        if (h) L += 2.0 * h[i] * fabs(phi[i]);
        out[i] = L;
    }
}

static double ipow(double x, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= x;
    return r;
}

/* H_MD(phi, p; tau), Eq. (3), with V(phi) = phi^M. */
double or_hmd(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
              const double* val, const double* h, int kind, const double* prm, int M,
              double tau, const double* phi, const double* p)
{
    or_problem pr = {N, J, row_ptr, col, val, h};
    double alpha, beta;
    or_schedule(kind, prm, tau, &alpha, &beta);
    double kin = 0.0, pair = 0.0, field = 0.0;
    for (int32_t i = 0; i < N; ++i) kin += 0.5 * p[i] * p[i] + ipow(phi[i], M);
    for (int32_t i = 0; i < N; ++i) pair += phi[i] * coupling_sum(&pr, phi, i);
    pair *= 0.5;
    if (h)
        for (int32_t i = 0; i < N; ++i) field += h[i] * fabs(phi[i]) * phi[i];
    return alpha * kin + beta * (pair + field);
}

/* dH_MD/dphi_i = alpha M phi^(M-1) + beta (sum_j J_ij phi_j + 2 h_i |phi_i|). */
void or_force(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
              const double* val, const double* h, int kind, const double* prm, int M, double tau,
              const double* phi, double* F)
{
    double alpha, beta;
    or_schedule(kind, prm, tau, &alpha, &beta);
    or_beta_field(N, J, row_ptr, col, val, h, phi, F);
    for (int32_t i = 0; i < N; ++i) F[i] = alpha * M * ipow(phi[i], M - 1) + beta * F[i];
}

/* alpha, beta at tau = k * dt / 2 (half-step grid).  kind 2 reads the
 * caller's tables: ta[k] = alpha at tau = k dt/2 (k = 0..2S), tb[m] = beta
 * at tau = m dt (m = 0..S). */
static void sched_at_half(int kind, const double* prm, const double* ta, const double* tb, double dt,
                          int64_t k, double* alpha, double* beta)
{
    if (kind == 2) {
        *alpha = ta[k];
        *beta = (k % 2 == 0) ? tb[k / 2] : NAN;
        return;
    }
    or_schedule(kind, prm, 0.5 * (double)k * dt, alpha, beta);
}

/* ------------------------------------------------------------------ */
/* Leapfrog MD run (Methods, "Leapfrog algorithm"), one replica.        */
/*   p^(1/2)   = p^(0)   - (h/2) [alpha^(0) V'(phi^(0)) + beta^(0) B(phi^(0))]   */
/*   phi^(1)   = phi^(0) + h alpha^(1/2) p^(1/2)                          */
/*   p^(m+3/2) = p^(m+1/2) - h [alpha^(m+1) V'(phi^(m+1)) + beta^(m+1) B(phi^(m+1))] */
/*   phi^(m+2) = phi^(m+1) + h alpha^(m+3/2) p^(m+3/2)                     */
/* with B = or_beta_field and V' = M phi^(M-1).  S kicks and S drifts     */
/* produce phi^(S) and p^(S-1/2).  The window mean averages phi^(m) for   */
/* m = max(1, S-W+1) .. S.                                                */
/* hmd_trace (optional, S+1 values): H_MD at integer step m with           */
/* p^(m) = (p^(m-1/2) + p^(m+1/2)) / 2 for 0 < m < S, p^(0) at m = 0 and   */
/* at m = S the value p^(S-1/2) + (h/2)(-F(phi^(S))) is used (half kick).   */
/* ------------------------------------------------------------------ */
int or_md_run(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
              const double* val, const double* h, int kind, const double* prm, const double* ta,
              const double* tb, int M, double hstep, double dt, int64_t S, int32_t W,
              const double* phi0, const double* p0, double* out_phi, double* out_p,
              double* out_phibar, double* hmd_trace)
{
    if (S < 1 || N < 1) return 1;
    double* phi = (double*)malloc(sizeof(double) * N);
    double* p = (double*)malloc(sizeof(double) * N);
    double* Bf = (double*)malloc(sizeof(double) * N);
    double* wsum = (double*)calloc((size_t)N, sizeof(double));
    double* pprev = hmd_trace ? (double*)malloc(sizeof(double) * N) : NULL;
    double* pint = hmd_trace ? (double*)malloc(sizeof(double) * N) : NULL;
    memcpy(phi, phi0, sizeof(double) * N);
    memcpy(p, p0, sizeof(double) * N);
    int64_t first_window = S - W + 1;
    if (first_window < 1) first_window = 1;

    for (int64_t m = 0; m < S; ++m) {
        /* kick at integer step m: F(phi^(m), tau_m) */
        double alpha, beta, alpha_half, dummy;
        sched_at_half(kind, prm, ta, tb, dt, 2 * m, &alpha, &beta);
        sched_at_half(kind, prm, ta, tb, dt, 2 * m + 1, &alpha_half, &dummy);
        or_beta_field(N, J, row_ptr, col, val, h, phi, Bf);
        double c = (m == 0) ? 0.5 : 1.0;
        if (hmd_trace) memcpy(pprev, p, sizeof(double) * N);
        for (int32_t i = 0; i < N; ++i) {
            double F = alpha * M * ipow(phi[i], M - 1) + beta * Bf[i];
            p[i] = p[i] - c * hstep * F;
        }
        if (hmd_trace) {
            /* H_MD at integer step m (before the drift) */
            for (int32_t i = 0; i < N; ++i) pint[i] = (m == 0) ? pprev[i] : 0.5 * (pprev[i] + p[i]);
            hmd_trace[m] = or_hmd(N, J, row_ptr, col, val, h, kind == 2 ? 0 : kind, prm, M,
                                  (double)m * dt, phi, pint);
            if (kind == 2) hmd_trace[m] = NAN; /* table schedules: no closed form for H_MD */
        }
        /* drift with alpha^(m+1/2) */
        for (int32_t i = 0; i < N; ++i) phi[i] = phi[i] + hstep * alpha_half * p[i];
        if (m + 1 >= first_window)
            for (int32_t i = 0; i < N; ++i) wsum[i] += phi[i];
    }
    if (hmd_trace) {
        double alpha, beta;
        sched_at_half(kind, prm, ta, tb, dt, 2 * S, &alpha, &beta);
        or_beta_field(N, J, row_ptr, col, val, h, phi, Bf);
        for (int32_t i = 0; i < N; ++i) {
            double F = alpha * M * ipow(phi[i], M - 1) + beta * Bf[i];
            pint[i] = p[i] - 0.5 * hstep * F;
        }
        hmd_trace[S] = (kind == 2) ? NAN
                                   : or_hmd(N, J, row_ptr, col, val, h, kind, prm, M,
                                            (double)S * dt, phi, pint);
    }
    int64_t nwin = S - first_window + 1;
    memcpy(out_phi, phi, sizeof(double) * N);
    memcpy(out_p, p, sizeof(double) * N);
    if (out_phibar)
        for (int32_t i = 0; i < N; ++i) out_phibar[i] = wsum[i] / (double)nwin;
    free(phi); free(p); free(Bf); free(wsum); free(pprev); free(pint);
    return 0;
}

/* Many independent replicas (used to time the oracle on the host cores).
 * phi0/p0/out_* are [R][N]; the loop over replicas is the only parallelism. */
int or_md_run_replicas(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                       const double* val, const double* h, int kind, const double* prm, int M,
                       double hstep, double dt, int64_t S, int32_t W, int32_t R,
                       const double* phi0, const double* p0, double* out_phi, double* out_p,
                       double* out_phibar, int32_t threads)
{
    int rc = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
#endif
    for (int32_t r = 0; r < R; ++r) {
        size_t o = (size_t)r * (size_t)N;
        rc |= or_md_run(N, J, row_ptr, col, val, h, kind, prm, NULL, NULL, M, hstep, dt, S, W,
                        phi0 + o, p0 + o, out_phi + o, out_p + o,
                        out_phibar ? out_phibar + o : NULL, NULL);
    }
    return rc;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Readout: projection and sorting (Results, "Sorting frozen and        */
/* ambivalent variables"; HQA section).                                 */
/*   s_i = sgn(phibar_i) (sgn(0) = +1)                                  */
/*   order spins by (|phibar_i|, i) ascending; the first n are          */
/*   ambivalent (frozen = 0), the rest frozen (frozen = 1).             */
/* n is clamped to [0, N].  Rank of spin i = number of spins that come  */
/* before it in that order (a plain O(N^2) count).                      */
/* ------------------------------------------------------------------ */
void or_readout(int32_t N, const double* phibar, int32_t n, int8_t* spins, uint8_t* frozen)
{
    if (n < 0) n = 0;
    if (n > N) n = N;
    for (int32_t i = 0; i < N; ++i) {
        spins[i] = (phibar[i] >= 0.0) ? 1 : -1;
        double a = fabs(phibar[i]);
        int64_t rank = 0;
        for (int32_t j = 0; j < N; ++j) {
            double b = fabs(phibar[j]);
            if (b < a || (b == a && j < i)) ++rank;
        }
        frozen[i] = (rank >= n) ? 1 : 0;
    }
}

/* ------------------------------------------------------------------ */
/* Integer Ising energy, Eq. (1): H(s) = 1/2 sum_{i != j} J_ij s_i s_j  */
/* + sum_i h_i s_i, for integer-valued J and h, in int64.                */
/* Each term J_ij s_i s_j is taken once per ordered pair, then halved   */
/* (the ordered-pair sum is even for symmetric J).                       */
/* ------------------------------------------------------------------ */
static int64_t as_int(double v) { return (int64_t)llround(v); }

int64_t or_energy_int(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                      const double* val, const double* h, const int8_t* s)
{
    int64_t ordered = 0, field = 0;
    for (int32_t i = 0; i < N; ++i) {
        if (J) {
            for (int32_t j = 0; j < N; ++j)
                if (j != i) ordered += as_int(J[(int64_t)i * N + j]) * s[i] * s[j];
        } else {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                if (col[k] != i) ordered += as_int(val[k]) * s[i] * s[col[k]];
        }
        if (h) field += as_int(h[i]) * s[i];
    }
    return ordered / 2 + field;
}

/* Ising energy for real couplings and field (Results Eq. (1)), FP64:
 *   H(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i,
 * the pair sum taken over unordered pairs i < j directly. */
double or_energy_f64(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                     const double* val, const double* h, const int8_t* s)
{
    double pair = 0.0, field = 0.0;
    for (int32_t i = 0; i < N; ++i) {
        if (J) {
            for (int32_t j = i + 1; j < N; ++j) pair += J[(int64_t)i * N + j] * s[i] * s[j];
        } else {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                if (col[k] > i) pair += val[k] * s[i] * s[col[k]];
        }
        if (h) field += h[i] * s[i];
    }
    return pair + field;
}

/* MAX-CUT value C(s) = 1/2 sum_{(ij) in E} w_ij (1 - s_i s_j) (Methods,
 * "MAX-CUT and Ising spin-glass"), edges = unordered pairs i < j with
 * w_ij = J_ij != 0.  Written as the edge sum itself, not via C_0. */
int64_t or_cut_int(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                   const double* val, const int8_t* s)
{
    int64_t twice = 0;
    for (int32_t i = 0; i < N; ++i) {
        if (J) {
            for (int32_t j = i + 1; j < N; ++j) twice += as_int(J[(int64_t)i * N + j]) * (1 - s[i] * s[j]);
        } else {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                if (col[k] > i) twice += as_int(val[k]) * (1 - s[i] * s[col[k]]);
        }
    }
    return twice / 2;
}

/* Brute force ground state of Eq. (1) for N <= 24: x in [0, 2^N), bit i
 * of x = 1 <=> s_i = -1; returns min energy, *argmin = smallest x. */
int64_t or_brute_force(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                       const double* val, const double* h, uint64_t* argmin)
{
    int8_t* s = (int8_t*)malloc((size_t)N);
    int64_t best = INT64_MAX;
    uint64_t bx = 0;
    for (uint64_t x = 0; x < (1ull << N); ++x) {
        for (int32_t i = 0; i < N; ++i) s[i] = ((x >> i) & 1u) ? -1 : 1;
        int64_t e = or_energy_int(N, J, row_ptr, col, val, h, s);
        if (e < best) { best = e; bx = x; }
    }
    free(s);
    *argmin = bx;
    return best;
}

/* ------------------------------------------------------------------ */
/* Reduced Ising problem and its exact solution (HQA section, Eqs.      */
/* (6)-(7)).  Frozen spins keep s = spins_in; the n ambivalent spins    */
/* a_0 < a_1 < ... (ascending index) form                               */
/*   H'(s) = sum_{a<b} J_ab s_a s_b + sum_a h_eff_a s_a,                */
/*   h_eff_a = h_a + sum_{k frozen} J_ak s_k.                           */
/* Every x in [0, 2^n) is evaluated from that definition (bit k of x =  */
/* 1 <=> s_{a_k} = -1); the minimum with the smallest x wins.  The full  */
/* assignment is written to spins_out and its full energy (Eq. (1)) is  */
/* returned.  *xmin and *emin report the reduced optimum.  n <= 30.      */
/* ------------------------------------------------------------------ */
int64_t or_subsolve(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                    const double* val, const double* h, const int8_t* spins_in,
                    const uint8_t* frozen, int8_t* spins_out, uint64_t* xmin, int64_t* emin)
{
    int32_t n = 0;
    for (int32_t i = 0; i < N; ++i) n += frozen[i] ? 0 : 1;
    int32_t* amb = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * N);
    for (int32_t i = 0, k = 0; i < N; ++i) {
        pos[i] = -1;
        if (!frozen[i]) { amb[k] = i; pos[i] = k; ++k; }
    }
    /* J_eff (n x n, int64) and h_eff (Eq. (7)) */
    int64_t* Je = (int64_t*)calloc((size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t* he = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    for (int32_t a = 0; a < n; ++a) {
        int32_t i = amb[a];
        he[a] = h ? as_int(h[i]) : 0;
        if (J) {
            for (int32_t j = 0; j < N; ++j) {
                if (j == i) continue;
                int64_t w = as_int(J[(int64_t)i * N + j]);
                if (frozen[j]) he[a] += w * spins_in[j];
                else Je[(int64_t)a * n + pos[j]] = w;
            }
        } else {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col[k];
                if (j == i) continue;
                int64_t w = as_int(val[k]);
                if (frozen[j]) he[a] += w * spins_in[j];
                else Je[(int64_t)a * n + pos[j]] += w;
            }
        }
    }
    int64_t best = INT64_MAX;
    uint64_t bx = 0;
    int8_t* s = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
    for (uint64_t x = 0; x < (1ull << n); ++x) {
        for (int32_t a = 0; a < n; ++a) s[a] = ((x >> a) & 1u) ? -1 : 1;
        int64_t e = 0;
        for (int32_t a = 0; a < n; ++a) {
            for (int32_t b = a + 1; b < n; ++b) e += Je[(int64_t)a * n + b] * s[a] * s[b];
            e += he[a] * s[a];
        }
        if (e < best) { best = e; bx = x; }
    }
    for (int32_t i = 0; i < N; ++i) spins_out[i] = spins_in[i];
    for (int32_t a = 0; a < n; ++a) spins_out[amb[a]] = ((bx >> a) & 1u) ? -1 : 1;
    *xmin = bx;
    *emin = best;
    int64_t full = or_energy_int(N, J, row_ptr, col, val, h, spins_out);
    free(amb); free(pos); free(Je); free(he); free(s);
    return full;
}

/* ------------------------------------------------------------------ */
/* Surrogate MLP (a learned gate added on top of the method; the paper */
/* has none).  6 inputs -> 64 ReLU -> 64 ReLU -> 2 logits; each logit   */
/* is an independent sigmoid output with binary cross-entropy:          */
/*   loss = (1/n) sum_samples sum_o [ softplus(z_o) - y_o z_o ].        */
/* params: W1[64][6], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].     */
/* The backward pass is the chain rule written out layer by layer.      */
/* Returns the mean loss; grad (if not NULL) receives d loss / d params; */
/* logits (if not NULL) receives z [n][2].                              */
/* ------------------------------------------------------------------ */
#define OR_MLP_IN 6
#define OR_MLP_H 64
#define OR_MLP_OUT 2

static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

double or_mlp_loss_grad(int64_t n, const double* x, const double* y, const double* params,
                        double* grad, double* logits)
{
    const double* W1 = params;
    const double* b1 = W1 + OR_MLP_H * OR_MLP_IN;
    const double* W2 = b1 + OR_MLP_H;
    const double* b2 = W2 + OR_MLP_H * OR_MLP_H;
    const double* W3 = b2 + OR_MLP_H;
    const double* b3 = W3 + OR_MLP_OUT * OR_MLP_H;
    const int P = OR_MLP_H * OR_MLP_IN + OR_MLP_H + OR_MLP_H * OR_MLP_H + OR_MLP_H +
                  OR_MLP_OUT * OR_MLP_H + OR_MLP_OUT;
    double *gW1 = NULL, *gb1 = NULL, *gW2 = NULL, *gb2 = NULL, *gW3 = NULL, *gb3 = NULL;
    if (grad) {
        memset(grad, 0, sizeof(double) * P);
        gW1 = grad;
        gb1 = gW1 + OR_MLP_H * OR_MLP_IN;
        gW2 = gb1 + OR_MLP_H;
        gb2 = gW2 + OR_MLP_H * OR_MLP_H;
        gW3 = gb2 + OR_MLP_H;
        gb3 = gW3 + OR_MLP_OUT * OR_MLP_H;
    }
    double loss = 0.0;
    double a1[OR_MLP_H], h1[OR_MLP_H], a2[OR_MLP_H], h2[OR_MLP_H], z[OR_MLP_OUT];
    double dz[OR_MLP_OUT], dh2[OR_MLP_H], da2[OR_MLP_H], dh1[OR_MLP_H], da1[OR_MLP_H];
    for (int64_t s = 0; s < n; ++s) {
        const double* xs = x + s * OR_MLP_IN;
        /* forward */
        for (int k = 0; k < OR_MLP_H; ++k) {
            a1[k] = b1[k];
            for (int i = 0; i < OR_MLP_IN; ++i) a1[k] += W1[k * OR_MLP_IN + i] * xs[i];
            h1[k] = a1[k] > 0 ? a1[k] : 0.0;
        }
        for (int j = 0; j < OR_MLP_H; ++j) {
            a2[j] = b2[j];
            for (int k = 0; k < OR_MLP_H; ++k) a2[j] += W2[j * OR_MLP_H + k] * h1[k];
            h2[j] = a2[j] > 0 ? a2[j] : 0.0;
        }
        for (int o = 0; o < OR_MLP_OUT; ++o) {
            z[o] = b3[o];
            for (int j = 0; j < OR_MLP_H; ++j) z[o] += W3[o * OR_MLP_H + j] * h2[j];
            loss += softplus(z[o]) - y[s * OR_MLP_OUT + o] * z[o];
            if (logits) logits[s * OR_MLP_OUT + o] = z[o];
        }
        if (!grad) continue;
        /* backward: d loss/d z = (sigmoid(z) - y) / n */
        for (int o = 0; o < OR_MLP_OUT; ++o) dz[o] = (sigmoid(z[o]) - y[s * OR_MLP_OUT + o]) / (double)n;
        for (int j = 0; j < OR_MLP_H; ++j) {
            dh2[j] = 0.0;
            for (int o = 0; o < OR_MLP_OUT; ++o) dh2[j] += W3[o * OR_MLP_H + j] * dz[o];
            da2[j] = a2[j] > 0 ? dh2[j] : 0.0;
        }
        for (int k = 0; k < OR_MLP_H; ++k) {
            dh1[k] = 0.0;
            for (int j = 0; j < OR_MLP_H; ++j) dh1[k] += W2[j * OR_MLP_H + k] * da2[j];
            da1[k] = a1[k] > 0 ? dh1[k] : 0.0;
        }
        for (int o = 0; o < OR_MLP_OUT; ++o) {
            gb3[o] += dz[o];
            for (int j = 0; j < OR_MLP_H; ++j) gW3[o * OR_MLP_H + j] += dz[o] * h2[j];
        }
        for (int j = 0; j < OR_MLP_H; ++j) {
            gb2[j] += da2[j];
            for (int k = 0; k < OR_MLP_H; ++k) gW2[j * OR_MLP_H + k] += da2[j] * h1[k];
        }
        for (int k = 0; k < OR_MLP_H; ++k) {
            gb1[k] += da1[k];
            for (int i = 0; i < OR_MLP_IN; ++i) gW1[k * OR_MLP_IN + i] += da1[k] * xs[i];
        }
    }
    return loss / (double)n;
}

/* AdamW (Loshchilov and Hutter, "Decoupled weight decay regularization",
 * ICLR 2019), step t >= 1 on P parameters, in place, FP64:
 *   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *   mhat = m / (1 - b1^t),   vhat = v / (1 - b2^t),
 *   w <- w - lr (mhat / (sqrt(vhat) + eps) + wd w). */
void or_adamw(int64_t P, double* w, const double* g, double* m, double* v, int64_t t, double lr,
              double b1, double b2, double eps, double wd)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t k = 0; k < P; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        const double mh = m[k] / c1, vh = v[k] / c2;
        w[k] = w[k] - lr * (mh / (sqrt(vh) + eps) + wd * w[k]);
    }
}


/* ------------------------------------------------------------------ */
/* Tabu search on the reduced problem, for ambivalent sets too large to   */
/* enumerate (the role QBSolv's tabu search plays in HQA(TS1000), HQA   */
/* section).  Deterministic single-flip tabu search, restated here as  */
/* the definition the GPU kernel must reproduce bit for bit:            */
/*   f_a = h_a + sum_{j != a} J_aj s_j for ambivalent a; flipping a     */
/*   changes the energy by d_a = -2 s_a f_a.                            */
/*   Iteration it = 1..iters: among ambivalent a that are not tabu      */
/*   (tabu_until[a] < it) or that would set a new best (E + d_a <       */
/*   E_best: aspiration), take the smallest (d_a, a); flip it (even     */
/*   uphill), update the fields of its neighbours, make it tabu until   */
/*   it + tenure; a strictly lower E becomes the new best.              */
/*   The best assignment (the input if nothing improves) is written to  */
/*   spins_out; its full energy is returned.  Integer couplings only.    */
/* ------------------------------------------------------------------ */
int64_t or_subsolve_tabu(int32_t N, const double* J, const int64_t* row_ptr, const int32_t* col,
                         const double* val, const double* h, const int8_t* spins_in,
                         const uint8_t* frozen, int32_t iters, int32_t tenure, int8_t* spins_out)
{
    int8_t* s = (int8_t*)malloc((size_t)N);
    int64_t* f = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    int64_t* until = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    memcpy(s, spins_in, (size_t)N);
    memcpy(spins_out, spins_in, (size_t)N);
    for (int32_t a = 0; a < N; ++a) {
        if (frozen[a]) continue;
        int64_t g = h ? as_int(h[a]) : 0;
        if (J) {
            for (int32_t j = 0; j < N; ++j)
                if (j != a) g += as_int(J[(int64_t)a * N + j]) * s[j];
        } else {
            for (int64_t k = row_ptr[a]; k < row_ptr[a + 1]; ++k)
                if (col[k] != a) g += as_int(val[k]) * s[col[k]];
        }
        f[a] = g;
    }
    int64_t E = 0, best = 0;   /* energies relative to the input assignment */
    for (int64_t it = 1; it <= iters; ++it) {
        int32_t w = -1;
        int64_t dw = 0;
        for (int32_t a = 0; a < N; ++a) {
            if (frozen[a]) continue;
            const int64_t d = -2 * (int64_t)s[a] * f[a];
            if (!(until[a] < it || E + d < best)) continue;
            if (w < 0 || d < dw) {   /* ascending a: ties keep the smaller index */
                w = a;
                dw = d;
            }
        }
        if (w < 0) continue;
        s[w] = (int8_t)-s[w];
        E += dw;
        /* neighbours' fields: J_jw changes sign in its contribution J_jw s_w */
        if (J) {
            for (int32_t j = 0; j < N; ++j)
                if (j != w) f[j] += 2 * as_int(J[(int64_t)j * N + w]) * s[w];
        } else {
            for (int64_t k = row_ptr[w]; k < row_ptr[w + 1]; ++k)
                if (col[k] != w) f[col[k]] += 2 * as_int(val[k]) * s[w];
        }
        until[w] = it + tenure;
        if (E < best) {
            best = E;
            memcpy(spins_out, s, (size_t)N);
        }
    }
    free(s);
    free(f);
    free(until);
    return or_energy_int(N, J, row_ptr, col, val, h, spins_out);
}
