"""ctypes front end of the FP64 CPU oracle (oracle/hqa_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing here is shared
with, or imported by, the CUDA library.  Every function converts its numpy
arguments to FP64 / int64 and calls the C routine of the same name; the
arithmetic lives in the C file, which cites the paper section each routine
restates.

Parity status: all routines are pinned by tests/test_oracle_*.py (the surrogate
gate's routines at the end by reductions and invariants, listed there).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hqa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# schedule kinds (same meaning as the library's, numbered independently)
PAPER, LINEAR_GAMMA, TABLE = 0, 1, 2
PAPER_PRM = (0.008, 4.0, 3.0, 0.12, 0.05, 1.0, 0.032)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP over replicas)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i32, i64, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint64
            vp = C.c_void_p
            lib.or_schedule.argtypes = [C.c_int, vp, d, vp, vp]
            lib.or_splitmix64_at.argtypes = [u64, u64]
            lib.or_splitmix64_at.restype = u64
            lib.or_initial_momenta.argtypes = [u64, i64, i32, vp]
            lib.or_initial_flux_random.argtypes = [u64, i64, i32, vp]
            lib.or_beta_field.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp]
            lib.or_hmd.argtypes = [i32, vp, vp, vp, vp, vp, C.c_int, vp, C.c_int, d, vp, vp]
            lib.or_hmd.restype = d
            lib.or_force.argtypes = [i32, vp, vp, vp, vp, vp, C.c_int, vp, C.c_int, d, vp, vp]
            lib.or_md_run.argtypes = [i32, vp, vp, vp, vp, vp, C.c_int, vp, vp, vp, C.c_int, d, d,
                                      i64, i32, vp, vp, vp, vp, vp, vp]
            lib.or_md_run.restype = C.c_int
            lib.or_md_run_replicas.argtypes = [i32, vp, vp, vp, vp, vp, C.c_int, vp, C.c_int, d, d,
                                               i64, i32, i32, vp, vp, vp, vp, vp, i32]
            lib.or_md_run_replicas.restype = C.c_int
            lib.or_max_threads.restype = C.c_int
            lib.or_readout.argtypes = [i32, vp, i32, vp, vp]
            lib.or_energy_int.argtypes = [i32, vp, vp, vp, vp, vp, vp]
            lib.or_energy_int.restype = i64
            lib.or_energy_f64.argtypes = [i32, vp, vp, vp, vp, vp, vp]
            lib.or_energy_f64.restype = d
            lib.or_cut_int.argtypes = [i32, vp, vp, vp, vp, vp]
            lib.or_cut_int.restype = i64
            lib.or_brute_force.argtypes = [i32, vp, vp, vp, vp, vp, vp]
            lib.or_brute_force.restype = i64
            lib.or_subsolve.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.or_subsolve.restype = i64
            lib.or_subsolve_tabu.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp]
            lib.or_subsolve_tabu.restype = i64
            lib.or_mlp_loss_grad.argtypes = [i64, vp, vp, vp, vp, vp]
            lib.or_mlp_loss_grad.restype = d
            lib.or_adamw.argtypes = [i64, vp, vp, vp, vp, i64, d, d, d, d, d]
            lib.or_adamw.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Problem:
    """Couplings in FP64: dense ``J`` (N x N) or CSR (row_ptr, col, val); field ``h``."""

    def __init__(self, N, J=None, row_ptr=None, col=None, val=None, h=None):
        self.N = int(N)
        self.J = None if J is None else np.ascontiguousarray(J, dtype=np.float64)
        self.row_ptr = None if row_ptr is None else np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = None if col is None else np.ascontiguousarray(col, dtype=np.int32)
        self.val = None if val is None else np.ascontiguousarray(val, dtype=np.float64)
        self.h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
        if self.J is None and self.row_ptr is None:
            raise ValueError("need dense J or CSR")

    @classmethod
    def from_instance(cls, inst):
        if inst.dense is not None:
            return cls(inst.N, J=inst.dense, h=inst.h)
        return cls(inst.N, row_ptr=inst.row_ptr, col=inst.col, val=inst.val, h=inst.h)

    def args(self):
        return (self.N, _ptr(self.J), _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                _ptr(self.h))


def _prm(prm):
    return np.ascontiguousarray(prm if prm is not None else PAPER_PRM, dtype=np.float64)


def schedule(tau, kind=PAPER, prm=None):
    lib = _load()
    p = _prm(prm)
    a, b = C.c_double(), C.c_double()
    lib.or_schedule(kind, _ptr(p), float(tau), C.byref(a), C.byref(b))
    return a.value, b.value


def splitmix64_at(seed, counter):
    return int(_load().or_splitmix64_at(seed, counter))


def initial_momenta(seed, replica, N):
    out = np.empty(N, np.float64)
    _load().or_initial_momenta(seed, replica, N, _ptr(out))
    return out


def initial_flux_random(seed, replica, N):
    out = np.empty(N, np.float64)
    _load().or_initial_flux_random(seed, replica, N, _ptr(out))
    return out


def beta_field(pr: Problem, phi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    out = np.empty(pr.N, np.float64)
    _load().or_beta_field(*pr.args(), _ptr(phi), _ptr(out))
    return out


def hmd(pr: Problem, tau, phi, p, kind=PAPER, prm=None, M=6):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    pp = _prm(prm)
    return float(_load().or_hmd(*pr.args(), kind, _ptr(pp), M, float(tau), _ptr(phi), _ptr(p)))


def force(pr: Problem, tau, phi, kind=PAPER, prm=None, M=6):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    pp = _prm(prm)
    out = np.empty(pr.N, np.float64)
    _load().or_force(*pr.args(), kind, _ptr(pp), M, float(tau), _ptr(phi), _ptr(out))
    return out


def md_run(pr: Problem, steps, dt=None, phi0=None, p0=None, kind=PAPER, prm=None, M=6, hstep=1.0,
           window=100, table_alpha=None, table_beta=None, trace=False):
    """One replica. Returns (phi^(S), p^(S-1/2), window mean[, H_MD trace])."""
    N, S = pr.N, int(steps)
    dt = 1.0 / S if dt is None else float(dt)
    phi0 = np.zeros(N) if phi0 is None else np.ascontiguousarray(phi0, dtype=np.float64)
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    pp = _prm(prm)
    ta = None if table_alpha is None else np.ascontiguousarray(table_alpha, dtype=np.float64)
    tb = None if table_beta is None else np.ascontiguousarray(table_beta, dtype=np.float64)
    phi, p, pbar = np.empty(N), np.empty(N), np.empty(N)
    tr = np.empty(S + 1) if trace else None
    rc = _load().or_md_run(*pr.args(), kind, _ptr(pp), _ptr(ta), _ptr(tb), M, float(hstep), dt, S,
                           int(window), _ptr(phi0), _ptr(p0), _ptr(phi), _ptr(p), _ptr(pbar),
                           _ptr(tr))
    if rc != 0:
        raise ValueError("oracle md_run rejected its arguments")
    return (phi, p, pbar, tr) if trace else (phi, p, pbar)


def md_run_replicas(pr: Problem, steps, phi0, p0, dt=None, kind=PAPER, prm=None, M=6, hstep=1.0,
                    window=100, threads=0):
    """R independent replicas ([R][N] inputs), OpenMP over replicas."""
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    R, N = p0.shape
    S = int(steps)
    dt = 1.0 / S if dt is None else float(dt)
    pp = _prm(prm)
    phi, p, pbar = np.empty((R, N)), np.empty((R, N)), np.empty((R, N))
    rc = _load().or_md_run_replicas(*pr.args(), kind, _ptr(pp), M, float(hstep), dt, S,
                                    int(window), R, _ptr(phi0), _ptr(p0), _ptr(phi), _ptr(p),
                                    _ptr(pbar), int(threads))
    if rc != 0:
        raise ValueError("oracle md_run_replicas rejected its arguments")
    return phi, p, pbar


def md_run_dense_batch(pr: Problem, steps, phi0, p0, dt=None, M=6, hstep=1.0, window=100):
    """R replicas of a dense problem at once, for long runs at many seeds.

    The same leapfrog as md_run (Methods, "Leapfrog algorithm"; the paper's
    schedules, Methods "Scheduling functions for MD"), step for step and in the
    same order, with the coupling sum of all replicas taken as one FP64 matrix
    product (a library primitive; only the summation order differs from the C
    routine's loop).  Inputs [R][N]; returns (phi^(S), p^(S-1/2), window mean)."""
    if pr.J is None:
        raise ValueError("md_run_dense_batch needs dense couplings")
    S = int(steps)
    dt = 1.0 / S if dt is None else float(dt)
    J = pr.J.copy()
    np.fill_diagonal(J, 0.0)          # the sums run over j != i
    phi = np.array(phi0, dtype=np.float64)
    p = np.array(p0, dtype=np.float64)
    wsum = np.zeros_like(phi)
    first_window = max(1, S - int(window) + 1)
    for m in range(S):
        alpha, beta = schedule(m * dt)
        alpha_half, _ = schedule((m + 0.5) * dt)
        L = phi @ J.T
        if pr.h is not None:
            L += 2.0 * pr.h * np.abs(phi)
        pw = phi.copy()               # phi^(M-1) as repeated products, like the C routine
        for _ in range(M - 2):
            pw *= phi
        F = alpha * M * pw + beta * L
        c = 0.5 if m == 0 else 1.0
        p = p - c * hstep * F
        phi = phi + hstep * alpha_half * p
        if m + 1 >= first_window:
            wsum += phi
    return phi, p, wsum / (S - first_window + 1)


def max_threads():
    return int(_load().or_max_threads())


def readout(phibar, n):
    phibar = np.ascontiguousarray(phibar, dtype=np.float64)
    N = phibar.shape[0]
    s = np.empty(N, np.int8)
    f = np.empty(N, np.uint8)
    _load().or_readout(N, _ptr(phibar), int(n), _ptr(s), _ptr(f))
    return s, f


def energy_int(pr: Problem, s):
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(_load().or_energy_int(*pr.args(), _ptr(s)))


def energy_f64(pr: Problem, s):
    """Ising energy for real J, h in FP64 (pair sum over i < j)."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    return float(_load().or_energy_f64(*pr.args(), _ptr(s)))


def cut_int(pr: Problem, s):
    s = np.ascontiguousarray(s, dtype=np.int8)
    N, J, rp, col, val, _ = pr.args()
    return int(_load().or_cut_int(N, J, rp, col, val, _ptr(s)))


def brute_force(pr: Problem):
    x = C.c_uint64()
    e = _load().or_brute_force(*pr.args(), C.byref(x))
    return int(e), int(x.value)


def subsolve(pr: Problem, spins, frozen):
    """Returns (full spins, full energy, reduced argmin x, reduced min energy)."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    out = np.empty(pr.N, np.int8)
    x, em = C.c_uint64(), C.c_int64()
    e = _load().or_subsolve(*pr.args(), _ptr(spins), _ptr(frozen), _ptr(out), C.byref(x),
                            C.byref(em))
    return out, int(e), int(x.value), int(em.value)


def subsolve_tabu(pr: Problem, spins, frozen, iters, tenure):
    """Deterministic tabu search on the reduced problem: (full spins, full energy)."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    out = np.empty(pr.N, np.int8)
    e = _load().or_subsolve_tabu(*pr.args(), _ptr(spins), _ptr(frozen), int(iters), int(tenure),
                                 _ptr(out))
    return out, int(e)


MLP_IN, MLP_H, MLP_OUT = 6, 64, 2
MLP_P = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT


def mlp_loss_grad(x, y, params, want_grad=True):
    """Surrogate MLP: mean BCE loss, gradient [P] and logits [n][2] (FP64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    n = x.shape[0]
    g = np.empty(MLP_P) if want_grad else None
    z = np.empty((n, MLP_OUT))
    loss = _load().or_mlp_loss_grad(n, _ptr(x), _ptr(y), _ptr(params), _ptr(g), _ptr(z))
    return float(loss), g, z


def adamw(params, grads, lr, beta1, beta2, eps, weight_decay):
    """AdamW from zero moments: applies the gradients ``grads`` (a sequence of [P]
    arrays) as steps t = 1, 2, ... and returns the parameters after each step."""
    w = np.array(params, dtype=np.float64)
    m, v = np.zeros_like(w), np.zeros_like(w)
    out = []
    for t, g in enumerate(grads, 1):
        g = np.ascontiguousarray(g, dtype=np.float64)
        _load().or_adamw(w.size, _ptr(w), _ptr(g), _ptr(m), _ptr(v), t, float(lr), float(beta1),
                         float(beta2), float(eps), float(weight_decay))
        out.append(w.copy())
    return out


# ---------------------------------------------------------------------------
# Surrogate gate (an addition to the method: the paper has no learned part).
# Plain compositions of the pinned routines above.  Parity pins:
#   surrogate_features  segments = 1 reduces to (phi, p, J.phi, 0, phibar, 0) of one
#                       md_run; Z2 covariance at h = 0; z-scored columns have mean 0, var 1
#   surrogate_readout   sigma(z_f) = 1 reduces to the method's readout on z_s; z_s = 0
#                       gives (N - n) / 2 expected errors
# ---------------------------------------------------------------------------
def segment_lengths(steps, segments):
    """The first steps % segments segments are one step longer."""
    return [steps // segments + (1 if k < steps % segments else 0) for k in range(segments)]


def surrogate_features_raw(pr: Problem, steps, segments, p0, dt, window=100, M=6, kind=PAPER,
                           prm=None, phi0=None):
    """One replica, [N][6] before z-scoring: phi and p after `steps` steps, mean and
    (population) variance of the local field L = J.phi + 2h|phi| over the states at the
    segment ends, the window mean over the last min(window, last segment) steps, and
    the fraction of consecutive segment-end states between which sgn(phi) changed
    (sgn(0) = +1).  Every segment-end state is an independent md_run from the start."""
    lens = segment_lengths(int(steps), int(segments))
    ends = np.cumsum(lens)
    Ls, sg = [], []
    for k, m in enumerate(ends):
        last = k == len(ends) - 1
        phi, p, pbar = md_run(pr, int(m), dt=dt, phi0=phi0, p0=p0, kind=kind, prm=prm, M=M,
                              window=min(window, lens[-1]) if last else window)
        Ls.append(beta_field(pr, phi))
        sg.append(np.where(phi >= 0, 1.0, -1.0))
    Ls = np.array(Ls)
    mean_L = Ls.mean(axis=0)
    var_L = np.maximum((Ls ** 2).mean(axis=0) - mean_L ** 2, 0.0)
    sg = np.array(sg)
    flips = (sg[1:] != sg[:-1]).sum(axis=0) / max(len(ends) - 1, 1)
    return np.stack([phi, p, mean_L, var_L, pbar, flips], axis=1)


def zscore(f):
    """Each column over the rows: (f - mean) / population std; a column with
    variance <= 1e-20 maps to 0."""
    mu = f.mean(axis=0)
    var = (f ** 2).mean(axis=0) - mu ** 2
    inv = np.where(var > 1e-20, 1.0 / np.sqrt(np.maximum(var, 1e-300)), 0.0)
    return (f - mu) * inv


def surrogate_readout(logits, n, max_expected_errors):
    """logits [N][2] = (z_f, z_s) of one replica.  Spins sgn(z_s) (sgn(0) = +1); the
    n spins with the smallest confidence sigma(z_f) |2 sigma(z_s) - 1| are ambivalent
    (ties by index); expected wrong frozen signs E = sum_frozen (1 - |2 sigma(z_s) - 1|)/2.
    Returns (spins, frozen, accept, E)."""
    z = np.asarray(logits, dtype=np.float64)
    sig = lambda t: 1.0 / (1.0 + np.exp(-t))
    conf = sig(z[:, 0]) * np.abs(2.0 * sig(z[:, 1]) - 1.0)
    spins = np.where(z[:, 1] >= 0, 1, -1).astype(np.int8)
    order = np.lexsort((np.arange(len(conf)), conf))
    frozen = np.ones(len(conf), np.uint8)
    frozen[order[:max(0, min(int(n), len(conf)))]] = 0
    E = float(np.sum(frozen * 0.5 * (1.0 - np.abs(2.0 * sig(z[:, 1]) - 1.0))))
    return spins, frozen, E <= max_expected_errors, E
