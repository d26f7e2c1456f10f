"""ctypes binding of libhqa.so (include/hqa.h).

Argument marshalling only: every step of HQA-MD runs in the CUDA library.
PyTorch supplies device memory and the current CUDA stream.  If the library
has not been built, ``lib()`` raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhqa.so")

HQA_OK = 0
STATUS_NAMES = {
    0: "HQA_OK", 1: "HQA_ERR_INVALID_ARG", 2: "HQA_ERR_ASYMMETRIC", 3: "HQA_ERR_NONFINITE_INPUT",
    4: "HQA_ERR_OOM", 5: "HQA_ERR_CUDA", 6: "HQA_ERR_UNSUPPORTED", 7: "HQA_ERR_NONFINITE",
    8: "HQA_ERR_TIMEOUT", 9: "HQA_ERR_TOO_LARGE",
}
SCHED_PAPER, SCHED_LINEAR_GAMMA, SCHED_TABLE = 0, 1, 2
INIT_PAPER, INIT_RANDOM_FLUX, INIT_GIVEN = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_BF16X2, PREC_FP16, PREC_FP16X2 = 0, 1, 2, 3, 4
J_BF16, J_FP16, J_FP32, J_FP8 = 1, 2, 4, 8
KERNEL_AUTO, KERNEL_SCALAR, KERNEL_VECTOR, KERNEL_DENSE, KERNEL_LOWDEG, KERNEL_STREAM = \
    0, 1, 2, 3, 4, 5

# every symbol include/hqa.h declares
EXPORTS = (
    "hqa_schedule_default", "hqa_run_opts_default", "hqa_create_dense", "hqa_create_csr",
    "hqa_create_batch",
    "hqa_ctx_info", "hqa_run", "hqa_local_field", "hqa_readout", "hqa_energy", "hqa_solve_sub",
    "hqa_solve_sub_noalloc", "hqa_plan_query", "hqa_sync", "hqa_status_string", "hqa_destroy",
    "hqa_mlp_create", "hqa_mlp_params", "hqa_mlp_forward", "hqa_mlp_grad", "hqa_mlp_adamw",
    "hqa_mlp_destroy", "hqa_run_features", "hqa_surrogate_readout",
    "hqa_capture_begin", "hqa_capture_end", "hqa_graph_launch", "hqa_graph_destroy",
    "hqa_autotune", "hqa_hmd", "hqa_energy_f64", "hqa_run_trace", "hqa_solve_sub_tabu",
    "hqa_arm_wait_check", "hqa_probe_smem_bandwidth", "hqa_probe_l2_bandwidth",
)
MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS = 6, 64, 2, 4738


class HQAError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


class Schedule(C.Structure):
    _fields_ = [
        ("kind", C.c_int32),
        ("alpha_f", C.c_double), ("rho1", C.c_double), ("rho2", C.c_double),
        ("beta_f", C.c_double), ("kappa1", C.c_double), ("kappa2", C.c_double),
        ("gamma0", C.c_double),
        ("M", C.c_int32),
        ("hstep", C.c_double),
        ("window", C.c_int32),
        ("n_ambivalent", C.c_int32),
        ("table_alpha", C.c_void_p),
        ("table_beta", C.c_void_p),
    ]


class RunOpts(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("init", C.c_int32),
        ("phi0", C.c_void_p),
        ("p0", C.c_void_p),
        ("replicas_per_block", C.c_int32),
        ("kernel", C.c_int32),
        ("start_step", C.c_int64),
    ]


class PlanInfo(C.Structure):
    _fields_ = [
        ("kernel", C.c_int32), ("replicas_per_block", C.c_int32), ("blocks", C.c_int32),
        ("threads", C.c_int32), ("smem_bytes", C.c_int64), ("pad_ratio", C.c_double),
        ("conflict_ratio", C.c_double), ("balance", C.c_double), ("chunks", C.c_int32),
    ]


class TuneEntry(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("replicas_per_block", C.c_int32),
                ("ms_per_step", C.c_double)]


class Result(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("phi", "p", "phibar", "spins", "frozen", "energy", "cut", "tally")]


_lock = threading.Lock()
_lib = None


def lib() -> C.CDLL:
    """Loads the in-tree CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libhqa.so not built ({LIB_PATH}); run __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_uint32
            L.hqa_schedule_default.argtypes = [C.POINTER(Schedule)]
            L.hqa_run_opts_default.argtypes = [C.POINTER(RunOpts)]
            L.hqa_create_dense.argtypes = [i32, vp, vp, u32, C.POINTER(vp)]
            L.hqa_create_csr.argtypes = [i32, i64, vp, vp, vp, vp, u32, C.POINTER(vp)]
            L.hqa_ctx_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]
            L.hqa_create_batch.argtypes = [i32, C.POINTER(vp), C.POINTER(vp)]
            L.hqa_run.argtypes = [vp, C.POINTER(Schedule), C.c_double, i64, i32, u64,
                                  C.POINTER(RunOpts), C.POINTER(Result), vp]
            L.hqa_local_field.argtypes = [vp, i32, vp, vp, C.POINTER(RunOpts), vp]
            L.hqa_readout.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp]
            L.hqa_energy.argtypes = [vp, i32, vp, vp, vp, vp]
            L.hqa_solve_sub.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp]
            L.hqa_solve_sub_noalloc.argtypes = [vp, i32, vp, vp, i32, vp, vp, vp]
            L.hqa_sync.argtypes = [vp, vp]
            L.hqa_plan_query.argtypes = [vp, i32, C.POINTER(RunOpts), C.POINTER(PlanInfo)]
            L.hqa_mlp_create.argtypes = [vp, C.POINTER(vp)]
            L.hqa_mlp_params.argtypes = [vp, vp]
            L.hqa_mlp_forward.argtypes = [vp, i64, vp, vp, i32, vp]
            L.hqa_mlp_grad.argtypes = [vp, i64, vp, vp, vp, vp, i32, vp]
            L.hqa_mlp_adamw.argtypes = [vp, vp, C.c_float, C.c_float, C.c_float, C.c_float,
                                        C.c_float, vp]
            L.hqa_run_features.argtypes = [vp, C.POINTER(Schedule), C.c_double, i64, i32, i32, u64,
                                           C.POINTER(RunOpts), vp, vp, vp, vp]
            L.hqa_run_features.restype = C.c_int
            L.hqa_surrogate_readout.argtypes = [vp, i32, vp, i32, C.c_float, vp, vp, vp, vp, vp]
            L.hqa_surrogate_readout.restype = C.c_int
            L.hqa_mlp_destroy.argtypes = [vp]
            L.hqa_mlp_destroy.restype = None
            for name in ("hqa_mlp_create", "hqa_mlp_params", "hqa_mlp_forward", "hqa_mlp_grad",
                         "hqa_mlp_adamw"):
                getattr(L, name).restype = C.c_int
            L.hqa_autotune.argtypes = [vp, C.POINTER(Schedule), i32, C.POINTER(RunOpts), i32,
                                       C.POINTER(RunOpts), C.POINTER(TuneEntry), i32,
                                       C.POINTER(i32), vp]
            L.hqa_autotune.restype = C.c_int
            L.hqa_probe_smem_bandwidth.argtypes = [C.POINTER(C.c_double), vp]
            L.hqa_probe_smem_bandwidth.restype = C.c_int
            L.hqa_probe_l2_bandwidth.argtypes = [C.POINTER(C.c_double), vp]
            L.hqa_probe_l2_bandwidth.restype = C.c_int
            L.hqa_arm_wait_check.argtypes = [vp, vp, i64, i64]
            L.hqa_arm_wait_check.restype = C.c_int
            L.hqa_solve_sub_tabu.argtypes = [vp, i32, vp, vp, i32, i32, i32, vp, vp, vp]
            L.hqa_solve_sub_tabu.restype = C.c_int
            L.hqa_run_trace.argtypes = [vp, C.POINTER(Schedule), C.c_double, i64, i64, i32, u64,
                                        C.POINTER(RunOpts), vp, vp, vp, vp]
            L.hqa_run_trace.restype = C.c_int
            L.hqa_energy_f64.argtypes = [vp, i32, vp, vp, vp]
            L.hqa_energy_f64.restype = C.c_int
            L.hqa_hmd.argtypes = [vp, C.POINTER(Schedule), C.c_double, i32, vp, vp, i32, vp,
                                  C.POINTER(RunOpts), vp]
            L.hqa_hmd.restype = C.c_int
            L.hqa_capture_begin.argtypes = [vp]
            L.hqa_capture_begin.restype = C.c_int
            L.hqa_capture_end.argtypes = [vp, C.POINTER(vp)]
            L.hqa_capture_end.restype = C.c_int
            L.hqa_graph_launch.argtypes = [vp, vp]
            L.hqa_graph_launch.restype = C.c_int
            L.hqa_graph_destroy.argtypes = [vp]
            L.hqa_graph_destroy.restype = None
            L.hqa_status_string.argtypes = [C.c_int]
            L.hqa_status_string.restype = C.c_char_p
            L.hqa_destroy.argtypes = [vp]
            L.hqa_destroy.restype = None
            for name in ("hqa_create_dense", "hqa_create_csr", "hqa_create_batch", "hqa_ctx_info", "hqa_run",
                         "hqa_local_field", "hqa_readout", "hqa_energy", "hqa_solve_sub",
                         "hqa_solve_sub_noalloc", "hqa_plan_query", "hqa_sync"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(st: int, what: str):
    if st != HQA_OK:
        raise HQAError(st, what)


def schedule(**kw) -> Schedule:
    """The paper's schedule (hqa_schedule_default) with keyword overrides."""
    s = Schedule()
    lib().hqa_schedule_default(C.byref(s))
    for k, v in kw.items():
        if k in ("table_alpha", "table_beta"):
            raise ValueError("use table=(alpha, beta) for HQA_SCHED_TABLE")
        setattr(s, k, v)
    return s


def _stream_ptr(stream=None):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(st.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def smem_bandwidth_probe(stream=None) -> float:
    """hqa_probe_smem_bandwidth: measured shared-memory bandwidth of the current GPU, GB/s."""
    v = C.c_double()
    _check(lib().hqa_probe_smem_bandwidth(C.byref(v), _stream_ptr(stream)),
           "hqa_probe_smem_bandwidth")
    return v.value


def l2_bandwidth_probe(stream=None) -> float:
    """hqa_probe_l2_bandwidth: measured L2 read bandwidth of the current GPU, GB/s."""
    v = C.c_double()
    _check(lib().hqa_probe_l2_bandwidth(C.byref(v), _stream_ptr(stream)), "hqa_probe_l2_bandwidth")
    return v.value


class Context:
    """Owns an hqa_ctx (device copies of the couplings)."""

    def __init__(self, handle: C.c_void_p, N: int):
        self._h = handle
        self.N = N
        self.members = None      # batch contexts: the member Contexts (kept alive here)

    @classmethod
    def batch(cls, members):
        """hqa_create_batch over existing contexts.  Spin-indexed outputs are the members'
        [R][N_k] blocks back to back (see split()); per-replica outputs are [count][R]."""
        arr = (C.c_void_p * len(members))(*[m._h.value for m in members])
        out = C.c_void_p()
        _check(lib().hqa_create_batch(len(members), arr, C.byref(out)), "hqa_create_batch")
        c = cls(out, sum(m.N for m in members))
        c.members = list(members)
        return c

    def split(self, t, R):
        """Per-member views [R][N_k] of a batch output laid out as hqa_run writes it."""
        flat = t.reshape(-1)
        views, off = [], 0
        for m in self.members:
            views.append(flat[off:off + R * m.N].view(R, m.N))
            off += R * m.N
        return views

    @classmethod
    def from_dense(cls, J, h=None, flags=0):
        """hqa_create_dense; ``flags`` (J_BF16 | J_FP16 | J_FP32) builds those coupling
        operands at create instead of on first use."""
        J = np.ascontiguousarray(J, dtype=np.float32)
        N = J.shape[0]
        hh = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
        out = C.c_void_p()
        _check(lib().hqa_create_dense(N, J.ctypes.data, None if hh is None else hh.ctypes.data,
                                      int(flags), C.byref(out)), "hqa_create_dense")
        return cls(out, N)

    @classmethod
    def from_csr(cls, N, row_ptr, col, val, h=None):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cc = np.ascontiguousarray(col, dtype=np.int32)
        vv = np.ascontiguousarray(val, dtype=np.float32)
        hh = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
        out = C.c_void_p()
        _check(lib().hqa_create_csr(int(N), int(rp[-1]), rp.ctypes.data, cc.ctypes.data,
                                    vv.ctypes.data, None if hh is None else hh.ctypes.data, 0,
                                    C.byref(out)), "hqa_create_csr")
        return cls(out, int(N))

    @classmethod
    def from_instance(cls, inst, flags=0):
        if inst.dense is not None:
            return cls.from_dense(inst.dense, inst.h, flags)
        return cls.from_csr(inst.N, inst.row_ptr, inst.col, inst.val, inst.h)

    def info(self):
        N, nnz, integ = C.c_int32(), C.c_int64(), C.c_int32()
        _check(lib().hqa_ctx_info(self._h, C.byref(N), C.byref(nnz), C.byref(integ)), "hqa_ctx_info")
        return {"N": N.value, "nnz": nnz.value, "integer": bool(integ.value)}

    def run(self, steps, replicas, seed=0, sched=None, dt=None, precision=PREC_FP32,
            init=INIT_PAPER, phi0=None, p0=None, replicas_per_block=0, outputs=None,
            out=None, stream=None, table=None, kernel=KERNEL_AUTO, start_step=0):
        """hqa_run. Returns a dict of device tensors (phi, p, phibar, spins, frozen, energy,
        cut, tally) -- those named in ``outputs`` (default: all), or the caller's ``out``."""
        import torch
        R, N = int(replicas), self.N
        sched = sched if sched is not None else schedule()
        keep = []
        if table is not None:
            ta = np.ascontiguousarray(table[0], dtype=np.float64)
            tb = np.ascontiguousarray(table[1], dtype=np.float64)
            keep += [ta, tb]
            sched.kind = SCHED_TABLE
            sched.table_alpha = ta.ctypes.data
            sched.table_beta = tb.ctypes.data
        opts = RunOpts()
        lib().hqa_run_opts_default(C.byref(opts))
        opts.precision = precision
        opts.init = init
        opts.phi0 = None if phi0 is None else phi0.data_ptr()
        opts.p0 = None if p0 is None else p0.data_ptr()
        opts.replicas_per_block = replicas_per_block
        opts.kernel = kernel
        opts.start_step = int(start_step)
        if out is None:
            dev = torch.device("cuda")
            names = outputs or ("phi", "p", "phibar", "spins", "frozen", "energy", "cut", "tally")
            Rr = R * (len(self.members) if self.members else 1)   # per-replica results
            shapes = {"phi": ((R, N), torch.float32), "p": ((R, N), torch.float32),
                      "phibar": ((R, N), torch.float32), "spins": ((R, N), torch.int8),
                      "frozen": ((R, N), torch.uint8), "energy": ((Rr,), torch.int64),
                      "cut": ((Rr,), torch.int64), "tally": ((Rr, 2), torch.int32)}
            out = {k: torch.empty(*shapes[k][:1], dtype=shapes[k][1], device=dev) for k in names}
        res = Result(**{k: (v.data_ptr() if v is not None else None) for k, v in out.items()})
        dt = (1.0 / steps if steps > 0 else 1.0) if dt is None else dt
        _check(lib().hqa_run(self._h, C.byref(sched), float(dt), int(steps), R, int(seed),
                             C.byref(opts), C.byref(res), _stream_ptr(stream)), "hqa_run")
        del keep
        return out

    def local_field(self, phi, precision=PREC_FP32, replicas_per_block=0, kernel=KERNEL_AUTO,
                    stream=None):
        import torch
        R = phi.shape[0]
        L = torch.empty_like(phi)
        opts = RunOpts()
        lib().hqa_run_opts_default(C.byref(opts))
        opts.precision = precision
        opts.replicas_per_block = replicas_per_block
        opts.kernel = kernel
        _check(lib().hqa_local_field(self._h, R, _ptr(phi), _ptr(L), C.byref(opts),
                                     _stream_ptr(stream)), "hqa_local_field")
        return L

    def readout(self, phibar, n, stream=None):
        import torch
        R, N = phibar.shape
        spins = torch.empty((R, N), dtype=torch.int8, device=phibar.device)
        frozen = torch.empty((R, N), dtype=torch.uint8, device=phibar.device)
        tally = torch.empty((R, 2), dtype=torch.int32, device=phibar.device)
        _check(lib().hqa_readout(self._h, R, _ptr(phibar), int(n), _ptr(spins), _ptr(frozen),
                                 _ptr(tally), _stream_ptr(stream)), "hqa_readout")
        return spins, frozen, tally

    def energy(self, spins, stream=None, out=None):
        import torch
        R = spins.shape[0]
        if out is None:
            out = (torch.empty(R, dtype=torch.int64, device=spins.device),
                   torch.empty(R, dtype=torch.int64, device=spins.device))
        e, c = out
        _check(lib().hqa_energy(self._h, R, _ptr(spins), _ptr(e), _ptr(c), _stream_ptr(stream)),
               "hqa_energy")
        return e, c

    def trace(self, steps, replicas, stride, seed=0, sched=None, dt=None, precision=PREC_FP32,
              kernel=KERNEL_AUTO, stream=None):
        """hqa_run_trace: (phibar snapshots [T][R][N], final phi [R][N], final p [R][N])."""
        import torch
        R, N = int(replicas), self.N
        sched = sched if sched is not None else schedule()
        opts = RunOpts()
        lib().hqa_run_opts_default(C.byref(opts))
        opts.precision = precision
        opts.kernel = kernel
        T = (int(steps) + int(stride) - 1) // int(stride)
        dev = torch.device("cuda")
        tr = torch.empty((T, R, N), dtype=torch.float32, device=dev)
        phi = torch.empty((R, N), dtype=torch.float32, device=dev)
        p = torch.empty((R, N), dtype=torch.float32, device=dev)
        dt = (1.0 / steps) if dt is None else dt
        _check(lib().hqa_run_trace(self._h, C.byref(sched), float(dt), int(steps), int(stride), R,
                                   int(seed), C.byref(opts), _ptr(tr), _ptr(phi), _ptr(p),
                                   _stream_ptr(stream)), "hqa_run_trace")
        return tr, phi, p

    def energy_f64(self, spins, stream=None):
        """hqa_energy_f64: FP64 Ising energies [R] for any real couplings and field."""
        import torch
        R = spins.shape[0]
        e = torch.empty(R, dtype=torch.float64, device=spins.device)
        _check(lib().hqa_energy_f64(self._h, R, _ptr(spins), _ptr(e), _stream_ptr(stream)),
               "hqa_energy_f64")
        return e

    def solve_sub(self, spins, frozen, n, stream=None, out=None):
        import torch
        R = spins.shape[0]
        if out is None:
            out = (torch.empty_like(spins), torch.empty(R, dtype=torch.int64, device=spins.device))
        out, e = out
        _check(lib().hqa_solve_sub(self._h, R, _ptr(spins), _ptr(frozen), int(n), _ptr(out),
                                   _ptr(e), _stream_ptr(stream)), "hqa_solve_sub")
        return out, e

    def arm_wait_check(self, flag, step, limit_ns):
        """hqa_arm_wait_check: the next dense MD launch waits for flag[0] != 0 before `step`."""
        _check(lib().hqa_arm_wait_check(self._h, _ptr(flag), int(step), int(limit_ns)),
               "hqa_arm_wait_check")

    def solve_sub_tabu(self, spins, frozen, n, iters, tenure, stream=None):
        """hqa_solve_sub_tabu: (spins [R][N], full energies [R]) of the tabu search."""
        import torch
        R = spins.shape[0]
        out = torch.empty_like(spins)
        e = torch.empty(R, dtype=torch.int64, device=spins.device)
        _check(lib().hqa_solve_sub_tabu(self._h, R, _ptr(spins), _ptr(frozen), int(n), int(iters),
                                        int(tenure), _ptr(out), _ptr(e), _stream_ptr(stream)),
               "hqa_solve_sub_tabu")
        return out, e

    def solve_sub_noalloc(self, spins, frozen, n, out_spins, out_energy=None, stream=None):
        """hqa_solve_sub_noalloc: the sub-solve with the library's fixed scratch array,
        for callers that cannot let the library allocate device memory.  The caller
        passes the output buffers; nothing is allocated here or in the library.
        The library writes R*N int8 spins and R int64 energies through the raw
        pointers, so every buffer is checked first: spins and out_spins int8 (R, N),
        frozen uint8 (R, N), out_energy None or int64 (R,), all contiguous and on one
        CUDA device (ValueError otherwise)."""
        import torch
        if spins.dim() != 2 or spins.shape[1] != self.N:
            raise ValueError(f"spins must have shape (R, {self.N})")
        R = spins.shape[0]
        want = [("spins", spins, torch.int8, (R, self.N)),
                ("frozen", frozen, torch.uint8, (R, self.N)),
                ("out_spins", out_spins, torch.int8, (R, self.N))]
        if out_energy is not None:
            want.append(("out_energy", out_energy, torch.int64, (R,)))
        for name, t, dtype, shape in want:
            if not isinstance(t, torch.Tensor):
                raise ValueError(f"{name} must be a torch tensor")
            if t.dtype != dtype or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be {dtype} of shape {shape}, got {t.dtype} "
                                 f"{tuple(t.shape)}")
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
            if t.device.type != "cuda" or t.device != spins.device:
                raise ValueError(f"{name} must be on {spins.device} (a CUDA device)")
        _check(lib().hqa_solve_sub_noalloc(self._h, spins.shape[0], _ptr(spins), _ptr(frozen),
                                           int(n), _ptr(out_spins), _ptr(out_energy),
                                           _stream_ptr(stream)), "hqa_solve_sub_noalloc")
        return out_spins, out_energy

    def plan(self, replicas, precision=PREC_FP32, replicas_per_block=0, kernel=KERNEL_AUTO):
        """hqa_plan_query: the launch plan hqa_run would use, as a dict."""
        opts = RunOpts()
        lib().hqa_run_opts_default(C.byref(opts))
        opts.precision = precision
        opts.replicas_per_block = replicas_per_block
        opts.kernel = kernel
        info = PlanInfo()
        _check(lib().hqa_plan_query(self._h, int(replicas), C.byref(opts), C.byref(info)),
               "hqa_plan_query")
        return {f: getattr(info, f) for f, _ in PlanInfo._fields_}

    def hmd(self, phi, p, tau, sched=None, half_kick=False, precision=PREC_FP32, stream=None):
        """hqa_hmd: H_MD per replica (device float64 [R])."""
        import torch
        sched = sched if sched is not None else schedule()
        opts = RunOpts()
        lib().hqa_run_opts_default(C.byref(opts))
        opts.precision = precision
        R = phi.shape[0]
        out = torch.empty(R, dtype=torch.float64, device=phi.device)
        _check(lib().hqa_hmd(self._h, C.byref(sched), float(tau), R, _ptr(phi), _ptr(p),
                             1 if half_kick else 0, _ptr(out), C.byref(opts),
                             _stream_ptr(stream)), "hqa_hmd")
        return out

    def autotune(self, replicas, precision=PREC_FP32, probe_steps=64, sched=None, stream=None):
        """hqa_autotune: (best opts as a dict, [(kernel, replicas_per_block, ms_per_step)])."""
        sched = sched if sched is not None else schedule()
        opts = RunOpts()
        lib().hqa_run_opts_default(C.byref(opts))
        opts.precision = precision
        best = RunOpts()
        table = (TuneEntry * 32)()
        n = C.c_int32()
        _check(lib().hqa_autotune(self._h, C.byref(sched), int(replicas), C.byref(opts),
                                  int(probe_steps), C.byref(best), table, 32, C.byref(n),
                                  _stream_ptr(stream)), "hqa_autotune")
        rows = [(table[i].kernel, table[i].replicas_per_block, table[i].ms_per_step)
                for i in range(min(n.value, 32))]
        return {"kernel": best.kernel, "replicas_per_block": best.replicas_per_block,
                "precision": best.precision}, rows

    def features(self, steps, replicas, seed=0, sched=None, dt=None, segments=10,
                 precision=PREC_FP32, replicas_per_block=0, kernel=KERNEL_AUTO, stream=None):
        """hqa_run_features: ([R*N, 6] features, phi [R][N], p [R][N]) after `steps` steps."""
        import torch
        R, N = int(replicas), self.N
        sched = sched if sched is not None else schedule()
        opts = RunOpts()
        lib().hqa_run_opts_default(C.byref(opts))
        opts.precision = precision
        opts.replicas_per_block = replicas_per_block
        opts.kernel = kernel
        dev = torch.device("cuda")
        feat = torch.empty((R * N, MLP_IN), dtype=torch.float32, device=dev)
        phi = torch.empty((R, N), dtype=torch.float32, device=dev)
        p = torch.empty((R, N), dtype=torch.float32, device=dev)
        _check(lib().hqa_run_features(self._h, C.byref(sched), float(dt), int(steps), int(segments),
                                      R, int(seed), C.byref(opts), _ptr(feat), _ptr(phi), _ptr(p),
                                      _stream_ptr(stream)), "hqa_run_features")
        return feat, phi, p

    def surrogate_readout(self, logits, replicas, n, max_expected_errors=1.0, stream=None):
        """hqa_surrogate_readout: spins, frozen, accept [R] (uint8), expected errors [R]."""
        import torch
        R, N = int(replicas), self.N
        dev = logits.device
        spins = torch.empty((R, N), dtype=torch.int8, device=dev)
        frozen = torch.empty((R, N), dtype=torch.uint8, device=dev)
        acc = torch.empty(R, dtype=torch.uint8, device=dev)
        err = torch.empty(R, dtype=torch.float32, device=dev)
        _check(lib().hqa_surrogate_readout(self._h, R, _ptr(logits), int(n), float(max_expected_errors),
                                           _ptr(spins), _ptr(frozen), _ptr(acc), _ptr(err),
                                           _stream_ptr(stream)), "hqa_surrogate_readout")
        return spins, frozen, acc, err

    def sync(self, stream=None):
        _check(lib().hqa_sync(self._h, _stream_ptr(stream)), "hqa_sync (latched device status)")

    def close(self):
        if self._h:
            lib().hqa_destroy(self._h)
            self._h = None
        self.members = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """hqa_mlp: the surrogate gate's network (device parameters, AdamW state)."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (MLP_PARAMS,):
            raise ValueError(f"need {MLP_PARAMS} parameters")
        self._h = C.c_void_p()
        _check(lib().hqa_mlp_create(p.ctypes.data, C.byref(self._h)), "hqa_mlp_create")

    @staticmethod
    def init_params(seed=0):
        """He-style random initial parameters (host)."""
        rng = np.random.default_rng(seed)
        parts = [rng.normal(scale=np.sqrt(2 / MLP_IN), size=MLP_HIDDEN * MLP_IN), np.zeros(MLP_HIDDEN),
                 rng.normal(scale=np.sqrt(2 / MLP_HIDDEN), size=MLP_HIDDEN * MLP_HIDDEN),
                 np.zeros(MLP_HIDDEN),
                 rng.normal(scale=np.sqrt(1 / MLP_HIDDEN), size=MLP_OUT * MLP_HIDDEN), np.zeros(MLP_OUT)]
        return np.concatenate(parts).astype(np.float32)

    def params(self):
        out = np.empty(MLP_PARAMS, np.float32)
        _check(lib().hqa_mlp_params(self._h, out.ctypes.data), "hqa_mlp_params")
        return out

    def forward(self, x, precision=PREC_FP32, stream=None):
        import torch
        z = torch.empty((x.shape[0], MLP_OUT), dtype=torch.float32, device=x.device)
        _check(lib().hqa_mlp_forward(self._h, x.shape[0], _ptr(x), _ptr(z), precision,
                                     _stream_ptr(stream)), "hqa_mlp_forward")
        return z

    def grad(self, x, y, precision=PREC_FP32, stream=None):
        import torch
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(lib().hqa_mlp_grad(self._h, x.shape[0], _ptr(x), _ptr(y), _ptr(g), _ptr(loss),
                                  precision, _stream_ptr(stream)), "hqa_mlp_grad")
        return g, loss

    def adamw(self, g, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
        _check(lib().hqa_mlp_adamw(self._h, _ptr(g), lr, beta1, beta2, eps, weight_decay,
                                   _stream_ptr(stream)), "hqa_mlp_adamw")

    def close(self):
        if self._h:
            lib().hqa_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured sequence of library calls (hqa_capture_end); launch() replays it."""

    def __init__(self, handle):
        self._h = handle

    def launch(self, stream=None):
        _check(lib().hqa_graph_launch(self._h, _stream_ptr(stream)), "hqa_graph_launch")

    def close(self):
        if self._h:
            lib().hqa_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class capture:
    """Context manager: library calls made inside the block on ``stream`` (a
    torch.cuda.Stream, passed explicitly to every call, with caller-allocated
    outputs) are captured; ``.graph`` holds the Graph afterwards.  Each call must
    have been made once before without capture (hqa_capture_begin)."""

    def __init__(self, stream):
        self.stream = stream
        self.graph = None

    def __enter__(self):
        _check(lib().hqa_capture_begin(_stream_ptr(self.stream)), "hqa_capture_begin")
        return self

    def __exit__(self, et, ev, tb):
        h = C.c_void_p()
        st = lib().hqa_capture_end(_stream_ptr(self.stream), C.byref(h))
        if et is None:
            _check(st, "hqa_capture_end")
            self.graph = Graph(h)
        elif h:
            lib().hqa_graph_destroy(h)
        return False
