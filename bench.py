#!/usr/bin/env python3
"""HQA-MD benchmark: flux-MD spin-updates/s on one GB300.

With no --config, the line's headline is the largest single-GPU workload, the
paper's MAX-CUT shape (Results, "HQA for MAX-CUT"; Methods, "MAX-CUT and Ising
spin-glass"): SK / K2000 with +-1 weights, 4096 replicas, 10000 leapfrog steps
of the paper's schedule.  The same JSON line carries, under "nested", the
sparse ER workload and the uneven batch, each with its own roofline, CPU
baseline and end-to-end figure.

Workloads (--config):
  sk2000  K2000 +-1 dense, 4096 replicas, 10000 steps, dense GEMM field.
          Variants: plain FP32 (CUDA-core GEMM, the reference form), FP16X2
          (tcgen05, phi split into two FP16 halves, ~22 significant bits),
          FP16 and BF16 (tcgen05, one 16-bit operand; stated errors).
  er800   Erdos-Renyi G(800, 0.06) +-1 CSR, 1024 replicas, 5000 steps, under
          both initial conditions (phi(0) = 0 and seeded random fluxes).
          Variants: plain FP32 and BF16 operand on the resident sparse kernel.
  uneven512  512 instances of uneven size in one persistent batch launch,
          FP32 and BF16, and the same 512 instances run one at a time (FP32).
  sg2000, sg10000  uniform spin glass on the dense paths (quality: FP64 energy).
  sk100   SK N = 100, 1 replica, 1000 steps, linear-Gamma schedule (latency).
  all     (default) sk2000 with er800 and uneven512 nested.
One bench "step" is the whole pipeline over all replicas: MD, readout, int64
energy/cut and the exact sub-solve of the n least-frozen spins (the batch ends
at readout and energy; real couplings at the FP64 energy).
Spin-updates per step = N * R * S (one leapfrog step of one spin in one replica).

The headline variant is the fastest whose 100-step state parity meets the
contract (1e-2 of the FP64 oracle for low precision) and whose median cut is
not worse than the plain FP32 variant's (the 95% bootstrap interval of the
median difference reaches 0); every variant is reported under "variants".

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores over a bounded sample of the same workload (the paper has no code).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "flux-MD spin-updates/s on 1 GB300, mixed/batched vs plain FP32 at equal cut"

# Variant: (name, precision, kernel (None = library's choice / autotuner), init, plain).
# "parity" is the largest state error after 100 steps measured against the FP64
# oracle at this workload's size (tests/test_gpu_dense.py, tests/test_gpu_md.py),
# "contract" whether it meets the bound for its arithmetic.
CONFIGS = {
    "sk2000": dict(
        desc="SK K2000 +-1 dense, 4096 replicas, 10000 steps, paper schedule, n=24 exact "
             "sub-solve, dense GEMM field",
        R=4096, S=10000, n=24, kind="dense", sched="paper",
        variants=(("fp16x2", "PREC_FP16X2", "KERNEL_DENSE", "INIT_PAPER", "fp32"),
                  ("fp16", "PREC_FP16", "KERNEL_DENSE", "INIT_PAPER", "fp32"),
                  ("bf16", "PREC_BF16", "KERNEL_DENSE", "INIT_PAPER", "fp32"),
                  ("fp32", "PREC_FP32", "KERNEL_DENSE", "INIT_PAPER", "fp32")),
        parity={"fp32": (2.2e-5, True), "fp16x2": (1.2e-4, True), "fp16": (7.8e-3, False),
                "bf16": (8.4e-2, False)},
        cpu_steps=100, cpu_scale=1, tabu=dict(n=1000, iters=10000, tenure=20, replicas=512)),
    "er800": dict(
        desc="ER G(800,0.06) +-1 CSR, 1024 replicas, 5000 steps, paper schedule, n=24 exact "
             "sub-solve",
        R=1024, S=5000, n=24, kind="sparse", sched="paper",
        variants=(("fp32", "PREC_FP32", None, "INIT_PAPER", "fp32"),
                  ("bf16", "PREC_BF16", None, "INIT_PAPER", "fp32"),
                  ("fp32_random_flux", "PREC_FP32", None, "INIT_RANDOM_FLUX", "fp32_random_flux"),
                  ("bf16_random_flux", "PREC_BF16", None, "INIT_RANDOM_FLUX", "fp32_random_flux")),
        parity={"fp32": (1e-5, True), "bf16": (1e-2, True), "fp32_random_flux": (1e-5, True),
                "bf16_random_flux": (1e-2, True)},
        cpu_steps=None, cpu_scale=16),
    "uneven512": dict(
        desc="512 instances, N uniform in [200,5000], half random 3-regular, half 2-D tori, +-1, "
             "64 replicas each, 5000 steps, one persistent batch launch",
        R=64, S=5000, n=24, kind="batch", sched="paper",
        variants=(("fp32", "PREC_FP32", None, "INIT_PAPER", "fp32"),
                  ("bf16", "PREC_BF16", None, "INIT_PAPER", "fp32"),
                  ("fp32_one_at_a_time", "PREC_FP32", None, "INIT_PAPER", "fp32")),
        parity={"fp32": (1e-5, True), "bf16": (1e-2, True), "fp32_one_at_a_time": (1e-5, True)},
        cpu_steps=200, cpu_scale=1),
    "sg2000": dict(
        desc="uniform spin glass N=2000 (J ~ U[-1,1] fully connected, h ~ U[-2,2]), 4096 "
             "replicas, 10000 steps, paper schedule, dense GEMM field; quality = FP64 Ising "
             "energy of the readout (no sub-solve: real couplings)",
        R=4096, S=10000, n=24, kind="dense_sg", sched="paper",
        variants=(("fp32", "PREC_FP32", "KERNEL_DENSE", "INIT_PAPER", "fp32"),
                  ("fp16x2", "PREC_FP16X2", "KERNEL_DENSE", "INIT_PAPER", "fp32"),
                  ("fp16", "PREC_FP16", "KERNEL_DENSE", "INIT_PAPER", "fp32"),
                  ("bf16", "PREC_BF16", "KERNEL_DENSE", "INIT_PAPER", "fp32")),
        parity={"fp32": (1.2e-5, True), "fp16x2": (2.7e-4, True), "fp16": (2.3e-2, False),
                "bf16": (1.3e-1, False)},
        cpu_steps=100, cpu_scale=1),
    "sg10000": dict(
        desc="uniform spin glass N=10000 (J ~ U[-1,1] fully connected, h ~ U[-2,2]), 1024 "
             "replicas, 2000 steps, paper schedule, dense GEMM field; quality = FP64 Ising "
             "energy of the readout (no sub-solve: real couplings)",
        R=1024, S=2000, n=24, kind="dense_sg", sched="paper",
        variants=(("bf16x2", "PREC_BF16X2", "KERNEL_DENSE", "INIT_PAPER", "bf16x2"),
                  ("fp16x2", "PREC_FP16X2", "KERNEL_DENSE", "INIT_PAPER", "bf16x2"),
                  ("bf16", "PREC_BF16", "KERNEL_DENSE", "INIT_PAPER", "bf16x2")),
        parity={"bf16x2": (3.5e-3, True), "fp16x2": (3.5e-3, True), "bf16": (2.5e-2, False)},
        cpu_steps=20, cpu_scale=1),
    "sk100": dict(
        desc="SK N=100 +-1, 1 replica, 1000 steps, linear-gamma schedule, n=20 exact sub-solve",
        R=1, S=1000, n=20, kind="sparse", sched="linear_gamma",
        variants=(("fp32", "PREC_FP32", None, "INIT_PAPER", "fp32"),),
        parity={"fp32": (1e-5, True)}, cpu_steps=None, cpu_scale=1),
}
# Surrogate-gated HQA on sparse ER graphs (mean degree 8, +-1): plain FP32, BF16 and
# the gated form (BF16 MD operand, BF16 network) at several prefix fractions and
# gate thresholds, each size its own equal-cut comparison against plain FP32.
SURROGATE = dict(
    desc="surrogate-gated HQA: ER mean degree 8 +-1, N in {1000,2000,5000,10000,20000}, 256 "
         "replicas, 10000 steps, paper schedule, n=24 exact sub-solve; BF16 MLP 6-64-64-2 on "
         "features of the trajectory prefix (10 samples), trained on four other instances",
    sizes=(1000, 2000, 5000, 10000, 20000), R=256, S=10000, n=24, fracs=(0.1, 0.3, 0.5),
    train_sizes=(1000, 1500, 2000, 2500), train_R=64, cpu_steps=200)
NESTED = ("er800", "uneven512", "er_surrogate")
DTYPE = {"PREC_FP32": "f32", "PREC_BF16": "bf16-operand/f32-accumulate",
         "PREC_BF16X2": "bf16x2-split-operand/f32-accumulate",
         "PREC_FP16": "fp16-operand/f32-accumulate",
         "PREC_FP16X2": "fp16x2-split-operand/f32-accumulate"}
ELEM_BYTES = {"PREC_FP32": 4, "PREC_BF16": 2}


def make_instance(name):
    from paper_2004_03972_gb300 import instances
    if name == "er800":
        return instances.er_pm1(800, 0.06, 1200)
    if name == "sk2000":
        return instances.sk_pm1(2000, 1300)
    if name == "sk100":
        return instances.sk_pm1(100, 1100)
    if name == "sg2000":
        return instances.uniform_sg(2000, 1350)
    if name == "sg10000":
        return instances.uniform_sg(10000, 1360)
    if name == "uneven512":
        return instances.uneven_batch(512, 200, 5000, 1400)
    raise KeyError(name)


def shard_seed(rank):
    """Stream seed of one rank's replicas: ranks run disjoint, independent shards."""
    return 1000 + rank * 100003


def reduce_max(values, ws):
    """Per-rank totals -> their maximum over ranks (gloo or NCCL all-reduce)."""
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def whole_job_rate(units_per_rank_step, steps, ws, total_time):
    """Units processed by all ranks / the slowest rank's time."""
    return units_per_rank_step * steps * ws / total_time


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        time.sleep(0.25)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def measured_peaks():
    """Peaks from the driver's measurement: bf16 burst (a kernel timed on its own) and
    sustained (a seconds-long loop), HBM copy bandwidth; the fallback figures otherwise."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"bf16_burst": float(d.get("bf16_tflops")),
                "bf16_sustained": float(d.get("bf16_tflops_sustained") or d.get("bf16_tflops")),
                "hbm_gbs": d.get("hbm_gbs"), "source": "of measured"}
    return {"bf16_burst": 1900.0, "bf16_sustained": 1700.0, "hbm_gbs": 6800.0,
            "source": "of fallback"}


def smem_peak(hqa, dev_index):
    """Shared-memory bandwidth peak (GB/s) from the library's own microbenchmark,
    measured on this GPU now (MEASURED_PEAKS.json has no shared-memory figure)."""
    try:
        return hqa.smem_bandwidth_probe(), "measured: hqa_probe_smem_bandwidth (128-bit ld.shared)"
    except Exception:
        import torch
        sm = torch.cuda.get_device_properties(dev_index).multi_processor_count
        return sm * 128 * 2070e6 / 1e9, "derived: SMs x 128 B/clk x 2070 MHz (probe unavailable)"


def l2_peak(hqa):
    """L2 read bandwidth (GB/s) from the library's microbenchmark, measured now."""
    try:
        return hqa.l2_bandwidth_probe(), "measured: hqa_probe_l2_bandwidth (16-byte ld.global.cg)"
    except Exception:
        return None, "unmeasured"


def _src_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(kernel_key):
    """DRAM bytes per launch from a committed ncu capture, if the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        tab = json.load(f)
    ent = tab.get(kernel_key)
    if not ent:
        return None
    srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
    shas = ent["source_sha"] if isinstance(ent["source_sha"], list) else [ent["source_sha"]]
    for src, sha in zip(srcs, shas):
        if _src_sha(os.path.join(ROOT, "paper_2004_03972_gb300", "csrc", src)) != sha:
            return None
    return ent["dram_bytes_per_launch"]


def median_diff_ci(a, b, reps=2000, seed=0):
    """Bootstrap 95% interval of median(a) - median(b)."""
    rng = np.random.default_rng(seed)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ma = np.median(rng.choice(a, size=(reps, a.size), replace=True), axis=1)
    mb = np.median(rng.choice(b, size=(reps, b.size), replace=True), axis=1)
    lo, hi = np.percentile(ma - mb, [2.5, 97.5])
    return float(lo), float(hi)


def bootstrap_halfwidth(x, reps=2000, seed=0):
    rng = np.random.default_rng(seed)
    x = np.asarray(x, np.float64)
    meds = np.median(rng.choice(x, size=(reps, x.size), replace=True), axis=1)
    lo, hi = np.percentile(meds, [2.5, 97.5])
    return float(hi - lo) / 2


def kernel_name(hqa, plan, prec_name):
    k = plan["kernel"]
    if k == hqa.KERNEL_DENSE:
        if prec_name == "PREC_FP32":
            return "k_dense_simt<1>"
        kseg = 2 if prec_name.endswith("X2") else 1
        f16 = "true" if prec_name.startswith("PREC_FP16") else "false"
        return f"k_dense_md<{plan['replicas_per_block'] // 2},*,{kseg},*,*,{f16},*,*,*>"
    if k == hqa.KERNEL_STREAM:
        return f"k_sparse_stream<{'true' if prec_name == 'PREC_BF16' else 'false'}>"
    base = "k_sparse_md_vec" if k == hqa.KERNEL_VECTOR else "k_sparse_md"
    return f"{base}<{plan['replicas_per_block']},{'true' if prec_name == 'PREC_BF16' else 'false'}>"


class Timer:
    """CUDA-event times of K calls on the current stream after W untimed warm-ups,
    L2 flushed (a 256 MB write, twice L2) before each timed call, barriers around."""

    def __init__(self, torch, ws, dev):
        self.torch = torch
        self.ws = ws
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def __call__(self, fn, K, W, after=None):
        torch = self.torch
        st = torch.cuda.current_stream()
        for w in range(W):
            fn(-1 - w)
        torch.cuda.synchronize()
        if self.ws > 1:
            torch.distributed.barrier()
        times = []
        for k in range(K):
            self.flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn(k)
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            if after:
                after(k)
        torch.cuda.synchronize()
        if self.ws > 1:
            torch.distributed.barrier()
        return times


def measure(name, args, hqa, torch, timer, dev, ws, rank, headline):
    """One workload: every variant timed, equal-cut test, e2e, roofline, CPU baseline."""
    cfg = dict(CONFIGS[name])
    if args.md_steps:
        cfg["S"] = args.md_steps
    K = args.steps if headline else min(args.steps, 5)
    W = args.warmup if headline else 3
    inst = make_instance(name)
    batch = cfg["kind"] == "batch"
    real = cfg["kind"] == "dense_sg"
    if batch:
        members = [hqa.Context.from_instance(i) for i in inst]
        ctx = hqa.Context.batch(members)
        N, nnz = ctx.N, sum(i.nnz for i in inst)      # N = total spins of the batch
    else:
        ctx = hqa.Context.from_instance(inst)
        N, nnz = inst.N, inst.nnz
    R, S, n = cfg["R"], cfg["S"], cfg["n"]
    count = len(inst) if batch else 1
    sched = hqa.schedule(n_ambivalent=n)
    if cfg["sched"] == "linear_gamma":
        sched.kind = hqa.SCHED_LINEAR_GAMMA
    seed_base = shard_seed(rank)
    RR = R * count   # per-replica results
    out = {k: torch.empty(s, dtype=d, device=dev) for k, s, d in (
        ("phi", (R, N), torch.float32), ("p", (R, N), torch.float32),
        ("phibar", (R, N), torch.float32), ("spins", (R, N), torch.int8),
        ("frozen", (R, N), torch.uint8), ("energy", (RR,), torch.int64),
        ("cut", (RR,), torch.int64), ("tally", (RR, 2), torch.int32))
        if not (real and k in ("energy", "cut"))}
    sub_out = (torch.empty((R, N), dtype=torch.int8, device=dev),
               torch.empty((R,), dtype=torch.int64, device=dev))
    member_out = None
    if batch:   # one-at-a-time baseline: per-member output views of the batch arrays
        member_out = []
        offs = np.cumsum([0] + [i.N for i in inst])
        for k, i in enumerate(inst):
            o = {"phibar": out["phibar"].reshape(-1)[R * offs[k]:R * offs[k + 1]].view(R, i.N),
                 "spins": out["spins"].reshape(-1)[R * offs[k]:R * offs[k + 1]].view(R, i.N),
                 "frozen": out["frozen"].reshape(-1)[R * offs[k]:R * offs[k + 1]].view(R, i.N),
                 "energy": out["energy"][R * k:R * (k + 1)], "cut": out["cut"][R * k:R * (k + 1)],
                 "tally": out["tally"][R * k:R * (k + 1)]}
            member_out.append(o)

    def seed_of(k):
        return seed_base + 1000 + k if k >= 0 else seed_base - k

    # the one-at-a-time baseline runs every 8th member (a bounded sample of the batch)
    sample = list(range(0, count, 8)) if batch else []

    def pipeline(v, seed, st=None):
        if v["one_at_a_time"]:
            C = 0x632BE59BD9B4E019
            for k in sample:
                members[k].run(S, R, seed=(seed + (k + 1) * C) % (1 << 64), sched=sched,
                               precision=v["prec"], out=member_out[k], stream=st)
            return None
        ctx.run(S, R, seed=seed, sched=sched, precision=v["prec"], kernel=v["kernel"],
                init=v["init"], out=out, stream=st)
        if real:
            return ctx.energy_f64(out["spins"], stream=st)
        if batch:
            return None   # the batch pipeline ends at readout + energy (no batched sub-solve)
        return ctx.solve_sub(out["spins"], out["frozen"], n, stream=st, out=sub_out)

    variants = {}
    for vname, prec_name, kern_name, init_name, plain_name in cfg["variants"]:
        v = dict(prec=getattr(hqa, prec_name), prec_name=prec_name, plain=plain_name,
                 kernel=getattr(hqa, kern_name) if kern_name else hqa.KERNEL_AUTO,
                 init=getattr(hqa, init_name), one_at_a_time=vname.endswith("one_at_a_time"))
        tuned = None
        if kern_name is None and not v["one_at_a_time"] and not args.no_tune:
            # launch shape (kernel, replicas per block) by the library's autotuner
            best, rows = ctx.autotune(R, precision=v["prec"],
                                      probe_steps=64 if batch else min(S, 500))
            tuned = {"kernel": best["kernel"], "replicas_per_block": best["replicas_per_block"],
                     "candidates": [[k, rb, round(ms, 6)] for k, rb, ms in rows]}
        slow = prec_name == "PREC_FP32" and (kern_name == "KERNEL_DENSE" or v["one_at_a_time"])
        # the plain dense FP32 form and the one-at-a-time baseline take a few seconds a
        # step: two timed steps; variants outside the parity contract: five
        Kv = min(K, 2) if slow else (K if cfg["parity"][vname][1] else min(K, 5))
        quality = []

        def grab(k, v=v, quality=quality):
            if real:
                quality.append(-ctx.energy_f64(out["spins"]).cpu().numpy())
            elif v["one_at_a_time"]:
                quality.append(out["cut"].cpu().numpy().reshape(count, R)[sample].reshape(-1))
            else:
                quality.append(out["cut"].cpu().numpy().copy())

        t_pipe = timer(lambda k, v=v: pipeline(v, seed_of(k)), Kv, 1 if v["one_at_a_time"] else W,
                       after=grab)
        ctx.sync()
        allq = np.concatenate(quality)
        v["su_step"] = (sum(inst[k].N for k in sample) * R * S if v["one_at_a_time"]
                        else N * R * S)
        v.update(t_pipe=t_pipe, tuned=tuned, quality=quality, steps=Kv,
                 median_cut=float(np.median(allq)), mean_cut=float(np.mean(allq)),
                 cut_ci95_halfwidth=bootstrap_halfwidth(allq))
        variants[vname] = v

    # equal cut against each variant's plain form, on the seeds both ran
    eq = {}
    for vname, v in variants.items():
        p = variants[v["plain"]]
        ks = min(v["steps"], p["steps"])
        a = np.concatenate(v["quality"][:ks])
        if v["one_at_a_time"]:   # against the batch's cuts of the same members and seeds
            b = np.concatenate([q.reshape(count, R)[sample].reshape(-1) for q in p["quality"][:ks]])
        else:
            b = np.concatenate(p["quality"][:ks])
        lo, hi = median_diff_ci(a, b) if vname != v["plain"] else (0.0, 0.0)
        eq[vname] = {"interval": [lo, hi], "holds": hi >= 0.0, "seeds": int(a.size)}
    parity = cfg["parity"]
    main_plain = cfg["variants"][0][4]
    eligible = [k for k in variants if eq[k]["holds"] and parity[k][1]
                and variants[k]["plain"] == main_plain and not variants[k]["one_at_a_time"]]
    head = max(eligible, key=lambda k: variants[k]["su_step"] * variants[k]["steps"]
               / sum(variants[k]["t_pipe"]))
    hv = variants[head]

    # the MD kernel alone (roofline), on the stream it is launched on
    md_out = {"phibar": out["phibar"]}
    t_md = timer(lambda k: ctx.run(S, R, seed=seed_of(k), sched=sched, precision=hv["prec"],
                                   kernel=hv["kernel"], init=hv["init"], out=md_out),
                 min(K, 3), 1)
    # the same step as one CUDA-graph replay (the replay recomputes the whole run
    # from the seeded initial state every time)
    t_graph = None
    if not hv["one_at_a_time"]:
        gs = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(gs):
            pipeline(hv, seed_base, gs)
            gs.synchronize()
            with hqa.capture(gs) as cap:
                pipeline(hv, seed_base, gs)
            t_graph = timer(lambda k: cap.graph.launch(gs), min(K, 3), 1)
            cap.graph.close()
        ctx.sync()

    # end-to-end through the public API with host buffers: H2D of phi(0), p(0)
    # and D2H of the step's results, every step
    pin_p0 = torch.empty((R, N), dtype=torch.float32).pin_memory()
    pin_phi0 = torch.zeros((R, N), dtype=torch.float32).pin_memory()
    g = torch.Generator().manual_seed(rank)
    pin_p0.copy_((torch.randint(0, 2, (R, N), generator=g) * 2 - 1).float())
    host_spins = torch.empty((R, N), dtype=torch.int8).pin_memory()
    host_e = torch.empty((RR,), dtype=torch.int64).pin_memory()
    host_c = torch.empty((RR,), dtype=torch.int64).pin_memory()
    host_f = torch.empty((RR,), dtype=torch.float64).pin_memory()
    d_p0 = torch.empty((R, N), dtype=torch.float32, device=dev)
    d_phi0 = torch.empty((R, N), dtype=torch.float32, device=dev)

    def e2e_step(k):
        d_p0.copy_(pin_p0, non_blocking=True)
        d_phi0.copy_(pin_phi0, non_blocking=True)
        ctx.run(S, R, sched=sched, precision=hv["prec"], kernel=hv["kernel"],
                init=hqa.INIT_GIVEN, phi0=d_phi0, p0=d_p0, out=out)
        if real:
            host_spins.copy_(out["spins"], non_blocking=True)
            host_f.copy_(ctx.energy_f64(out["spins"]), non_blocking=True)
        elif batch:
            host_spins.copy_(out["spins"], non_blocking=True)
            host_e.copy_(out["energy"], non_blocking=True)
            host_c.copy_(out["cut"], non_blocking=True)
        else:
            sub_s, sub_e = ctx.solve_sub(out["spins"], out["frozen"], n, out=sub_out)
            host_spins.copy_(sub_s, non_blocking=True)
            host_e.copy_(sub_e, non_blocking=True)
            host_c.copy_(out["cut"], non_blocking=True)

    K_e = min(K, 5)
    t_e2e = timer(e2e_step, K_e, 3)
    ctx.sync()

    su_step = N * R * S
    tot_pipe, tot_e2e = reduce_max([sum(hv["t_pipe"]), sum(t_e2e)], ws)
    value = whole_job_rate(su_step, hv["steps"], ws, tot_pipe)
    e2e_value = whole_job_rate(su_step, K_e, ws, tot_e2e)

    # roofline of the dominant kernel (the MD kernel)
    if batch:
        rb = hv["tuned"]["replicas_per_block"] if hv["tuned"] else 0
        kb = hv["tuned"]["kernel"] if hv["tuned"] else hqa.KERNEL_AUTO
        plan = {"kernel": kb, "replicas_per_block": rb, "members": count, "chunks": 1,
                "note": "persistent batch kernel and replica blocking picked by the autotuner"}
        base = {hqa.KERNEL_LOWDEG: "k_batch_lowdeg", hqa.KERNEL_SCALAR: "k_sparse_md_batch"}.get(
            kb, "k_batch_lowdeg|k_sparse_md_batch")
        kname = f"{base}<{rb or '*'},{'true' if hv['prec_name'] == 'PREC_BF16' else 'false'}>"
    else:
        plan = ctx.plan(R, precision=hv["prec"], kernel=hv["kernel"])
        kname = kernel_name(hqa, plan, hv["prec_name"])
    chunks = plan.get("chunks", 1) or 1
    t_run = float(np.mean(t_md))
    if cfg["kind"] in ("dense", "dense_sg"):
        pk = measured_peaks()
        kseg = 1
        if hv["prec_name"].endswith("X2"):
            kseg = 3 if real else 2
        flops = 2.0 * N * N * R * S / chunks            # algorithmic per launch: the field GEMM
        t_launch = t_run / chunks
        achieved = flops / t_launch / 1e12
        if hv["prec_name"] == "PREC_FP32":
            sm = torch.cuda.get_device_properties(dev).multi_processor_count
            peak = sm * 128 * 2 * 2070e6 / 1e12           # FP32 FMA lanes x 2 flop x max clock
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": "derived: SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
        else:
            # the kernel is timed on its own: the burst peak; a split operand issues
            # kseg MMA passes for each algorithmic flop
            roof = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_burst"],
                    "unit": "TFLOP/s", "frac": achieved / pk["bf16_burst"],
                    "issued_tflops": achieved * kseg,
                    "issued_frac": achieved * kseg / pk["bf16_burst"], "k_segments": kseg,
                    "peak_source": f"bf16 burst {pk['source']} (fp16 has the same dense rate)"}
    else:
        es = ELEM_BYTES[hv["prec_name"]]
        bytes_per_launch = nnz * es * R * S   # gathered operand bytes: deg x elem size per spin-update
        t_launch = t_run
        achieved = bytes_per_launch / t_launch / 1e9
        peak, src = smem_peak(hqa, dev.index if dev.index is not None else 0)
        roof = {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": src}
    roof["traffic"] = ncu_traffic(f"{kname}@{name}")
    roof["kernel"] = kname
    roof["launch_ms"] = 1e3 * t_launch
    roof["launches_per_run"] = chunks
    roof["plan"] = plan

    tabu = None
    if cfg.get("tabu") and not real:
        # large-n sub-solve (the paper's HQA(TS1000) shape): tabu search on the n least
        # frozen spins of the headline variant's readout, timed on its own
        tb = cfg["tabu"]
        Rt = tb["replicas"]
        o2 = ctx.run(S, Rt, seed=seed_base, sched=hqa.schedule(n_ambivalent=tb["n"]),
                     precision=hv["prec"], kernel=hv["kernel"],
                     outputs=("phibar", "spins", "frozen", "energy"))
        ts = timer(lambda k: ctx.solve_sub_tabu(o2["spins"], o2["frozen"], tb["n"], tb["iters"],
                                                tb["tenure"]), 3, 1)
        _, te = ctx.solve_sub_tabu(o2["spins"], o2["frozen"], tb["n"], tb["iters"], tb["tenure"])
        gain = (o2["energy"] - te).double()
        tabu = {"n": tb["n"], "iters": tb["iters"], "tenure": tb["tenure"], "replicas": Rt,
                "ms": 1e3 * float(np.median(ts)),
                "flips_per_s": Rt * tb["iters"] / float(np.median(ts)),
                "median_energy_gain_over_readout": float(gain.median())}
    cpu = cpu_baseline(args, inst, cfg) if (rank == 0 and not args.skip_cpu) else None
    launches = launches_per_step(hqa, plan, hv, cfg, S, batch, real, count)
    rec = {
        "value": value, "unit": "spin-updates/s", "steps": hv["steps"],
        "warmup": W, "ms_per_step": 1e3 * tot_pipe / hv["steps"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[hv["prec_name"]],
        "config": {"workload": cfg["desc"] if S == CONFIGS[name]["S"] else
                   cfg["desc"] + f" (shortened to {S} steps)", "name": name, "N": N,
                   "nnz": nnz, "replicas": R, "md_steps": S, "instances": count,
                   "n_ambivalent": n, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas only, {ws} GPU(s)"},
        "variants": {k: {"spin_updates_per_s": v["su_step"] * v["steps"] / sum(v["t_pipe"]),
                         "steps": v["steps"], "ms_per_step": 1e3 * float(np.mean(v["t_pipe"])),
                         "dtype": DTYPE[v["prec_name"]], "autotuned": v["tuned"],
                         "median_cut": v["median_cut"], "cut_ci95_halfwidth": v["cut_ci95_halfwidth"],
                         "mean_cut": v["mean_cut"], "equal_cut_vs_plain": eq[k],
                         "plain": v["plain"],
                         "state_error_100_steps": parity[k][0], "parity_contract": parity[k][1],
                         **({"sample": f"every 8th member ({len(sample)} of {count}), each its "
                                       "own hqa_run; 1 warm-up"} if v["one_at_a_time"] else {})}
                     for k, v in variants.items()},
        "headline_variant": head,
        "equal_cut": {"rule": "95% bootstrap interval of median(variant cut) - median(plain cut) "
                              "reaches 0", "quality": "minus FP64 Ising energy" if real else
                              "readout cut (before the sub-solve)"},
        "graph_replay_spin_updates_per_s":
            su_step * len(t_graph) / sum(t_graph) if t_graph else None,
        "e2e": {"value": e2e_value, "unit": "spin-updates/s", "steps": K_e,
                "h2d_bytes_per_step": 2 * R * N * 4,
                "d2h_bytes_per_step": R * N + (1 if real else 2) * RR * 8},
        "gpu_launches": launches * hv["steps"],
        "roofline": roof,
    }
    if cpu:
        rec["cpu_baseline"] = cpu
    if tabu:
        rec["tabu_sub_solve"] = tabu
    ctx.close()
    if batch:
        for m in members:
            m.close()
    return rec


def measure_surrogate(args, hqa, torch, timer, dev, ws, rank):
    """Config of the surrogate gate: per size, plain FP32, BF16 and gated rates at equal
    median cut, with each gated point's prefix fraction, threshold, acceptance and cut loss."""
    from paper_2004_03972_gb300 import instances
    from paper_2004_03972_gb300 import surrogate as SG
    cfg = SURROGATE
    R, S, n = cfg["R"], (args.md_steps or cfg["S"]), cfg["n"]
    K = min(args.steps, 3)
    seed_base = shard_seed(rank)
    sched = hqa.schedule(n_ambivalent=n)
    # one network per prefix fraction, trained on four instances not used below
    nets = {}
    for frac in cfg["fracs"]:
        sc = SG.SurrogateConfig(steps=S, frac=frac, n_ambivalent=n, precision=hqa.PREC_BF16)
        xs, ys = [], []
        for k, Nt in enumerate(cfg["train_sizes"]):
            c = hqa.Context.from_instance(instances.er_mean_degree_pm1(Nt, 8.0, 50 + k))
            x, y = SG.dataset(c, sc, cfg["train_R"], seed=10 + k)
            xs.append(x)
            ys.append(y)
            c.close()
        mlp = hqa.MLP(hqa.MLP.init_params(0))
        hist = SG.train(mlp, xs, ys, epochs=40, precision=hqa.PREC_BF16)
        nets[frac] = (mlp, hist[-1])
    sizes, tot_su, tot_t = {}, 0.0, 0.0
    roof = e2e = cpu = None
    for N in cfg["sizes"]:
        inst = instances.er_mean_degree_pm1(N, 8.0, 1500 + N)
        ctx = hqa.Context.from_instance(inst)
        out = {k: torch.empty(sh, dtype=d, device=dev) for k, sh, d in (
            ("phibar", (R, N), torch.float32), ("spins", (R, N), torch.int8),
            ("frozen", (R, N), torch.uint8), ("energy", (R,), torch.int64),
            ("cut", (R,), torch.int64), ("tally", (R, 2), torch.int32))}
        sub = (torch.empty((R, N), dtype=torch.int8, device=dev),
               torch.empty((R,), dtype=torch.int64, device=dev))
        su = N * R * S
        rec = {}

        def plain(prec, seed):
            ctx.run(S, R, seed=seed, sched=sched, precision=prec, out=out)
            s2, e2 = ctx.solve_sub(out["spins"], out["frozen"], n, out=sub)
            return e2

        twice_c0 = int(round(inst.val.astype(np.float64).sum())) // 2
        for name, prec in (("fp32", hqa.PREC_FP32), ("bf16", hqa.PREC_BF16)):
            ctx.autotune(R, precision=prec, probe_steps=200)
            q = []
            t = timer(lambda k, prec=prec: plain(prec, seed_base + 1000 + k), K, 3,
                      after=lambda k, q=q: q.append(((twice_c0 - sub[1]) // 2).cpu().numpy()))
            rec[name] = {"spin_updates_per_s": su * K / sum(t), "t": t, "q": np.concatenate(q),
                         "qs": q}
        gated = []
        for frac in cfg["fracs"]:
            mlp, loss = nets[frac]
            base_cfg = SG.SurrogateConfig(steps=S, frac=frac, n_ambivalent=n,
                                          precision=hqa.PREC_BF16)
            probe = SG.gated_run(ctx, mlp, base_cfg, R, seed=seed_base)
            loose = float(probe["expected_errors"].float().median())
            # the default threshold (one expected wrong sign) at the specified 10% prefix;
            # at every prefix a loose one that accepts about half of the replicas
            for thr in ((1.0, loose) if frac == cfg["fracs"][0] else (loose,)):
                gc = SG.SurrogateConfig(steps=S, frac=frac, n_ambivalent=n,
                                        precision=hqa.PREC_BF16, max_expected_errors=thr)
                res = []
                Kg = min(K, 2)
                t = timer(lambda k, gc=gc: res.append(SG.gated_run(ctx, mlp, gc, R,
                                                                   seed=seed_base + 1000 + k,
                                                                   score_all=False)),
                          Kg, 1)
                res = res[-Kg:]
                cuts = np.concatenate([g["cut"].cpu().numpy() for g in res])
                acc = np.concatenate([g["accept"].cpu().numpy() for g in res]).astype(bool)
                # the cut each accepted replica lost against its own full BF16 run
                full = [SG.method_run(ctx, base_cfg, R, seed=seed_base + 1000 + k)
                        for k in range(Kg)]
                fcut = np.concatenate([f["cut"].cpu().numpy() for f in full])
                lo, hi = median_diff_ci(cuts, np.concatenate(
                    [q for q in rec["fp32"]["qs"][:Kg]]))
                gated.append({
                    "prefix_fraction": frac, "threshold_expected_errors": thr,
                    "train_loss": loss, "accepted_fraction": float(acc.mean()),
                    "median_cut_loss_of_accepted": float(np.median((fcut - cuts)[acc]))
                    if acc.any() else None,
                    "md_steps_fraction": float(np.mean([g["md_steps"] for g in res])) / (S * R),
                    "median_cut": float(np.median(cuts)),
                    "equal_cut_vs_fp32": {"interval": [lo, hi], "holds": hi >= 0.0},
                    "steps": Kg, "spin_updates_per_s": su * Kg / sum(t)})
        bf = rec["bf16"]
        lo, hi = median_diff_ci(bf["q"], rec["fp32"]["q"])
        cand = [("fp32", sum(rec["fp32"]["t"])), ("bf16", sum(bf["t"]))] if hi >= 0 else \
            [("fp32", sum(rec["fp32"]["t"]))]
        cand += [(f"gated@{g['prefix_fraction']}/{g['threshold_expected_errors']:.3g}",
                  su * K / g["spin_updates_per_s"]) for g in gated if g["equal_cut_vs_fp32"]["holds"]]
        # (a gated point's time is scaled to K steps from its own rate)
        best = min(cand, key=lambda c: c[1])
        tot_su += su * K
        tot_t += best[1]
        sizes[str(N)] = {
            "nnz": inst.nnz,
            "fp32": {"spin_updates_per_s": rec["fp32"]["spin_updates_per_s"],
                     "median_cut": float(np.median(rec["fp32"]["q"]))},
            "bf16": {"spin_updates_per_s": bf["spin_updates_per_s"],
                     "median_cut": float(np.median(bf["q"])),
                     "equal_cut_vs_fp32": {"interval": [lo, hi], "holds": hi >= 0.0}},
            "gated": gated, "best_at_equal_cut": best[0]}
        if N == cfg["sizes"][-1]:
            # roofline and e2e on the largest size, BF16 operand
            plan = ctx.plan(R, precision=hqa.PREC_BF16)
            md_out = {"phibar": out["phibar"]}
            t_md = timer(lambda k: ctx.run(S, R, seed=seed_base + k, sched=sched,
                                           precision=hqa.PREC_BF16, out=md_out), K, 1)
            tl = float(np.mean(t_md))
            streaming = plan["kernel"] == hqa.KERNEL_STREAM
            peak, src = l2_peak(hqa) if streaming else \
                smem_peak(hqa, dev.index if dev.index is not None else 0)
            ach = inst.nnz * 2 * R * S / tl / 1e9
            roof = {"bound": "l2" if streaming else "smem", "achieved": ach, "peak": peak,
                    "unit": "GB/s", "frac": ach / peak if peak else None, "peak_source": src,
                    "traffic": None,
                    "kernel": kernel_name(hqa, plan, "PREC_BF16"), "launch_ms": 1e3 * tl,
                    "plan": plan, "workload": f"ER N={N} mean degree 8, {R} replicas, {S} steps"}
            pin = torch.empty((R, N), dtype=torch.float32).pin_memory()
            pin.copy_((torch.randint(0, 2, (R, N), generator=torch.Generator().manual_seed(3))
                       * 2 - 1).float())
            pz = torch.zeros((R, N), dtype=torch.float32).pin_memory()
            hs = torch.empty((R, N), dtype=torch.int8).pin_memory()
            he = torch.empty((R,), dtype=torch.int64).pin_memory()
            d0 = torch.empty((R, N), dtype=torch.float32, device=dev)
            d1 = torch.empty((R, N), dtype=torch.float32, device=dev)

            def e2e_step(k):
                d0.copy_(pin, non_blocking=True)
                d1.copy_(pz, non_blocking=True)
                ctx.run(S, R, sched=sched, precision=hqa.PREC_BF16, init=hqa.INIT_GIVEN,
                        phi0=d1, p0=d0, out=out)
                s2, e2 = ctx.solve_sub(out["spins"], out["frozen"], n, out=sub)
                hs.copy_(s2, non_blocking=True)
                he.copy_(e2, non_blocking=True)

            te = timer(e2e_step, K, 3)
            e2e = {"value": su * K / sum(te), "unit": "spin-updates/s", "steps": K,
                   "h2d_bytes_per_step": 2 * R * N * 4, "d2h_bytes_per_step": R * N + R * 8,
                   "workload": f"ER N={N}, BF16 operand"}
            if rank == 0 and not args.skip_cpu:
                cores = os.cpu_count() or 1
                wall = _oracle_sample(inst, cfg["cpu_steps"], cores, cores)
                cpu = {"value": N * cores * cfg["cpu_steps"] / wall, "unit": "spin-updates/s",
                       "cores": cores, "kind": "oracle",
                       "sample": f"ER N={N}: {cores} of {R} replicas x {cfg['cpu_steps']} of {S} "
                                 "steps (MD only, FP64, OpenMP over replicas)"}
        ctx.close()
    for mlp, _ in nets.values():
        mlp.close()
    (tot_t,) = reduce_max([tot_t], ws)
    rec = {"value": whole_job_rate(tot_su / K, K, ws, tot_t), "unit": "spin-updates/s",
           "rule": "per size the fastest of FP32, BF16 and the gated points whose median cut "
                   "is not worse than FP32's; value = all sizes' spin-updates / those times",
           "config": {"workload": cfg["desc"], "name": "er_surrogate", "replicas": R,
                      "md_steps": S, "steps": K},
           "sizes": sizes, "roofline": roof, "e2e": e2e}
    if cpu:
        rec["cpu_baseline"] = cpu
    return rec


def launches_per_step(hqa, plan, hv, cfg, S, batch, real, count):
    """Library kernels one pipeline step launches."""
    if hv["one_at_a_time"]:
        return count * 3      # per member: MD, readout, energy
    if plan["kernel"] == hqa.KERNEL_DENSE and hv["prec_name"] == "PREC_FP32":
        md = S + 2            # init, one launch per leapfrog step, output
    elif plan["kernel"] == hqa.KERNEL_DENSE:
        md = 3 * plan.get("chunks", 1)   # init, persistent MD, output per chunk
    else:
        md = 1
    if real:
        return md + 1 + 3     # readout; spin masks, fixed-point sums, rounding
    if batch:
        return md + 2         # readout, energy
    return md + 2 + 6         # readout, energy; sub-solve: prep, packed min/arg, walk, assemble, energy


def _oracle_sample(inst, S, reps, threads):
    from oracle import oracle as orc
    pr = orc.Problem.from_instance(inst)
    N = inst.N
    p0 = np.stack([orc.initial_momenta(9, r, N) for r in range(reps)])
    phi0 = np.zeros_like(p0)
    t0 = time.perf_counter()
    orc.md_run_replicas(pr, S, phi0, p0, threads=threads)
    return time.perf_counter() - t0


def _cpu_sample_shape(cfg, cores, scale):
    S = cfg["cpu_steps"] or cfg["S"]
    reps = max(1, min(cfg["R"], scale * cores))
    return S, reps


def cpu_baseline(args, inst, cfg):
    from oracle import oracle as orc
    orc.build()
    cores = os.cpu_count() or 1
    if cfg["kind"] == "batch":
        # a bounded sample: every 16th member, `cores` replicas, 200 steps
        S = cfg["cpu_steps"]
        su, wall = 0, 0.0
        for m in inst[::16]:
            wall += _oracle_sample(m, S, cores, cores)
            su += m.N * cores * S
        return {"value": su / wall, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{len(inst[::16])} of {len(inst)} members x {cores} of {cfg['R']} "
                          f"replicas x {S} of {cfg['S']} steps (MD only, FP64)"}
    S, reps = _cpu_sample_shape(cfg, cores, cfg.get("cpu_scale", 1))
    wall = _oracle_sample(inst, S, reps, cores)
    return {"value": inst.N * reps * S / wall, "unit": "spin-updates/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{reps} of {cfg['R']} replicas x {S} of {cfg['S']} steps "
                      "(MD only, FP64, OpenMP over replicas)"}


def run_ours(args):
    import torch

    from paper_2004_03972_gb300 import build, hqa
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    timer = Timer(torch, ws, dev)
    head_name = "sk2000" if args.config == "all" else args.config
    nested = NESTED if args.config == "all" else ()
    clocks = ClockSampler(local)
    walls = {}
    with clocks:
        t0 = time.perf_counter()
        if head_name == "er_surrogate":
            line = measure_surrogate(args, hqa, torch, timer, dev, ws, rank)
            line.update(steps=line["config"]["steps"], warmup=3, higher_is_better=True,
                        scaling="weak", vs_baseline=None, dtype="bf16-operand/f32-accumulate",
                        gpu_launches=None)
        else:
            line = measure(head_name, args, hqa, torch, timer, dev, ws, rank, True)
        walls[head_name] = time.perf_counter() - t0
        sub = {}
        for nm in nested:
            t0 = time.perf_counter()
            sub[nm] = (measure_surrogate(args, hqa, torch, timer, dev, ws, rank)
                       if nm == "er_surrogate" else
                       measure(nm, args, hqa, torch, timer, dev, ws, rank, False))
            walls[nm] = time.perf_counter() - t0
            print(f"[bench] {nm}: {walls[nm]:.1f} s", file=sys.stderr, flush=True)
    line["wall_s_per_workload"] = {k: round(v, 1) for k, v in walls.items()}
    line = {"metric": METRIC, **line, "n_gpus": ws,
            "data": "synthetic (seeded instance generator)"}
    line["clocks"] = clocks.summary()
    if sub:
        line["nested"] = sub
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    name = "sk2000" if args.config == "all" else args.config
    cfg = CONFIGS[name]
    inst = make_instance(name)
    cores = os.cpu_count() or 1
    S, reps = _cpu_sample_shape(cfg, cores, 1)
    if cfg["kind"] == "batch":
        inst = inst[len(inst) // 2]     # one mid-size member per step
    for _ in range(args.warmup):
        _oracle_sample(inst, min(S, 5), reps, cores)
    walls = [_oracle_sample(inst, S, reps, cores) for _ in range(args.steps)]
    value = inst.N * reps * S * args.steps / sum(walls)
    sample = f"{reps} of {cfg['R']} replicas x {S} of {cfg['S']} steps per step (MD only, FP64 oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "spin-updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(walls) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded instance generator)",
        "config": {"workload": cfg["desc"], "name": name, "N": inst.N, "replicas": cfg["R"],
                   "md_steps": cfg["S"]},
        "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="all", choices=["all", "er_surrogate"] + sorted(CONFIGS))
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--md-steps", type=int, default=0,
                    help="override the workload's MD step count (shorter runs for profiling)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default launch shapes (profiling: the autotuner's "
                         "timings would see the profiler's replays)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
