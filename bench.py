#!/usr/bin/env python3
"""HQA-MD benchmark: flux-MD spin-updates/s on one GB300.

Workloads (--config):
  er800  (default) Erdos-Renyi G(800, 0.06) with +-1 weights in CSR, 1024
         replicas with seeded +-1 initial momenta, 5000 leapfrog steps of the
         paper's schedule (dt = 1/5000).  Variants: plain FP32 operand and BF16
         operand (FP32 accumulate, FP32 state) on the resident sparse kernel.
  sk2000 SK / K2000 with +-1 weights (dense), 4096 replicas, 10000 steps.
         Variants on the tcgen05 dense kernel: split BF16 operand (hi + lo,
         ~16 significant bits: the FP32-accurate reference variant) and plain
         BF16 operand.
  sg2000, sg10000  uniform spin glass (J ~ U[-1, 1], h ~ U[-2, 2]) at N = 2000
         (4096 replicas, 10000 steps) and N = 10000 (1024 replicas, 2000 steps)
         on the dense kernel; quality is the FP64 energy of the readout.
  uneven512  512 instances of uneven size in one persistent batch launch.
  sk100  SK N = 100, 1 replica, 1000 steps, linear-Gamma schedule (latency).
One bench "step" is the whole pipeline over all replicas: MD, readout,
int64 energy/cut and the exact sub-solve of the n least-frozen spins.
Spin-updates per step = N * R * S (one leapfrog step of one spin in one replica).

The headline value is the fastest variant whose median cut is not worse than
the plain variant's (the 95% bootstrap interval of the median difference
reaches 0); every variant is reported under "variants".

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

CONFIGS = {
    "er800": dict(desc="ER G(800,0.06) +-1 CSR, 1024 replicas, 5000 steps, paper schedule, "
                       "n=24 exact sub-solve",
                  R=1024, S=5000, n=24, kind="sparse", sched="paper",
                  variants=(("fp32", "PREC_FP32"), ("bf16", "PREC_BF16")), plain="fp32",
                  cpu_steps=None),
    "sk2000": dict(desc="SK K2000 +-1 dense, 4096 replicas, 10000 steps, paper schedule, "
                        "n=24 exact sub-solve, tcgen05 field",
                   R=4096, S=10000, n=24, kind="dense", sched="paper",
                   variants=(("bf16x2", "PREC_BF16X2"), ("bf16", "PREC_BF16")), plain="bf16x2",
                   cpu_steps=200, tabu=dict(n=1000, iters=10000, tenure=20, replicas=512)),
    "sg2000": dict(desc="uniform spin glass N=2000 (J ~ U[-1,1] fully connected, h ~ U[-2,2]), "
                        "4096 replicas, 10000 steps, paper schedule, tcgen05 field; quality = "
                        "FP64 Ising energy of the readout (no sub-solve: real couplings)",
                   R=4096, S=10000, n=24, kind="dense_sg", sched="paper",
                   variants=(("bf16x2", "PREC_BF16X2"), ("bf16", "PREC_BF16")), plain="bf16x2",
                   cpu_steps=200),
    "sg10000": dict(desc="uniform spin glass N=10000 (J ~ U[-1,1] fully connected, h ~ U[-2,2]), "
                         "1024 replicas, 2000 steps, paper schedule, tcgen05 field; quality = "
                         "FP64 Ising energy of the readout (no sub-solve: real couplings)",
                    R=1024, S=2000, n=24, kind="dense_sg", sched="paper",
                    variants=(("bf16x2", "PREC_BF16X2"), ("bf16", "PREC_BF16")), plain="bf16x2",
                    cpu_steps=50),
    "uneven512": dict(desc="512 instances, N uniform in [200,5000], half random 3-regular, half "
                           "2-D tori, +-1, 64 replicas each, 5000 steps, one persistent batch launch",
                      R=64, S=5000, n=24, kind="batch", sched="paper",
                      variants=(("fp32", "PREC_FP32"), ("bf16", "PREC_BF16")), plain="fp32",
                      cpu_steps=200),
    "sk100": dict(desc="SK N=100 +-1, 1 replica, 1000 steps, linear-gamma schedule, "
                       "n=20 exact sub-solve",
                  R=1, S=1000, n=20, kind="sparse", sched="linear_gamma",
                  variants=(("fp32", "PREC_FP32"),), plain="fp32", cpu_steps=None),
}

ELEM_BYTES = {"PREC_FP32": 4, "PREC_BF16": 2, "PREC_BF16X2": 4}


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
    """Tensor peak (TFLOP/s) for a seconds-long kernel: the driver's sustained figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        t = d.get("bf16_tflops_sustained") or d.get("bf16_tflops")
        return {"bf16_tflops": float(t), "hbm_gbs": d.get("hbm_gbs"), "source": "of measured"}
    return {"bf16_tflops": 1700.0, "hbm_gbs": 6800.0, "source": "of fallback (sustained)"}


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
    src = os.path.join(ROOT, "paper_2004_03972_gb300", "csrc", ent["source"])
    if _src_sha(src) != ent["source_sha"]:
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
        split = "true" if prec_name == "PREC_BF16X2" else "false"
        return f"k_dense_md<{plan['replicas_per_block'] // 2},*,{split}>"
    base = "k_sparse_md_vec" if k == hqa.KERNEL_VECTOR else "k_sparse_md"
    return f"{base}<{plan['replicas_per_block']},{'true' if prec_name == 'PREC_BF16' else 'false'}>"


def run_ours(args):
    import torch

    from paper_2004_03972_gb300 import build, hqa
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    build.build()
    cfg = dict(CONFIGS[args.config])
    if args.md_steps:
        cfg["S"] = args.md_steps
    inst = make_instance(args.config)
    batch = cfg["kind"] == "batch"
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
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    seed_base = shard_seed(rank)

    RR = R * count   # per-replica results
    real = cfg["kind"] == "dense_sg"   # real couplings: FP64 energy, no integer cut or sub-solve
    out = {k: torch.empty(s, dtype=d, device=dev) for k, s, d in (
        ("phi", (R, N), torch.float32), ("p", (R, N), torch.float32),
        ("phibar", (R, N), torch.float32), ("spins", (R, N), torch.int8),
        ("frozen", (R, N), torch.uint8), ("energy", (RR,), torch.int64),
        ("cut", (RR,), torch.int64), ("tally", (RR, 2), torch.int32))
        if not (real and k in ("energy", "cut"))}

    sub_out = (torch.empty((R, N), dtype=torch.int8, device=dev),
               torch.empty((R,), dtype=torch.int64, device=dev))

    def pipeline(prec, seed, st=None):
        ctx.run(S, R, seed=seed, sched=sched, precision=prec, out=out, stream=st)
        if real:
            return ctx.energy_f64(out["spins"], stream=st)
        if batch:
            return None   # the batch pipeline ends at readout + energy (no batched sub-solve)
        return ctx.solve_sub(out["spins"], out["frozen"], n, stream=st, out=sub_out)

    def timed(fn, K, W):
        """CUDA-event times of K calls on the current stream, L2 flushed before each."""
        st = torch.cuda.current_stream()
        for w in range(W):
            fn(w)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        times = []
        for k in range(K):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn(W + k)
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        return times

    variants = {}
    clocks = ClockSampler(local)
    with clocks:
        for name, prec_name in cfg["variants"]:
            prec = getattr(hqa, prec_name)
            tuned = None
            if cfg["kind"] not in ("dense", "dense_sg") and not args.no_tune:
                # launch shape (kernel, replicas per block) by the library's autotuner
                best, rows = ctx.autotune(R, precision=prec, probe_steps=64 if batch else min(S, 500))
                tuned = {"kernel": best["kernel"], "replicas_per_block": best["replicas_per_block"],
                         "candidates": [[k, rb, round(ms, 6)] for k, rb, ms in rows]}
            t_pipe = timed(lambda k, prec=prec: pipeline(prec, seed_base + k), args.steps, args.warmup)
            ctx.sync()
            # quality: MD readout cuts over the same seeds for every variant
            cuts = []
            for k in range(args.steps):
                ctx.run(S, R, seed=seed_base + 7 * k, sched=sched, precision=prec, out=out)
                if real:   # quality: minus the FP64 energy (higher is better, like a cut)
                    cuts.append(-ctx.energy_f64(out["spins"]).cpu().numpy())
                else:
                    cuts.append(out["cut"].cpu().numpy().copy())
            ctx.sync()
            allcuts = np.concatenate(cuts)
            md_out = {"phibar": out["phibar"]}   # MD kernel alone (roofline timing)
            t_md = timed(lambda k, prec=prec: ctx.run(S, R, seed=seed_base + k, sched=sched,
                                                      precision=prec, out=md_out), args.steps, 1)
            t_graph = None
            if cfg["kind"] not in ("dense", "dense_sg"):
                # the same step as one CUDA-graph replay (fixed seed: the replay recomputes
                # the whole run from the seeded initial state every time)
                gs = torch.cuda.Stream(device=dev)
                with torch.cuda.stream(gs):
                    pipeline(prec, seed_base, gs)
                    gs.synchronize()
                    with hqa.capture(gs) as cap:
                        pipeline(prec, seed_base, gs)
                    t_graph = timed(lambda k: cap.graph.launch(gs), args.steps, args.warmup)
                    cap.graph.close()
                ctx.sync()
            variants[name] = dict(prec=prec, prec_name=prec_name, t_pipe=t_pipe, t_md=t_md,
                                  t_graph=t_graph, tuned=tuned,
                                  cuts=allcuts, median_cut=float(np.median(allcuts)),
                                  cut_ci95_halfwidth=bootstrap_halfwidth(allcuts),
                                  mean_cut=float(np.mean(allcuts)))
        # headline: fastest variant at equal cut with the plain one
        plain = variants[cfg["plain"]]
        eq = {}
        for name, v in variants.items():
            lo, hi = median_diff_ci(v["cuts"], plain["cuts"]) if name != cfg["plain"] else (0.0, 0.0)
            eq[name] = {"interval": [lo, hi], "holds": hi >= 0.0}
        head = min((k for k in variants if eq[k]["holds"]),
                   key=lambda k: np.mean(variants[k]["t_pipe"]))
        best_prec = variants[head]["prec"]
        # end-to-end through the public API with host buffers
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
            if real:
                d_p0.copy_(pin_p0, non_blocking=True)
                d_phi0.copy_(pin_phi0, non_blocking=True)
                ctx.run(S, R, sched=sched, precision=best_prec, init=hqa.INIT_GIVEN, phi0=d_phi0,
                        p0=d_p0, out=out)
                e = ctx.energy_f64(out["spins"])
                host_spins.copy_(out["spins"], non_blocking=True)
                host_f.copy_(e, non_blocking=True)
                return
            if batch:   # initial state in the batch layout ([R][N_k] blocks of every member)
                d_p0.copy_(pin_p0, non_blocking=True)
                d_phi0.copy_(pin_phi0, non_blocking=True)
                ctx.run(S, R, sched=sched, precision=best_prec, init=hqa.INIT_GIVEN, phi0=d_phi0,
                        p0=d_p0, out=out)
                host_spins.copy_(out["spins"], non_blocking=True)
                host_e.copy_(out["energy"], non_blocking=True)
                host_c.copy_(out["cut"], non_blocking=True)
                return
            d_p0.copy_(pin_p0, non_blocking=True)
            d_phi0.copy_(pin_phi0, non_blocking=True)
            ctx.run(S, R, sched=sched, precision=best_prec, init=hqa.INIT_GIVEN, phi0=d_phi0,
                    p0=d_p0, out=out)
            sub_s, sub_e = ctx.solve_sub(out["spins"], out["frozen"], n)
            host_spins.copy_(sub_s, non_blocking=True)
            host_e.copy_(sub_e, non_blocking=True)
            host_c.copy_(out["cut"], non_blocking=True)

        t_e2e = timed(e2e_step, args.steps, args.warmup)
    ctx.sync()

    su_step = N * R * S
    tot_pipe = sum(variants[head]["t_pipe"])
    tot_e2e = sum(t_e2e)
    tot_pipe, tot_e2e = reduce_max([tot_pipe, tot_e2e], ws)
    value = whole_job_rate(su_step, args.steps, ws, tot_pipe)
    e2e_value = whole_job_rate(su_step, args.steps, ws, tot_e2e)

    # roofline of the dominant kernel (the MD kernel), timed alone with CUDA events
    clk = clocks.summary()
    hv = variants[head]
    if batch:
        rb = hv["tuned"]["replicas_per_block"] if hv["tuned"] else 0
        kb = hv["tuned"]["kernel"] if hv["tuned"] else hqa.KERNEL_AUTO
        plan = {"kernel": kb, "replicas_per_block": rb, "members": count,
                "note": "persistent batch kernel and replica blocking picked by the autotuner"
                        if rb else "persistent batch kernel and blocking picked by the library"}
        base = {hqa.KERNEL_LOWDEG: "k_batch_lowdeg", hqa.KERNEL_SCALAR: "k_sparse_md_batch"}.get(
            kb, "k_batch_lowdeg|k_sparse_md_batch")
        kname = f"{base}<{rb or '*'},{'true' if hv['prec_name'] == 'PREC_BF16' else 'false'}>"
    else:
        plan = ctx.plan(R, precision=hv["prec"])
        kname = kernel_name(hqa, plan, hv["prec_name"])
    t_md = float(np.mean(hv["t_md"]))
    if cfg["kind"] in ("dense", "dense_sg"):
        pk = measured_peaks()
        flops = 2.0 * N * N * R * S                     # algorithmic: the field GEMM
        kseg = (3 if real else 2) if hv["prec_name"] == "PREC_BF16X2" else 1
        mma = flops * kseg                              # issued: one MMA pass per K segment
        achieved = flops / t_md / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"],
                "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops"],
                "mma_tflops_issued": mma / t_md / 1e12, "peak_source": pk["source"]}
    else:
        es = ELEM_BYTES[hv["prec_name"]]
        bytes_per_launch = nnz * es * R * S   # gathered operand bytes: deg x elem size per spin-update
        achieved = bytes_per_launch / t_md / 1e9
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clk.get("sm_max_mhz") or 2070.0
        peak = sm_count * 128 * mhz * 1e6 / 1e9     # GB/s: 128 B/clk/SM shared-memory bandwidth
        roof = {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "peak_source": "derived: SMs x 128 B/clk x max SM clock (shared-memory bandwidth)"}
    roof["traffic"] = ncu_traffic(f"{kname}@{args.config}")
    roof["kernel"] = kname
    roof["kernel_ms"] = 1e3 * t_md
    roof["plan"] = plan

    tabu = None
    if cfg.get("tabu"):
        # large-n sub-solve (the paper's HQA(TS1000) shape): tabu search on the n least
        # frozen spins of the headline run's readout, timed on its own with CUDA events
        tb = cfg["tabu"]
        Rt = tb["replicas"]
        o2 = ctx.run(S, Rt, seed=seed_base, sched=hqa.schedule(n_ambivalent=tb["n"]),
                     precision=hv["prec"], outputs=("phibar", "spins", "frozen", "energy"))
        ts = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, te = ctx.solve_sub_tabu(o2["spins"], o2["frozen"], tb["n"], tb["iters"], tb["tenure"])
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        gain = (o2["energy"] - te).double()
        tabu = {"n": tb["n"], "iters": tb["iters"], "tenure": tb["tenure"], "replicas": Rt,
                "ms": float(np.median(ts)),
                "flips_per_s": Rt * tb["iters"] / (float(np.median(ts)) / 1e3),
                "median_energy_gain_over_readout": float(gain.median()),
                "bound": "issue: two block-wide argmins and 2 barriers per flip, row loads from L2"}
    cpu = cpu_baseline(args, inst, cfg) if (rank == 0 and not args.skip_cpu) else None
    # launches per pipeline step: MD (+ init and output copy per chunk on the dense
    # path), readout, energy (real couplings: spin masks, fixed-point sums, rounding);
    # the exact sub-solve adds prep, packed minimum, packed argmin, scalar walk
    # (returns at once for packed replicas), assemble and energy
    launches = (3 * plan.get("chunks", 1) if plan["kernel"] == hqa.KERNEL_DENSE else 1) + 1 + \
        (3 if real else 1) + (0 if batch or real else 6)
    line = {
        "metric": METRIC, "value": value, "unit": "spin-updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_pipe / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"PREC_FP32": "f32", "PREC_BF16": "bf16-operand/f32-accumulate",
                  "PREC_BF16X2": "bf16x2-split-operand/f32-accumulate"}[hv["prec_name"]],
        "data": "synthetic (seeded instance generator)",
        "config": {"workload": cfg["desc"] if S == CONFIGS[args.config]["S"] else
                   cfg["desc"] + f" (shortened to {S} steps)", "N": N, "nnz": nnz,
                   "replicas": R, "md_steps": S, "instances": count,
                   "n_ambivalent": n, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas only, {ws} GPU(s)"},
        "variants": {k: {"spin_updates_per_s": su_step * args.steps / sum(v["t_pipe"]),
                         "graph_replay_spin_updates_per_s":
                             su_step * args.steps / sum(v["t_graph"]) if v["t_graph"] else None,
                         "autotuned": v["tuned"],
                         "md_kernel_ms": 1e3 * float(np.mean(v["t_md"])),
                         "median_cut": v["median_cut"], "cut_ci95_halfwidth": v["cut_ci95_halfwidth"],
                         "mean_cut": v["mean_cut"], "equal_cut_vs_plain": eq[k]}
                     for k, v in variants.items()},
        "headline_variant": head,
        "equal_cut": {"rule": "95% bootstrap interval of median(variant cut) - median(plain cut) "
                              "reaches 0", "plain": cfg["plain"]},
        "e2e": {"value": e2e_value, "unit": "spin-updates/s",
                "h2d_bytes_per_step": 2 * R * N * 4,
                "d2h_bytes_per_step": R * N + (1 if real else 2) * RR * 8},
        "gpu_launches": launches * args.steps,
        "roofline": roof,
        "clocks": clk,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if tabu:
        line["tabu_sub_solve"] = tabu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


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
    S, reps = _cpu_sample_shape(cfg, cores, 16 if cfg["kind"] == "sparse" else 2)
    wall = _oracle_sample(inst, S, reps, cores)
    return {"value": inst.N * reps * S / wall, "unit": "spin-updates/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{reps} of {cfg['R']} replicas x {S} of {cfg['S']} steps "
                      "(MD only, FP64, OpenMP over replicas)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    cfg = CONFIGS[args.config]
    inst = make_instance(args.config)
    cores = os.cpu_count() or 1
    S, reps = _cpu_sample_shape(cfg, cores, 1)
    if cfg["kind"] == "batch":
        inst = inst[len(inst) // 2]     # one mid-size member per step
    for _ in range(args.warmup):
        _oracle_sample(inst, min(S, 20), reps, cores)
    walls = [_oracle_sample(inst, S, reps, cores) for _ in range(args.steps)]
    value = inst.N * reps * S * args.steps / sum(walls)
    sample = f"{reps} of {cfg['R']} replicas x {S} of {cfg['S']} steps per step (MD only, FP64 oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "spin-updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(walls) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded instance generator)",
        "config": {"workload": cfg["desc"], "N": inst.N, "replicas": cfg["R"], "md_steps": cfg["S"]},
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
    ap.add_argument("--config", default="er800", choices=sorted(CONFIGS))
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
