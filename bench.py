#!/usr/bin/env python3
"""HQA-MD benchmark: flux-MD spin-updates/s on one GB300.

Workload (default, --config er800): Erdos-Renyi G(800, 0.06) with +-1 weights
in CSR, 1024 replicas with seeded +-1 initial momenta, 5000 leapfrog steps of
the paper's schedule (dt = 1/5000), then readout, int64 energy/cut and the
exact sub-solve of the n = 24 least-frozen spins per replica.  One bench
"step" is that whole pipeline over the 1024 replicas.  Spin-updates per step
= N * R * S (one leapfrog step of one spin in one replica).

Variants: plain FP32 operand and BF16 operand (FP32 accumulate, FP32 state).
The headline value is the faster variant whose median cut is not below the
plain variant's median cut minus its bootstrap 95% half-width (equal-cut
rule); both are reported under "variants".

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores over a bounded sample of the same workload.
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

CONFIGS = {
    # name: (builder, N-ish label, replicas, steps, n_ambivalent)
    "er800": dict(desc="ER G(800,0.06) +-1 CSR, 1024 replicas, 5000 steps, paper schedule, n=24 exact sub-solve",
                  R=1024, S=5000, n=24),
    "sk100": dict(desc="SK N=100 +-1, 1 replica, 1000 steps, linear-gamma schedule, n=20 exact sub-solve",
                  R=1, S=1000, n=20),
}


def make_instance(name):
    from paper_2004_03972_gb300 import instances
    if name == "er800":
        return instances.er_pm1(800, 0.06, 1200)
    if name == "sk100":
        return instances.sk_pm1(100, 1100)
    raise KeyError(name)


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
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


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


def run_ours(args):
    import torch

    from paper_2004_03972_gb300 import build, hqa
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    build.build()
    cfg = CONFIGS[args.config]
    inst = make_instance(args.config)
    N, R, S, n = inst.N, cfg["R"], cfg["S"], cfg["n"]
    ctx = hqa.Context.from_instance(inst)
    sched = hqa.schedule(n_ambivalent=n)
    if args.config == "sk100":
        sched.kind = hqa.SCHED_LINEAR_GAMMA
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    launches_per_step = 1 + 1 + 1 + 4   # md, readout, energy, sub-solve (prep, enum, assemble, energy)
    seed_base = 1000 + rank * 100003

    out = {k: torch.empty(s, dtype=d, device=dev) for k, s, d in (
        ("phi", (R, N), torch.float32), ("p", (R, N), torch.float32),
        ("phibar", (R, N), torch.float32), ("spins", (R, N), torch.int8),
        ("frozen", (R, N), torch.uint8), ("energy", (R,), torch.int64),
        ("cut", (R,), torch.int64), ("tally", (R, 2), torch.int32))}

    def pipeline(prec, seed):
        ctx.run(S, R, seed=seed, sched=sched, precision=prec, out=out)
        sub_s, sub_e = ctx.solve_sub(out["spins"], out["frozen"], n)
        return sub_s, sub_e

    def timed(fn, K, W):
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
            e0.record(stream)
            fn(W + k)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        return times

    variants = {}
    clocks = ClockSampler(local)
    with clocks:
        for name, prec in (("fp32", hqa.PREC_FP32), ("bf16", hqa.PREC_BF16)):
            cuts = []

            def step(k, prec=prec, cuts=cuts):
                pipeline(prec, seed_base + k)
            t_pipe = timed(step, args.steps, args.warmup)
            ctx.sync()
            # quality at equal cut: MD readout cuts over the same seeds for both variants
            for k in range(args.steps):
                ctx.run(S, R, seed=seed_base + 7 * k, sched=sched, precision=prec, out=out)
                cuts.append(out["cut"].cpu().numpy().copy())
            ctx.sync()
            allcuts = np.concatenate(cuts)
            # MD kernel alone (roofline)
            md_out = {"phibar": out["phibar"]}

            def md_only(k, prec=prec):
                ctx.run(S, R, seed=seed_base + k, sched=sched, precision=prec, out=md_out)
            t_md = timed(md_only, args.steps, 1)
            variants[name] = dict(prec=prec, t_pipe=t_pipe, t_md=t_md, cuts=allcuts,
                                  median_cut=float(np.median(allcuts)),
                                  cut_ci95_halfwidth=bootstrap_halfwidth(allcuts),
                                  mean_cut=float(np.mean(allcuts)))
        # end-to-end through the public API with host buffers
        pin_p0 = torch.empty((R, N), dtype=torch.float32).pin_memory()
        pin_phi0 = torch.zeros((R, N), dtype=torch.float32).pin_memory()
        g = torch.Generator().manual_seed(rank)
        pin_p0.copy_((torch.randint(0, 2, (R, N), generator=g) * 2 - 1).float())
        host_spins = torch.empty((R, N), dtype=torch.int8).pin_memory()
        host_e = torch.empty((R,), dtype=torch.int64).pin_memory()
        host_c = torch.empty((R,), dtype=torch.int64).pin_memory()
        d_p0 = torch.empty((R, N), dtype=torch.float32, device=dev)
        d_phi0 = torch.empty((R, N), dtype=torch.float32, device=dev)
        best_prec = hqa.PREC_FP32

        def e2e_step(k):
            d_p0.copy_(pin_p0, non_blocking=True)
            d_phi0.copy_(pin_phi0, non_blocking=True)
            ctx.run(S, R, sched=sched, precision=best_prec, init=hqa.INIT_GIVEN, phi0=d_phi0,
                    p0=d_p0, out=out)
            sub_s, sub_e = ctx.solve_sub(out["spins"], out["frozen"], n)
            host_spins.copy_(sub_s, non_blocking=True)
            host_e.copy_(sub_e, non_blocking=True)
            host_c.copy_(out["cut"], non_blocking=True)

        fp, bf = variants["fp32"], variants["bf16"]
        # equal cut: the 95% interval of median(bf16) - median(fp32) reaches 0 or above
        diff_lo, diff_hi = median_diff_ci(bf["cuts"], fp["cuts"])
        equal_cut = diff_hi >= 0.0
        head = "bf16" if (equal_cut and np.mean(bf["t_pipe"]) < np.mean(fp["t_pipe"])) else "fp32"
        best_prec = variants[head]["prec"]
        t_e2e = timed(e2e_step, args.steps, args.warmup)
    ctx.sync()

    su_step = N * R * S
    tot_pipe = sum(variants[head]["t_pipe"])
    tot_e2e = sum(t_e2e)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([tot_pipe, tot_e2e], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_pipe, tot_e2e = float(t[0]), float(t[1])
    value = su_step * args.steps * ws / tot_pipe
    e2e_value = su_step * args.steps * ws / tot_e2e

    # roofline of the dominant kernel (the resident sparse MD kernel)
    clk = clocks.summary()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    es = 2 if head == "bf16" else 4
    nnz = inst.nnz
    bytes_per_launch = nnz * es * R * S     # gathered operand bytes: deg x elem size per spin-update
    t_md = float(np.mean(variants[head]["t_md"]))
    achieved = bytes_per_launch / t_md / 1e9
    mhz = clk.get("sm_max_mhz") or 2070.0
    peak_smem = sm_count * 128 * mhz * 1e6 / 1e9    # GB/s: 128 B/clk/SM shared-memory bandwidth
    plan = ctx.plan(R, precision=variants[head]["prec"])
    rb = plan["replicas_per_block"]
    kname = ("k_sparse_md_vec" if plan["kernel"] == hqa.KERNEL_VECTOR else "k_sparse_md") + \
        f"<{rb},{'true' if head == 'bf16' else 'false'}>"
    traffic = ncu_traffic(f"{kname}@{args.config}")

    cpu = cpu_baseline(args, inst, cfg) if (rank == 0 and not args.skip_cpu) else None
    line = {
        "metric": "flux-MD spin-updates/s on 1 GB300, mixed/batched vs plain FP32 at equal cut",
        "value": value, "unit": "spin-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_pipe / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if head == "fp32" else "bf16-operand/f32-accumulate",
        "data": "synthetic (seeded instance generator)",
        "config": {"workload": cfg["desc"], "N": N, "nnz": nnz, "replicas": R, "md_steps": S,
                   "n_ambivalent": n, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas only, {ws} GPU(s)"},
        "variants": {k: {"spin_updates_per_s": su_step * args.steps / sum(v["t_pipe"]),
                         "md_kernel_ms": 1e3 * float(np.mean(v["t_md"])),
                         "median_cut": v["median_cut"], "cut_ci95_halfwidth": v["cut_ci95_halfwidth"],
                         "mean_cut": v["mean_cut"]} for k, v in variants.items()},
        "headline_variant": head,
        "equal_cut": {"rule": "95% bootstrap interval of median(bf16 cut) - median(fp32 cut) reaches 0",
                      "interval": [diff_lo, diff_hi], "holds": bool(equal_cut)},
        "e2e": {"value": e2e_value, "unit": "spin-updates/s",
                "h2d_bytes_per_step": 2 * R * N * 4, "d2h_bytes_per_step": R * N + 2 * R * 8},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "smem", "achieved": achieved, "peak": peak_smem, "unit": "GB/s",
                     "frac": achieved / peak_smem, "traffic": traffic,
                     "kernel": kname, "plan": plan,
                     "peak_source": "derived: SMs x 128 B/clk x max SM clock (shared-memory bandwidth)"},
        "clocks": clk,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _oracle_sample(inst, cfg, reps, threads):
    from oracle import oracle as orc
    pr = orc.Problem.from_instance(inst)
    N, S = inst.N, cfg["S"]
    p0 = np.stack([orc.initial_momenta(9, r, N) for r in range(reps)])
    phi0 = np.zeros_like(p0)
    t0 = time.perf_counter()
    orc.md_run_replicas(pr, S, phi0, p0, threads=threads)
    return time.perf_counter() - t0


def cpu_baseline(args, inst, cfg):
    from oracle import oracle as orc
    orc.build()
    cores = os.cpu_count() or 1
    reps = max(1, min(cfg["R"], 16 * cores))
    wall = _oracle_sample(inst, cfg, reps, cores)
    return {"value": inst.N * reps * cfg["S"] / wall, "unit": "spin-updates/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{reps} of {cfg['R']} replicas x {cfg['S']} steps (MD only, FP64, OpenMP over replicas)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    cfg = CONFIGS[args.config]
    inst = make_instance(args.config)
    cores = os.cpu_count() or 1
    reps = max(1, min(cfg["R"], cores))
    for _ in range(args.warmup):
        _oracle_sample(inst, dict(cfg, S=50), reps, cores)
    walls = [_oracle_sample(inst, cfg, reps, cores) for _ in range(args.steps)]
    value = inst.N * reps * cfg["S"] * args.steps / sum(walls)
    sample = f"{reps} of {cfg['R']} replicas x {cfg['S']} steps per step (MD only, FP64 oracle)"
    print(json.dumps({
        "impl": "reference",
        "metric": "flux-MD spin-updates/s on 1 GB300, mixed/batched vs plain FP32 at equal cut",
        "value": value, "unit": "spin-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
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
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
