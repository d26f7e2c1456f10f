"""Surrogate-gated HQA: a learned early stop on top of the method (the paper has
no learned component).  Every numerical step runs in libhqa's kernels; this
module sequences the calls.

  dataset()     features of the first fraction of each trajectory (hqa_run_features)
                and labels from the full run of the same trajectory:
                label 0 = spin ends frozen (rank split with n), label 1 = s = +1
  train()       minibatch AdamW on hqa_mlp_grad
  gated_run()   features -> network -> surrogate readout -> exact sub-solve of the
                accepted replicas (of every replica when scoring); replicas the gate
                does not accept resume the MD from the feature point to the full
                length (the fallback) and take the method's own readout + sub-solve
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import hqa


@dataclass
class SurrogateConfig:
    steps: int              # full trajectory length S
    frac: float = 0.1       # features from the first frac * S steps
    segments: int = 10      # feature samples
    n_ambivalent: int = 24
    precision: int = hqa.PREC_FP32
    max_expected_errors: float = 1.0

    @property
    def steps_c(self) -> int:
        return max(self.segments, int(round(self.frac * self.steps)))


def dataset(ctx, cfg: SurrogateConfig, replicas, seed, sched=None):
    """(x [R*N, 6], y [R*N, 2]) device tensors for one instance."""
    import torch
    sched = sched or hqa.schedule()
    sched.n_ambivalent = cfg.n_ambivalent
    dt = 1.0 / cfg.steps
    x, _, _ = ctx.features(cfg.steps_c, replicas, seed=seed, sched=sched, dt=dt,
                           segments=cfg.segments, precision=cfg.precision)
    full = ctx.run(cfg.steps, replicas, seed=seed, sched=sched, dt=dt, precision=cfg.precision,
                   outputs=("phibar", "spins", "frozen"))
    y = torch.stack([full["frozen"].reshape(-1).float(),
                     (full["spins"].reshape(-1) > 0).float()], dim=1).contiguous()
    return x, y


def train(mlp, xs, ys, epochs=30, batch=16384, lr=2e-3, weight_decay=1e-4, seed=0,
          precision=hqa.PREC_FP32):
    """Minibatch AdamW over the concatenated datasets; returns the loss history."""
    import torch
    x = torch.cat(xs).contiguous()
    y = torch.cat(ys).contiguous()
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(x.shape[0], generator=g).to(x.device)
        for k in range(0, x.shape[0], batch):
            idx = perm[k:k + batch]
            xb, yb = x[idx].contiguous(), y[idx].contiguous()
            grad, loss = mlp.grad(xb, yb, precision=precision)
            mlp.adamw(grad, lr=lr, weight_decay=weight_decay)
        hist.append(float(loss))
    return hist


def gated_run(ctx, mlp, cfg: SurrogateConfig, replicas, seed, sched=None, score_all=True):
    """Returns dict with spins/energy/cut per replica (device), accept mask, the
    surrogate-only results (score_all: for every replica, which costs a sub-solve of
    the rejected replicas too; else only for the accepted ones, the gated form's
    own work), and the MD steps actually spent."""
    import torch
    sched = sched or hqa.schedule()
    sched.n_ambivalent = cfg.n_ambivalent
    dt = 1.0 / cfg.steps
    R, n = replicas, cfg.n_ambivalent
    x, phi_c, p_c = ctx.features(cfg.steps_c, R, seed=seed, sched=sched, dt=dt,
                                 segments=cfg.segments, precision=cfg.precision)
    logits = mlp.forward(x, precision=cfg.precision)
    s_sur, f_sur, accept, err = ctx.surrogate_readout(logits, R, n, cfg.max_expected_errors)
    acc = accept.bool()
    rej = (~acc).nonzero().squeeze(1)
    n_fallback = int(rej.numel())
    out = {"accept": acc, "expected_errors": err}
    if score_all:
        sub_s, sub_e = ctx.solve_sub(s_sur, f_sur, n)
        e_sur, c_sur = ctx.energy(sub_s)
        out.update(surrogate_spins=sub_s, surrogate_energy=e_sur, surrogate_cut=c_sur)
        spins = sub_s.clone()
    else:
        # the exact sub-solve only where the gate stopped the replica
        spins = s_sur.clone()
        aidx = acc.nonzero().squeeze(1)
        if int(aidx.numel()):
            a_s, _ = ctx.solve_sub(s_sur.index_select(0, aidx).contiguous(),
                                   f_sur.index_select(0, aidx).contiguous(), n)
            spins[aidx] = a_s
    # fallback: the replicas the gate rejected resume the MD from the feature point to the
    # full length (bitwise the full trajectory) and take the method's own readout
    if n_fallback:
        rest = ctx.run(cfg.steps - cfg.steps_c, n_fallback, sched=sched, dt=dt,
                       precision=cfg.precision, init=hqa.INIT_GIVEN,
                       phi0=phi_c.index_select(0, rej).contiguous(),
                       p0=p_c.index_select(0, rej).contiguous(), start_step=cfg.steps_c,
                       outputs=("phibar", "spins", "frozen"))
        fs, _ = ctx.solve_sub(rest["spins"], rest["frozen"], n)
        spins[rej] = fs
    energy, cut = ctx.energy(spins)
    out.update(spins=spins, energy=energy, cut=cut,
               md_steps=cfg.steps_c * R + (cfg.steps - cfg.steps_c) * n_fallback)
    return out


def method_run(ctx, cfg: SurrogateConfig, replicas, seed, steps=None, sched=None):
    """The method without the network: MD for `steps` steps of the full-length schedule,
    the paper's readout (sgn and |phibar| rank) and the exact sub-solve."""
    sched = sched or hqa.schedule()
    sched.n_ambivalent = cfg.n_ambivalent
    steps = cfg.steps if steps is None else steps
    out = ctx.run(steps, replicas, seed=seed, sched=sched, dt=1.0 / cfg.steps,
                  precision=cfg.precision, outputs=("phibar", "spins", "frozen"))
    s, e = ctx.solve_sub(out["spins"], out["frozen"], cfg.n_ambivalent)
    e2, c = ctx.energy(s)
    return {"spins": s, "energy": e2, "cut": c, "md_spins": out["spins"], "frozen": out["frozen"]}


def score_against_full(gated, full, z2=True):
    """The full MD run as the reference for the surrogate: per replica, the fraction of
    spins whose surrogate result differs from the full run's (up to the global flip
    when z2, i.e. for instances without a field) and the cut lost (full - surrogate).
    Returns numpy arrays (mislabel, cut_loss, accepted)."""
    s = gated["surrogate_spins"].float()
    f = full["spins"].float()
    agree = (s == f).float().mean(1)
    if z2:
        agree = agree.maximum(1.0 - agree)
    mis = (1.0 - agree).cpu().numpy()
    loss = (full["cut"] - gated["surrogate_cut"]).cpu().numpy()
    return mis, loss, gated["accept"].cpu().numpy().astype(bool)
