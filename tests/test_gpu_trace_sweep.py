"""Strided phibar snapshots along an anneal (Fig. 4's frozen / ambivalent separation)
and the schedule / potential sweep (kappa2 in [-1, 1], M in {4, 8}) with the H_MD(tau=1)
diagnostic, against the oracle.

Snapshots are resumed segments of the same trajectory, so they equal stopped runs
bitwise; states after 100 steps agree with the FP64 oracle to 1e-5 of their scale
(FP32); H_MD of a state agrees to 1e-6 of the Hamiltonian's absolute scale."""
import numpy as np
import pytest

from paper_2004_03972_gb300 import instances

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hqa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_03972_gb300 import build, hqa as H
    build.build()
    return H


def test_snapshots_equal_stopped_runs(hqa):
    inst = instances.er_pm1(300, 0.05, 5)
    ctx = hqa.Context.from_instance(inst)
    R, S, K, dt = 5, 1000, 250, 1.0 / 1000
    tr, phi, p = ctx.trace(S, R, K, seed=8, dt=dt)
    full = ctx.run(S, R, seed=8, dt=dt, outputs=("phi", "p"))
    for t in range(S // K):
        part = ctx.run((t + 1) * K, R, seed=8, dt=dt, outputs=("phibar",))
        assert torch.equal(tr[t], part["phibar"]), t
    ctx.sync()
    assert torch.equal(phi, full["phi"]) and torch.equal(p, full["p"])


def test_first_snapshot_matches_oracle(hqa, orc):
    inst = instances.er_pm1(300, 0.05, 5)
    ctx = hqa.Context.from_instance(inst)
    dt = 1.0 / 1000
    tr, _, _ = ctx.trace(300, 3, 100, seed=2, dt=dt)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in range(3):
        ophi, _, opbar = orc.md_run(pr, 100, dt=dt, p0=orc.initial_momenta(2, r, inst.N))
        got = tr[0, r].cpu().numpy()
        assert np.max(np.abs(got - opbar)) <= 1e-5 * np.max(np.abs(ophi))


def test_frozen_fraction_grows_along_the_anneal(hqa):
    """Fig. 4's picture: early window means sit near zero (the fluxes oscillate through
    it), late ones are large (frozen); the fraction above a threshold grows."""
    inst = instances.er_pm1(800, 0.06, 1200)
    ctx = hqa.Context.from_instance(inst)
    tr, _, _ = ctx.trace(4000, 16, 400, seed=1)
    a = tr.abs().cpu().numpy()
    theta = 0.5 * np.median(a[-1])
    frac = (a > theta).mean(axis=(1, 2))
    assert frac[-1] > 0.8 and frac[0] < 0.5


@pytest.mark.parametrize("kappa2", [-1.0, 0.0, 1.0])
@pytest.mark.parametrize("M", [4, 8])
def test_schedule_and_potential_sweep(hqa, orc, kappa2, M):
    inst = instances.with_integer_field(instances.er_pm1(300, 0.05, 5), 2, 9)
    ctx = hqa.Context.from_instance(inst)
    pr = orc.Problem.from_instance(inst)
    prm = (0.008, 4.0, 3.0, 0.12, 0.05, kappa2, 0.032)
    sched = hqa.schedule(kappa2=kappa2, M=M)
    dt = 1.0 / 5000
    out = ctx.run(100, 4, seed=6, sched=sched, dt=dt, outputs=("phi", "p"))
    ctx.sync()
    for r in (0, 3):
        ophi, op, _ = orc.md_run(pr, 100, dt=dt, p0=orc.initial_momenta(6, r, inst.N), prm=prm, M=M)
        assert np.max(np.abs(out["phi"][r].cpu().numpy() - ophi)) <= 1e-5 * np.max(np.abs(ophi))
        assert np.max(np.abs(out["p"][r].cpu().numpy() - op)) <= 1e-5 * max(1.0, np.max(np.abs(op)))
    # H_MD at the end of a full anneal (tau = 1), the adiabaticity diagnostic of the sweep
    S = 400
    end = ctx.run(S, 4, seed=6, sched=sched, dt=1.0 / S, outputs=("phi", "p"))
    H = ctx.hmd(end["phi"], end["p"], 1.0, sched=sched, half_kick=True).cpu().numpy()
    for r in range(4):
        x = end["phi"][r].cpu().numpy().astype(np.float64)
        q = end["p"][r].cpu().numpy().astype(np.float64)
        q = q - 0.5 * orc.force(pr, 1.0, x, prm=prm, M=M)
        ref = orc.hmd(pr, 1.0, x, q, prm=prm, M=M)
        a, b = orc.schedule(1.0, prm=prm)
        scale = a * np.sum(0.5 * q * q + np.abs(x) ** M) + 0.5 * b * np.sum(
            np.abs(x) * (np.abs(inst.to_dense()) @ np.abs(x) + 2 * np.abs(inst.h) * np.abs(x)))
        assert abs(H[r] - ref) <= 1e-6 * scale
