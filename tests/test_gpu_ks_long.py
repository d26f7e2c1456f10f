"""Long-horizon parity over 1024 seeds on the dense and batched workloads.

Over 1000 paper-schedule steps (dt = 1/1000) the trajectories are chaotic, so
pointwise parity gives way to the distribution test the method's quality
rests on: over 1024 seeds, the GPU's final cuts (or Ising energies) must not
be stochastically worse than the FP64 oracle's (one-sided two-sample
Kolmogorov-Smirnov test, p = 0.01), for every arithmetic the dense path offers
and for a 64-member slice of the uneven batch.  Methods, "Leapfrog algorithm"
and "Scheduling functions for MD"; cuts and energies as in Results Eq. (1) and
Methods, "MAX-CUT and Ising spin-glass".
"""
import numpy as np
import pytest

from paper_2004_03972_gb300 import instances

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
stats = pytest.importorskip("scipy.stats")

R, S, SEED = 1024, 1000, 77


@pytest.fixture(scope="module")
def hqa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_03972_gb300 import build, hqa as H
    build.build()
    return H


def _not_worse(gpu, ref, higher_is_better):
    alt = "greater" if higher_is_better else "less"
    return stats.ks_2samp(gpu, ref, alternative=alt).pvalue


@pytest.fixture(scope="module")
def k2000(orc):
    inst = instances.sk_pm1(2000, 1300)
    pr = orc.Problem.from_instance(inst)
    p0 = np.stack([orc.initial_momenta(SEED, r, inst.N) for r in range(R)])
    _, _, pbar = orc.md_run_dense_batch(pr, S, np.zeros_like(p0), p0)
    cuts = np.array([orc.cut_int(pr, np.where(pbar[r] >= 0, 1, -1)) for r in range(R)])
    return inst, cuts


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_k2000_cut_distribution_not_worse(hqa, orc, k2000, prec):
    inst, ocuts = k2000
    ctx = hqa.Context.from_instance(inst)
    out = ctx.run(S, R, seed=SEED, precision=prec, kernel=hqa.KERNEL_DENSE,
                  outputs=("phibar", "spins", "cut"))
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    spins = out["spins"].cpu().numpy()
    cuts = out["cut"].cpu().numpy()
    for r in (0, 500, R - 1):
        assert int(cuts[r]) == orc.cut_int(pr, spins[r])
    p = _not_worse(cuts, ocuts, True)
    assert p > 0.01, (prec, p, np.median(cuts), np.median(ocuts))


@pytest.fixture(scope="module")
def sg2000(orc):
    inst = instances.uniform_sg(2000, 1350)
    pr = orc.Problem.from_instance(inst)
    p0 = np.stack([orc.initial_momenta(SEED, r, inst.N) for r in range(R)])
    _, _, pbar = orc.md_run_dense_batch(pr, S, np.zeros_like(p0), p0)
    en = np.array([orc.energy_f64(pr, np.where(pbar[r] >= 0, 1, -1)) for r in range(R)])
    return inst, en


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_spin_glass_energy_distribution_not_worse(hqa, orc, sg2000, prec):
    inst, oen = sg2000
    ctx = hqa.Context.from_instance(inst)
    out = ctx.run(S, R, seed=SEED, precision=prec, kernel=hqa.KERNEL_DENSE,
                  outputs=("phibar", "spins"))
    en = ctx.energy_f64(out["spins"])
    ctx.sync()
    en = en.cpu().numpy()
    pr = orc.Problem.from_instance(inst)
    spins = out["spins"].cpu().numpy()
    for r in (0, R - 1):
        assert abs(en[r] - orc.energy_f64(pr, spins[r])) <= 1e-9 * np.abs(inst.dense).sum()
    p = _not_worse(en, oen, False)
    assert p > 0.01, (prec, p, np.median(en), np.median(oen))


@pytest.fixture(scope="module")
def batch64(orc):
    members = instances.uneven_batch(512, 200, 5000, 1400)[:64]
    RM = R // len(members)
    fr = []
    for k, inst in enumerate(members):
        pr = orc.Problem.from_instance(inst)
        seed = (SEED + (k + 1) * 0x632BE59BD9B4E019) % (1 << 64)
        p0 = np.stack([orc.initial_momenta(seed, r, inst.N) for r in range(RM)])
        _, _, pbar = orc.md_run_replicas(pr, S, np.zeros_like(p0), p0)
        edges = len(inst.val) // 2
        fr += [orc.cut_int(pr, np.where(pbar[r] >= 0, 1, -1)) / edges for r in range(RM)]
    return members, RM, np.array(fr)


@pytest.mark.parametrize("prec", [0, 1])
def test_uneven_batch_cut_distribution_not_worse(hqa, orc, batch64, prec):
    """Cut fractions (cut / edges of the member) over 64 members x 16 seeds."""
    members, RM, ofr = batch64
    ctxs = [hqa.Context.from_instance(m) for m in members]
    b = hqa.Context.batch(ctxs)
    out = b.run(S, RM, seed=SEED, precision=prec, outputs=("phibar", "spins", "cut"))
    b.sync()
    cuts = out["cut"].cpu().numpy().reshape(len(members), RM)
    fr = np.concatenate([cuts[k] / (len(m.val) // 2) for k, m in enumerate(members)])
    spins = b.split(out["spins"], RM)
    pr = orc.Problem.from_instance(members[3])
    assert int(cuts[3, 5]) == orc.cut_int(pr, spins[3][5].cpu().numpy())
    p = _not_worse(fr, ofr, True)
    assert p > 0.01, (prec, p, np.median(fr), np.median(ofr))
