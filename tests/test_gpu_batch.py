"""Uneven batches (hqa_create_batch): one persistent launch over many instances of
different size must give every member exactly what a run of that member alone gives
(same kernel and blocking: bitwise), and match the FP64 oracle (FP32 tolerances)."""
import numpy as np
import pytest

from paper_2004_03972_gb300 import instances

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLD = 0x632BE59BD9B4E019
M64 = (1 << 64) - 1


def member_seed(seed, k):
    return (seed + (k + 1) * GOLD) & M64


@pytest.fixture(scope="module")
def hqa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_03972_gb300 import build, hqa as H
    build.build()
    return H


def _members():
    return [instances.regular3_pm1(50, 1), instances.torus_pm1(7, 8, 2),
            instances.with_integer_field(instances.regular3_pm1(120, 3), 1, 4),
            instances.torus_pm1(10, 12, 5), instances.regular3_pm1(301, 6),
            instances.torus_pm1(5, 20, 7)]


@pytest.mark.parametrize("rb", [1, 2, 4])
def test_batch_equals_member_runs_bitwise(hqa, rb):
    insts = _members()
    ctxs = [hqa.Context.from_instance(i) for i in insts]
    batch = hqa.Context.batch(ctxs)
    R, S, seed = 5, 80, 99
    sched = hqa.schedule(n_ambivalent=6)
    out = batch.run(S, R, seed=seed, sched=sched, dt=1 / 400, replicas_per_block=rb,
                    kernel=hqa.KERNEL_SCALAR)
    batch.sync()
    views = {k: batch.split(out[k], R) for k in ("phi", "p", "phibar", "spins", "frozen")}
    for k, c in enumerate(ctxs):
        alone = c.run(S, R, seed=member_seed(seed, k), sched=sched, dt=1 / 400,
                      replicas_per_block=rb, kernel=hqa.KERNEL_SCALAR)
        c.sync()
        for key in views:
            assert torch.equal(views[key][k], alone[key]), (k, key)
        assert torch.equal(out["energy"][k * R:(k + 1) * R], alone["energy"])
        assert torch.equal(out["cut"][k * R:(k + 1) * R], alone["cut"])
        assert torch.equal(out["tally"][k * R:(k + 1) * R], alone["tally"])


def test_batch_given_state_and_resume_bitwise(hqa):
    """HQA_INIT_GIVEN on a batch takes phi0 / p0 in the batch layout: every member
    equals its own run from its block, and a run split at step S1 (state handed over,
    start_step = S1) reproduces the whole run bitwise."""
    insts = _members()
    ctxs = [hqa.Context.from_instance(i) for i in insts]
    batch = hqa.Context.batch(ctxs)
    R, S, S1, dt = 5, 200, 80, 1 / 400
    sched = hqa.schedule(n_ambivalent=6)
    tot = sum(i.N for i in insts)
    g = torch.Generator().manual_seed(3)
    phi0 = ((torch.rand((R, tot), generator=g) - 0.5) * 0.2).cuda()
    p0 = (torch.randint(0, 2, (R, tot), generator=g) * 2 - 1).float().cuda()
    kw = dict(sched=sched, dt=dt, init=hqa.INIT_GIVEN, replicas_per_block=2,
              kernel=hqa.KERNEL_SCALAR)
    out = batch.run(S, R, phi0=phi0, p0=p0, **kw)
    batch.sync()
    keys = ("phi", "p", "phibar", "spins")
    views = {k: batch.split(out[k], R) for k in keys}
    ph_b, p_b = batch.split(phi0, R), batch.split(p0, R)
    for k, c in enumerate(ctxs):
        alone = c.run(S, R, phi0=ph_b[k].contiguous(), p0=p_b[k].contiguous(), **kw)
        c.sync()
        for key in keys:
            assert torch.equal(views[key][k], alone[key]), (k, key)
    a = batch.run(S1, R, phi0=phi0, p0=p0, outputs=("phi", "p"), **kw)
    b = batch.run(S - S1, R, phi0=a["phi"], p0=a["p"], start_step=S1,
                  outputs=("phi", "p", "phibar"), **kw)
    batch.sync()
    for key in ("phi", "p", "phibar"):   # the window (100 steps) lies in the second call
        assert torch.equal(b[key], out[key]), key


def test_lowdeg_kernel(hqa, orc):
    """The low-degree batch kernel (lists, operand and state of a work item on chip):
    the same bits at every replica blocking and as each member's own batch of one,
    FP32 states within 1e-5 of the FP64 oracle (BF16 operand: 1e-2), and a run split
    at step S1 equal to the whole run."""
    insts = _members()
    ctxs = [hqa.Context.from_instance(i) for i in insts]
    batch = hqa.Context.batch(ctxs)
    R, S, seed, dt = 6, 150, 21, 1 / 500
    kw = dict(seed=seed, dt=dt, kernel=hqa.KERNEL_LOWDEG, outputs=("phi", "p", "phibar"))
    runs = {rb: batch.run(S, R, replicas_per_block=rb, **kw) for rb in (1, 2, 4)}
    bf = batch.run(S, R, replicas_per_block=2, precision=hqa.PREC_BF16, **kw)
    batch.sync()
    for rb in (2, 4):
        for key in ("phi", "p", "phibar"):
            assert torch.equal(runs[rb][key], runs[1][key]), (rb, key)
    out = runs[2]
    views = {key: batch.split(out[key], R) for key in ("phi", "p", "phibar")}
    bviews = {key: batch.split(bf[key], R) for key in ("phi", "p")}
    for k, c in enumerate(ctxs):
        one = hqa.Context.batch([c])
        alone = one.run(S, R, replicas_per_block=2, **dict(kw, seed=(seed + k * GOLD) & M64))
        one.sync()
        for key in views:
            assert torch.equal(views[key][k], alone[key]), (k, key)
        pr = orc.Problem.from_instance(insts[k])
        for r in (0, R - 1):
            ophi, op, _ = orc.md_run(pr, S, dt=dt, p0=orc.initial_momenta(member_seed(seed, k), r,
                                                                          insts[k].N))
            for tol, src in ((1e-5, views), (1e-2, bviews)):
                g_phi = src["phi"][k][r].cpu().numpy().astype(np.float64)
                g_p = src["p"][k][r].cpu().numpy().astype(np.float64)
                assert np.max(np.abs(g_phi - ophi)) <= tol * np.max(np.abs(ophi)), (k, r, tol)
                assert np.max(np.abs(g_p - op)) <= tol * max(1.0, np.max(np.abs(op))), (k, r, tol)
    a = batch.run(40, R, replicas_per_block=2, **dict(kw, outputs=("phi", "p")))
    b = batch.run(S - 40, R, replicas_per_block=2, init=hqa.INIT_GIVEN, phi0=a["phi"], p0=a["p"],
                  start_step=40, **kw)
    batch.sync()
    for key in ("phi", "p", "phibar"):   # the window (100 steps) lies in the second call
        assert torch.equal(b[key], out[key]), key


def test_lowdeg_needs_low_degree(hqa):
    ctxs = [hqa.Context.from_instance(instances.torus_pm1(6, 6, 1)),
            hqa.Context.from_instance(instances.er_pm1(100, 0.1, 2))]   # degree ~10
    batch = hqa.Context.batch(ctxs)
    with pytest.raises(hqa.HQAError) as ei:
        batch.run(20, 4, kernel=hqa.KERNEL_LOWDEG)
    assert ei.value.status == 6
    x = batch.run(20, 4, outputs=("phi",))                  # AUTO: the list-streaming kernel
    y = batch.run(20, 4, outputs=("phi",), kernel=hqa.KERNEL_SCALAR)
    batch.sync()
    assert torch.equal(x["phi"], y["phi"])
    single = hqa.Context.from_instance(instances.torus_pm1(6, 6, 1))
    with pytest.raises(hqa.HQAError):
        single.run(20, 4, kernel=hqa.KERNEL_LOWDEG)


def test_batch_matches_oracle(hqa, orc):
    insts = _members()
    ctxs = [hqa.Context.from_instance(i) for i in insts]
    batch = hqa.Context.batch(ctxs)
    R, S, seed, dt = 4, 100, 7, 1 / 500
    out = batch.run(S, R, seed=seed, dt=dt, outputs=("phi", "p", "phibar"))
    batch.sync()
    phis, ps = batch.split(out["phi"], R), batch.split(out["p"], R)
    for k, inst in enumerate(insts):
        pr = orc.Problem.from_instance(inst)
        for r in (0, R - 1):
            p0 = orc.initial_momenta(member_seed(seed, k), r, inst.N)
            ophi, op, _ = orc.md_run(pr, S, dt=dt, p0=p0)
            g_phi = phis[k][r].cpu().numpy().astype(np.float64)
            g_p = ps[k][r].cpu().numpy().astype(np.float64)
            assert np.max(np.abs(g_phi - ophi)) <= 1e-5 * np.max(np.abs(ophi))
            assert np.max(np.abs(g_p - op)) <= 1e-5 * max(1.0, np.max(np.abs(op)))


def test_uneven_batch_structure(hqa, orc):
    """The benchmark ensemble's structure at reduced count: N uniform in [200, 5000],
    half 3-regular, half tori; readout and energies exact for sampled members."""
    insts = instances.uneven_batch(16, 200, 5000, 4)
    ctxs = [hqa.Context.from_instance(i) for i in insts]
    batch = hqa.Context.batch(ctxs)
    R, S, n = 8, 300, 24
    out = batch.run(S, R, seed=3, sched=hqa.schedule(n_ambivalent=n))
    batch.sync()
    pbar = batch.split(out["phibar"], R)
    spins = batch.split(out["spins"], R)
    for k in (0, 5, 15):
        pr = orc.Problem.from_instance(insts[k])
        for r in (0, R - 1):
            s, f = orc.readout(pbar[k][r].cpu().numpy().astype(np.float64), n)
            assert np.array_equal(spins[k][r].cpu().numpy(), s)
            assert int(out["energy"][k * R + r]) == orc.energy_int(pr, s)
            assert int(out["cut"][k * R + r]) == orc.cut_int(pr, s)
    assert torch.all(out["tally"][:, 1] == n)


def test_batch_rejects_unsupported(hqa):
    ctxs = [hqa.Context.from_instance(instances.torus_pm1(4, 4, 1))]
    batch = hqa.Context.batch(ctxs)
    with pytest.raises(hqa.HQAError):
        batch.local_field(torch.zeros((1, 16), device="cuda"))
    with pytest.raises(hqa.HQAError):
        hqa.Context.batch([batch])


def test_batch_spilled_state_bitwise(hqa):
    """Members too large to keep p and the window sums on chip use per-CTA slices in
    global memory; slices must not overlap across members of different size."""
    insts = [instances.regular3_pm1(4000, 11), instances.torus_pm1(50, 60, 12),
             instances.regular3_pm1(3400, 13), instances.torus_pm1(9, 9, 14),
             instances.regular3_pm1(4400, 15)]
    ctxs = [hqa.Context.from_instance(i) for i in insts]
    batch = hqa.Context.batch(ctxs)
    R, S, seed = 16, 60, 5
    out = batch.run(S, R, seed=seed, dt=1 / 300, replicas_per_block=4, kernel=hqa.KERNEL_SCALAR,
                    outputs=("phi", "p", "phibar"))
    batch.sync()
    for key in ("phi", "p", "phibar"):
        views = batch.split(out[key], R)
        for k, c in enumerate(ctxs):
            alone = c.run(S, R, seed=member_seed(seed, k), dt=1 / 300, replicas_per_block=4,
                          kernel=hqa.KERNEL_SCALAR, outputs=(key,))
            c.sync()
            assert torch.equal(views[k], alone[key]), (k, key)


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-2)])
def test_full_uneven512_batch_states(hqa, orc, prec, tol):
    """The benchmark's whole 512-member batch at its replica count (64) in the launch
    shape the autotuner picks for it (the low-degree kernel, 2 replicas per block):
    states after 100 steps of sampled members and replicas against the oracle, and
    the readout, int64 energies and cuts of sampled replicas exact."""
    insts = instances.uneven_batch(512, 200, 5000, 1400)
    ctxs = [hqa.Context.from_instance(i) for i in insts]
    batch = hqa.Context.batch(ctxs)
    R, S, seed, dt, n = 64, 100, 9, 1e-4, 24
    out = batch.run(S, R, seed=seed, dt=dt, precision=prec, replicas_per_block=2,
                    kernel=hqa.KERNEL_LOWDEG, sched=hqa.schedule(n_ambivalent=n))
    batch.sync()
    phis, ps, pbar = (batch.split(out[k], R) for k in ("phi", "p", "phibar"))
    spins = batch.split(out["spins"], R)
    for k in (0, 1, 255, 511):
        pr = orc.Problem.from_instance(insts[k])
        for r in (0, 37, R - 1):
            p0 = orc.initial_momenta(member_seed(seed, k), r, insts[k].N)
            ophi, op, _ = orc.md_run(pr, S, dt=dt, p0=p0, window=100)
            g_phi = phis[k][r].cpu().numpy().astype(np.float64)
            g_p = ps[k][r].cpu().numpy().astype(np.float64)
            assert np.max(np.abs(g_phi - ophi)) <= tol * np.max(np.abs(ophi))
            assert np.max(np.abs(g_p - op)) <= tol * max(1.0, np.max(np.abs(op)))
            s, _ = orc.readout(pbar[k][r].cpu().numpy().astype(np.float64), n)
            assert np.array_equal(spins[k][r].cpu().numpy(), s)
            assert int(out["energy"][k * R + r]) == orc.energy_int(pr, s)
            assert int(out["cut"][k * R + r]) == orc.cut_int(pr, s)
