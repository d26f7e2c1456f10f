"""Tabu-search sub-solve on the GPU (ambivalent sets of 40 to 1024 spins, too large
to enumerate) against the oracle's statement of the same deterministic search:
spins and energies bit-exact.  The cases span positions owned by both halves of the
block (n > 512), the maximum n = 1024, dense rows (K2000: the block walks 1999
neighbours per flip) and a tenure longer than the set, where every spin turns tabu
and iterations without an aspirating candidate flip nothing.  On small sets it never
beats the exact optimum and never returns worse than its input."""
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


@pytest.mark.parametrize("inst_name,n,iters,tenure", [
    ("er800", 48, 480, 8), ("er800", 200, 2000, 20), ("er800", 1000, 4000, 20),
    ("er_h", 120, 1200, 10), ("torus", 64, 640, 6), ("er800", 40, 400, 60),
    ("torus40", 1024, 3000, 30), ("sk2000", 1000, 3000, 20)])
def test_tabu_bit_exact(hqa, orc, inst_name, n, iters, tenure):
    inst = {"er800": lambda: instances.er_pm1(800, 0.06, 1200),
            "er_h": lambda: instances.with_integer_field(instances.er_pm1(300, 0.05, 5), 2, 9),
            "torus": lambda: instances.torus_pm1(20, 15, 3),
            "torus40": lambda: instances.torus_pm1(40, 40, 4),
            "sk2000": lambda: instances.sk_pm1(2000, 1300)}[inst_name]()
    ctx = hqa.Context.from_instance(inst)
    R = 4
    out = ctx.run(600, R, seed=12, sched=hqa.schedule(n_ambivalent=n),
                  outputs=("phibar", "spins", "frozen", "energy"))
    ts, te = ctx.solve_sub_tabu(out["spins"], out["frozen"], n, iters, tenure)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    s, f = out["spins"].cpu().numpy(), out["frozen"].cpu().numpy()
    for r in range(R):
        ws, we = orc.subsolve_tabu(pr, s[r], f[r], iters, tenure)
        assert np.array_equal(ts[r].cpu().numpy(), ws), r
        assert int(te[r]) == we
    assert torch.all(te <= out["energy"])


@pytest.mark.parametrize("hmax", [3, 600000])
def test_tabu_bit_exact_given_configurations(hqa, orc, hmax):
    """Random spins and masks (no MD run).  Fields up to 600,000 exceed 2^19, so the
    search takes its 64-bit keys; small fields take the 32-bit keys."""
    inst = instances.with_integer_field(instances.er_pm1(500, 0.04, 8), hmax, 10)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(hmax)
    R, n = 6, 700 if hmax > 3 else 300
    s = rng.choice(np.array([-1, 1], np.int8), size=(R, inst.N))
    f = np.ones((R, inst.N), np.uint8)
    for r in range(R):
        f[r, rng.permutation(inst.N)[:min(n, inst.N) - r]] = 0
    ts, te = ctx.solve_sub_tabu(torch.from_numpy(s).cuda(), torch.from_numpy(f).cuda(),
                                min(n, inst.N), 1500, 12)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in range(R):
        ws, we = orc.subsolve_tabu(pr, s[r], f[r], 1500, 12)
        assert np.array_equal(ts[r].cpu().numpy(), ws), r
        assert int(te[r]) == we


def test_tabu_hand_traced_triangle(hqa):
    """The hand-traced trajectory of tests/golden/tabu_triangle.txt, on the GPU."""
    import os
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                          "tabu_triangle.txt")
    J = -np.ones((3, 3)) + np.eye(3)
    ctx = hqa.Context.from_instance(instances.Instance("triangle", 3, dense=J, h=np.ones(3)))
    s = torch.ones((1, 3), dtype=torch.int8, device="cuda")
    f = torch.zeros((1, 3), dtype=torch.uint8, device="cuda")
    for line in open(golden):
        if not line.strip() or line.startswith("#"):
            continue
        tenure, iters, e_best, spins = line.split()
        out, e = ctx.solve_sub_tabu(s, f, 3, int(iters), int(tenure))
        ctx.sync()
        assert int(e[0]) == int(e_best), (tenure, iters)
        assert out[0].cpu().tolist() == [int(v) for v in spins.split(",")], (tenure, iters)


def test_tabu_against_exact_on_small_sets(hqa, orc):
    inst = instances.er_pm1(800, 0.06, 1200)
    ctx = hqa.Context.from_instance(inst)
    R, n = 16, 16
    out = ctx.run(600, R, seed=3, sched=hqa.schedule(n_ambivalent=n),
                  outputs=("phibar", "spins", "frozen", "energy"))
    ts, te = ctx.solve_sub_tabu(out["spins"], out["frozen"], n, 400, 4)
    xs, xe = ctx.solve_sub(out["spins"], out["frozen"], n)
    ctx.sync()
    assert torch.all(te >= xe) and torch.all(te <= out["energy"])
    assert (te == xe).float().mean().item() >= 0.5


def test_tabu_rejects(hqa):
    inst = instances.er_pm1(200, 0.05, 2)
    ctx = hqa.Context.from_instance(inst)
    s = torch.ones((2, inst.N), dtype=torch.int8, device="cuda")
    f = torch.zeros((2, inst.N), dtype=torch.uint8, device="cuda")   # all 200 ambivalent
    with pytest.raises(hqa.HQAError):
        ctx.solve_sub_tabu(s, f, 2000, 10, 2)                        # n above 1024
    o, _ = ctx.solve_sub_tabu(s, f, 100, 10, 2)                      # 200 ambivalent > n
    with pytest.raises(hqa.HQAError):
        ctx.sync()
    assert torch.equal(o, s)
    sg = hqa.Context.from_instance(instances.uniform_sg(64, 1))
    s2 = torch.ones((1, 64), dtype=torch.int8, device="cuda")
    with pytest.raises(hqa.HQAError):
        sg.solve_sub_tabu(s2, torch.ones_like(s2, dtype=torch.uint8), 4, 10, 2)
