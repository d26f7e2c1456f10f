"""GPU exact sub-solve (HQA section, Eqs. (6)-(7)) bit-exact against the oracle."""
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


def _masks(N, R, n, rng):
    frozen = np.ones((R, N), np.uint8)
    for r in range(R):
        frozen[r, rng.choice(N, size=n, replace=False)] = 0
    return frozen


@pytest.mark.parametrize("inst_name,n,R", [
    ("er", 0, 3), ("er", 1, 3), ("er", 3, 5), ("er", 12, 7), ("sk", 16, 4), ("er_h", 20, 3),
    ("torus", 9, 2)])
def test_subsolve_bit_exact(hqa, orc, inst_name, n, R):
    if inst_name == "er":
        inst = instances.er_pm1(200, 0.08, 3)
    elif inst_name == "sk":
        inst = instances.sk_pm1(64, 5)
    elif inst_name == "torus":
        inst = instances.torus_pm1(6, 7, 1)
    else:
        inst = instances.with_integer_field(instances.er_pm1(150, 0.1, 8), 3, 2)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(n + R)
    spins = rng.choice(np.array([-1, 1], np.int8), size=(R, inst.N))
    frozen = _masks(inst.N, R, n, rng)
    out, e = ctx.solve_sub(torch.from_numpy(spins).cuda(), torch.from_numpy(frozen).cuda(), n)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in range(R):
        ws, we, _, _ = orc.subsolve(pr, spins[r], frozen[r])
        assert np.array_equal(out[r].cpu().numpy(), ws)
        assert int(e[r]) == we


def test_subsolve_packed_and_scalar_walks_mixed(hqa, orc):
    """Replicas whose reduced energies fit in 16 bits take the packed four-lane walk,
    the others (here: spins with fields of 20000 in the ambivalent set) the scalar
    walk; both in one call, bit-exact against the oracle."""
    base = instances.er_pm1(150, 0.1, 8)
    rng = np.random.default_rng(77)
    h = np.zeros(base.N)
    big = rng.choice(base.N, size=15, replace=False)
    h[big] = rng.choice([-20000.0, 20000.0], size=15)
    inst = instances.Instance(base.name + "_bigh", base.N, None, base.row_ptr, base.col,
                              base.val, h, dict(base.meta))
    ctx = hqa.Context.from_instance(inst)
    R, n = 16, 8
    spins = rng.choice(np.array([-1, 1], np.int8), size=(R, inst.N))
    frozen = _masks(inst.N, R, n, rng)
    has_big = [bool(np.any(frozen[r, big] == 0)) for r in range(R)]
    assert any(has_big) and not all(has_big)
    out, e = ctx.solve_sub(torch.from_numpy(spins).cuda(), torch.from_numpy(frozen).cuda(), n)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in range(R):
        ws, we, _, _ = orc.subsolve(pr, spins[r], frozen[r])
        assert np.array_equal(out[r].cpu().numpy(), ws)
        assert int(e[r]) == we


def test_subsolve_n24_bit_exact(hqa, orc):
    """The configuration-5 sub-problem size: n = 24 (2^24 assignments)."""
    inst = instances.er_mean_degree_pm1(1000, 8.0, 11)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(24)
    R, n = 2, 24
    spins = rng.choice(np.array([-1, 1], np.int8), size=(R, inst.N))
    # ambivalent set drawn from a connected neighbourhood so J_eff is not empty
    frozen = np.ones((R, inst.N), np.uint8)
    for r in range(R):
        seen, front = [], [int(rng.integers(inst.N))]
        while len(seen) < n and front:
            v = front.pop(0)
            if v in seen:
                continue
            seen.append(v)
            front += inst.col[inst.row_ptr[v]:inst.row_ptr[v + 1]].tolist()
        while len(seen) < n:
            v = int(rng.integers(inst.N))
            if v not in seen:
                seen.append(v)
        frozen[r, seen] = 0
    out, e = ctx.solve_sub(torch.from_numpy(spins).cuda(), torch.from_numpy(frozen).cuda(), n)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in range(R):
        ws, we, _, _ = orc.subsolve(pr, spins[r], frozen[r])
        assert np.array_equal(out[r].cpu().numpy(), ws)
        assert int(e[r]) == we


def test_subsolve_all_ambivalent_is_ground_state(hqa, orc):
    inst = instances.sk_pm1(18, 9)
    ctx = hqa.Context.from_instance(inst)
    spins = np.ones((1, 18), np.int8)
    frozen = np.zeros((1, 18), np.uint8)
    out, e = ctx.solve_sub(torch.from_numpy(spins).cuda(), torch.from_numpy(frozen).cuda(), 18)
    ctx.sync()
    eb, xb = orc.brute_force(orc.Problem.from_instance(inst))
    assert int(e[0]) == eb
    want = np.array([-1 if (xb >> i) & 1 else 1 for i in range(18)], np.int8)
    assert np.array_equal(out[0].cpu().numpy(), want)


def test_subsolve_rejects_oversized_replica(hqa):
    inst = instances.er_pm1(100, 0.1, 1)
    ctx = hqa.Context.from_instance(inst)
    spins = torch.ones((2, 100), dtype=torch.int8, device="cuda")
    frozen = torch.ones((2, 100), dtype=torch.uint8, device="cuda")
    frozen[1, :10] = 0          # 10 ambivalent spins but n = 5
    out, e = ctx.solve_sub(spins, frozen, 5)
    with pytest.raises(hqa.HQAError):
        ctx.sync()
    with pytest.raises(hqa.HQAError):
        ctx.solve_sub(spins, frozen, 31)
