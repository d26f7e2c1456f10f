"""CPU pins of the oracle's tabu-search sub-solve (large ambivalent sets, where the
exact enumeration is out of reach):
  * no iterations: the input assignment comes back
  * one ambivalent spin, no tenure, one iteration: the better of s and its flip
  * it never returns an energy below the exact optimum (brute force, n <= 10), nor
    above the input's, never touches a frozen spin, and reports the energy of what
    it returns
  * with enough iterations on small sets it reaches the exact optimum
  * a hand-traced trajectory (tests/golden/tabu_triangle.txt): the uphill escape
    from a local minimum, the smallest-index tie-break, the tabu expiry
    until < it, the strict aspiration, and the cycling of tenure 0
"""
import os

import numpy as np
import pytest

from paper_2004_03972_gb300 import instances

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tabu_triangle.txt")


def test_hand_traced_triangle(orc):
    J = -np.ones((3, 3)) + np.eye(3)
    inst = instances.Instance("triangle", 3, dense=J, h=np.ones(3))
    pr = orc.Problem.from_instance(inst)
    s = np.ones(3, np.int8)
    f = np.zeros(3, np.uint8)
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 6
    for tenure, iters, e_best, spins in rows:
        out, e = orc.subsolve_tabu(pr, s, f, int(iters), int(tenure))
        assert e == int(e_best), (tenure, iters)
        assert out.tolist() == [int(v) for v in spins.split(",")], (tenure, iters)


def _case(orc, seed, N=120, n=8):
    inst = instances.with_integer_field(instances.er_pm1(N, 0.08, seed), 2, seed + 1)
    pr = orc.Problem.from_instance(inst)
    rng = np.random.default_rng(seed)
    s = rng.choice(np.array([-1, 1], np.int8), size=N)
    frozen = np.ones(N, np.uint8)
    frozen[rng.choice(N, size=n, replace=False)] = 0
    return inst, pr, s, frozen


def test_zero_iterations_return_the_input(orc):
    inst, pr, s, f = _case(orc, 1)
    out, e = orc.subsolve_tabu(pr, s, f, 0, 3)
    assert np.array_equal(out, s) and e == orc.energy_int(pr, s)


def test_single_spin_one_iteration(orc):
    inst, pr, s, f = _case(orc, 2, n=1)
    out, e = orc.subsolve_tabu(pr, s, f, 1, 0)
    a = int(np.flatnonzero(f == 0)[0])
    t = s.copy()
    t[a] = -t[a]
    assert e == min(orc.energy_int(pr, s), orc.energy_int(pr, t))


@pytest.mark.parametrize("seed", [3, 4, 5, 6])
def test_bounds_and_consistency(orc, seed):
    inst, pr, s, f = _case(orc, seed, n=10)
    out, e = orc.subsolve_tabu(pr, s, f, 15, 2)
    exact, e_opt, _, _ = orc.subsolve(pr, s, f)
    assert e_opt <= e <= orc.energy_int(pr, s)
    assert e == orc.energy_int(pr, out)
    assert np.array_equal(out[f == 1], s[f == 1])


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_reaches_the_optimum_on_small_sets(orc, seed):
    inst, pr, s, f = _case(orc, seed, n=8)
    _, e = orc.subsolve_tabu(pr, s, f, 400, 3)
    _, e_opt, _, _ = orc.subsolve(pr, s, f)
    assert e == e_opt
