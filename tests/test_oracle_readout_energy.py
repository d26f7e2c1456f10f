"""CPU pins of the oracle's readout, integer energy, cut and exact sub-solve.

Independent routes: numpy's lexsort for the rank split, numpy matrix
products for Eq. (1), the edge-sum vs. C_0 forms of the cut (Methods,
"MAX-CUT and Ising spin-glass"), exhaustive numpy enumeration for the
ground state, and the identity H(s) = H'(s_amb) + const of Eq. (6).
"""
import itertools

import numpy as np
import pytest

from paper_2004_03972_gb300 import instances


def _np_energy(J, h, s):
    s = s.astype(np.float64)
    e = 0.5 * s @ J @ s
    if h is not None:
        e += h @ s
    return int(round(e))


def test_readout_hand_cases(orc):
    phibar = np.array([0.5, -0.1, 0.0, 0.1, -0.5, 2.0])
    s, f = orc.readout(phibar, 3)
    assert s.tolist() == [1, -1, 1, 1, -1, 1]          # sgn(0) = +1
    # order by (|phibar|, index): 2 (0.0), 1 (0.1), 3 (0.1), 0 (0.5), 4 (0.5), 5
    assert f.tolist() == [1, 0, 0, 0, 1, 1]
    assert orc.readout(phibar, 0)[1].tolist() == [1] * 6
    assert orc.readout(phibar, 99)[1].tolist() == [0] * 6
    assert orc.readout(phibar, -3)[1].tolist() == [1] * 6


def test_readout_matches_lexsort(orc):
    rng = np.random.default_rng(1)
    phibar = np.round(rng.normal(size=500), 2)   # many exact ties
    n = 137
    s, f = orc.readout(phibar, n)
    order = np.lexsort((np.arange(500), np.abs(phibar)))
    want = np.ones(500, np.uint8)
    want[order[:n]] = 0
    assert np.array_equal(f, want)
    assert np.array_equal(s, np.where(phibar >= 0, 1, -1).astype(np.int8))


@pytest.mark.parametrize("kind", ["sk", "er", "torus"])
def test_energy_matches_matrix_form(orc, kind):
    if kind == "sk":
        inst = instances.with_integer_field(instances.sk_pm1(60, 2), 3, 1)
    elif kind == "er":
        inst = instances.with_integer_field(instances.er_pm1(120, 0.1, 3), 2, 4)
    else:
        inst = instances.torus_pm1(7, 5, 9)
    J = inst.to_dense()
    pr = orc.Problem.from_instance(inst)
    rng = np.random.default_rng(0)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], np.int8), size=inst.N)
        assert orc.energy_int(pr, s) == _np_energy(J, inst.h, s)


@pytest.mark.parametrize("kind", ["sk", "er"])
def test_cut_identity(orc, kind):
    """C(s) = -H(s)/2 + C_0 with C_0 = 1/4 sum_{i != j} J_ij (h = 0)."""
    inst = instances.sk_pm1(50, 5) if kind == "sk" else instances.er_pm1(90, 0.2, 6)
    J = inst.to_dense()
    pr = orc.Problem.from_instance(inst)
    twice_c0 = int(round(J.sum())) // 2          # 2 C_0 = 1/2 sum_{i != j} J_ij
    rng = np.random.default_rng(2)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], np.int8), size=inst.N)
        c = orc.cut_int(pr, s)
        e = orc.energy_int(pr, s)
        assert 2 * c == -e + twice_c0
        # C counts the weight of edges across the partition
        cross = sum(J[i, j] for i in range(inst.N) for j in range(i + 1, inst.N) if s[i] != s[j])
        assert c == int(round(cross))


def test_cut_dense_equals_csr(orc):
    inst = instances.sk_pm1(40, 1)
    rp, col, val = inst.to_csr()
    s = np.random.default_rng(0).choice(np.array([-1, 1], np.int8), size=40)
    a = orc.cut_int(orc.Problem(40, J=inst.dense), s)
    b = orc.cut_int(orc.Problem(40, row_ptr=rp, col=col, val=val), s)
    assert a == b


def _np_ground_state(J, h):
    N = J.shape[0]
    xs = np.arange(2 ** N, dtype=np.int64)
    S = np.where((xs[:, None] >> np.arange(N)) & 1, -1.0, 1.0)
    E = 0.5 * np.einsum("ki,ij,kj->k", S, J, S)
    if h is not None:
        E += S @ h
    E = np.round(E).astype(np.int64)
    k = int(np.argmin(E))      # argmin returns the first (smallest x) minimum
    return int(E[k]), k


@pytest.mark.parametrize("N,seed", [(10, 1), (12, 2), (14, 3)])
def test_brute_force_matches_numpy(orc, N, seed):
    inst = instances.with_integer_field(instances.sk_pm1(N, seed), 1, seed)
    pr = orc.Problem.from_instance(inst)
    assert orc.brute_force(pr) == _np_ground_state(inst.dense, inst.h)


def test_brute_force_z2_degenerate_picks_smallest_x(orc):
    inst = instances.sk_pm1(10, 7)   # h = 0: s and -s are both optimal
    e, x = orc.brute_force(orc.Problem.from_instance(inst))
    assert x < (1 << 9)              # the copy with s_9 = +1 comes first


def test_subsolve_all_ambivalent_equals_brute_force(orc):
    inst = instances.with_integer_field(instances.er_pm1(14, 0.4, 3), 1, 3)
    pr = orc.Problem.from_instance(inst)
    frozen = np.zeros(14, np.uint8)
    spins = np.ones(14, np.int8)
    out, e, x, emin = orc.subsolve(pr, spins, frozen)
    eb, xb = orc.brute_force(pr)
    assert (e, x, emin) == (eb, xb, eb)


def test_subsolve_reduced_problem_identity(orc):
    """H(s) restricted to the ambivalent set = H'(s_amb) + const (Eq. (6)); the
    sub-solve optimum equals exhaustive search of the full energy over the
    ambivalent spins with the frozen ones held."""
    inst = instances.with_integer_field(instances.sk_pm1(30, 4), 2, 8)
    J = inst.dense
    pr = orc.Problem.from_instance(inst)
    rng = np.random.default_rng(3)
    spins = rng.choice(np.array([-1, 1], np.int8), size=30)
    frozen = np.ones(30, np.uint8)
    amb = np.sort(rng.choice(30, size=9, replace=False))
    frozen[amb] = 0
    out, e, x, emin = orc.subsolve(pr, spins, frozen)
    best, bx, consts = None, None, set()
    for xx in range(2 ** 9):
        s = spins.copy()
        for k, a in enumerate(amb):
            s[a] = -1 if (xx >> k) & 1 else 1
        full = _np_energy(J, inst.h, s)
        # H'(s_amb) from the definition of J_eff, h_eff
        sa = s[amb].astype(np.int64)
        Jab = J[np.ix_(amb, amb)]
        fro = np.nonzero(frozen)[0]
        heff = inst.h[amb] + J[np.ix_(amb, fro)] @ spins[fro]
        red = 0.5 * sa @ Jab @ sa + heff @ sa
        consts.add(int(round(full - red)))
        if best is None or full < best:
            best, bx = full, xx
    assert len(consts) == 1
    assert (e, x) == (best, bx)
    assert emin == best - consts.pop()
    assert np.array_equal(out[frozen == 1], spins[frozen == 1])


def test_readout_cut_never_beats_optimum(orc):
    """Any readout assignment is a feasible cut, so it cannot exceed the brute-force maximum."""
    inst = instances.sk_pm1(16, 12)
    pr = orc.Problem.from_instance(inst)
    e_opt, _ = orc.brute_force(pr)
    J = inst.dense
    twice_c0 = int(round(J.sum())) // 2
    c_opt = (-e_opt + twice_c0) // 2
    for r in range(4):
        p0 = orc.initial_momenta(100, r, 16)
        _, _, pbar = orc.md_run(pr, 2000, p0=p0)
        s, _ = orc.readout(pbar, 0)
        assert orc.cut_int(pr, s) <= c_opt
        assert orc.energy_int(pr, s) >= e_opt


def test_energy_f64_pins(orc):
    """FP64 energy for real couplings: equals the int64 energy on integer instances;
    Z2 symmetry at h = 0; flipping spin k changes it by -2 s_k (sum_j J_kj s_j + h_k),
    with the field sum from the independent beta_field routine (which adds 2 h |s|)."""
    from paper_2004_03972_gb300 import instances
    ints = instances.with_integer_field(instances.er_pm1(90, 0.1, 4), 3, 5)
    pr = orc.Problem.from_instance(ints)
    rng = np.random.default_rng(0)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], np.int8), size=ints.N)
        assert orc.energy_f64(pr, s) == float(orc.energy_int(pr, s))
    sg = instances.uniform_sg(70, 3)
    pg = orc.Problem.from_instance(sg)
    p0 = orc.Problem(sg.N, J=sg.dense)          # h = 0
    s = rng.choice(np.array([-1, 1], np.int8), size=sg.N)
    assert orc.energy_f64(p0, s) == pytest.approx(orc.energy_f64(p0, -s), rel=1e-14, abs=1e-12)
    e = orc.energy_f64(pg, s)
    g = orc.beta_field(pg, s.astype(np.float64)) - 2.0 * sg.h     # sum_j J_kj s_j
    for k in (0, 17, 69):
        t = s.copy()
        t[k] = -t[k]
        assert orc.energy_f64(pg, t) - e == pytest.approx(-2.0 * s[k] * (g[k] + sg.h[k]), abs=1e-9)
