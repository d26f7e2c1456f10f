"""CPU pins of the oracle's schedules, RNG, Hamiltonian, force and leapfrog.

Each check ties the oracle to something other than itself: hand-evaluated
values (tests/golden/), a closed-form oscillator period, finite differences
of the Hamiltonian, exact time reversal, and the leapfrog's second-order
convergence (Methods, "Leapfrog algorithm").
"""
import math
import os

import numpy as np
import pytest
from scipy.special import beta as beta_fn

from paper_2004_03972_gb300 import instances

GOLD = os.path.join(os.path.dirname(__file__), "golden")
# alpha = alpha_f, beta = beta_f constant in tau (rho1 = kappa1 = 1, rho2 = kappa2 = 0)
FIXED = (0.032, 1.0, 0.0, 0.05, 1.0, 0.0, 0.0)


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def test_schedule_values(orc):
    for tau, a, b in _rows("schedule_values.txt"):
        alpha, beta = orc.schedule(float(tau))
        assert alpha == pytest.approx(float(a), abs=1e-12)
        assert beta == pytest.approx(float(b), abs=1e-12)


def test_linear_gamma_schedule(orc):
    for tau in (0.0, 0.3, 1.0):
        alpha, beta = orc.schedule(tau, kind=orc.LINEAR_GAMMA)
        assert alpha == pytest.approx(0.032 * (1 - tau), abs=1e-15)
        assert beta == pytest.approx(orc.schedule(tau)[1], abs=1e-15)


def test_splitmix64_published_values(orc):
    want = [int(r[0], 16) for r in _rows("splitmix64_seed0.txt")]
    assert [orc.splitmix64_at(0, c) for c in range(3)] == want


def test_initial_momenta_are_pm1_and_balanced(orc):
    p = np.concatenate([orc.initial_momenta(7, r, 1000) for r in range(8)])
    assert set(np.unique(p)) == {-1.0, 1.0}
    assert abs(p.mean()) < 5 / math.sqrt(p.size)
    # replica streams differ
    assert not np.array_equal(orc.initial_momenta(7, 0, 64), orc.initial_momenta(7, 1, 64))


def test_random_flux_range_and_exactness(orc):
    phi = orc.initial_flux_random(3, 0, 4096)
    assert phi.min() >= -0.125 and phi.max() < 0.125
    assert np.all(phi.astype(np.float32).astype(np.float64) == phi)
    assert abs(phi.mean()) < 0.01


def test_hmd_hand_value(orc):
    want = float(_rows("hmd_two_spin.txt")[0][0])
    J = np.array([[0.0, -1.0], [-1.0, 0.0]])
    pr = orc.Problem(2, J=J, h=np.array([1.0, 2.0]))
    got = orc.hmd(pr, 0.5, np.array([0.5, -1.0]), np.array([1.0, 2.0]))
    assert got == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("dense", [True, False])
def test_force_is_minus_fd_gradient(orc, dense):
    inst = instances.with_integer_field(instances.sk_pm1(24, 11), 2, 5)
    if dense:
        pr = orc.Problem(inst.N, J=inst.dense, h=inst.h)
    else:
        rp, col, val = inst.to_csr()
        pr = orc.Problem(inst.N, row_ptr=rp, col=col, val=val, h=inst.h)
    rng = np.random.default_rng(0)
    phi = rng.uniform(-1.2, 1.2, inst.N)
    p = rng.uniform(-1, 1, inst.N)
    tau = 0.37
    F = orc.force(pr, tau, phi)
    eps = 1e-6
    fd = np.empty(inst.N)
    for i in range(inst.N):
        e = np.zeros(inst.N)
        e[i] = eps
        fd[i] = (orc.hmd(pr, tau, phi + e, p) - orc.hmd(pr, tau, phi - e, p)) / (2 * eps)
    scale = np.abs(F).max()
    assert np.max(np.abs(F - fd)) <= 1e-7 * scale


def test_single_oscillator_period_closed_form(orc):
    """beta = 0, alpha fixed: H = alpha (p^2/2 + phi^6); phi(0)=0, p(0)=1 gives period
    T = (4 a / alpha) B(1/6, 1/2) / 6 with a = 2^(-1/6) (turning point phi^6 = 1/2)."""
    alpha = 0.032
    prm = (alpha, 1.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    T = 4 * 2 ** (-1 / 6) / alpha * beta_fn(1 / 6, 1 / 2) / 6
    assert T == pytest.approx(4.32736 / alpha, rel=1e-5)
    pr = orc.Problem(1, J=np.zeros((1, 1)))
    hstep = 0.25
    S = int(6 * T / hstep)
    # sample phi at each step by running progressively (window=1 gives phi^(S) itself)
    phis = []
    for s in range(1, S + 1, 1):
        phi, _, _ = orc.md_run(pr, s, dt=1e-9, p0=np.array([1.0]), prm=prm, hstep=hstep, window=1)
        phis.append(phi[0])
        if len(phis) > 1 and s > 5 * T / hstep:
            break
    phis = np.array(phis)
    t = hstep * np.arange(1, len(phis) + 1)
    # upward zero crossings (linear interpolation)
    k = np.nonzero((phis[:-1] < 0) & (phis[1:] >= 0))[0]
    tc = t[k] + (0 - phis[k]) * hstep / (phis[k + 1] - phis[k])
    periods = np.diff(tc)
    assert len(periods) >= 3
    assert np.allclose(periods, T, rtol=2e-3)


def _fixed_run(orc, pr, p0, hstep, S, phi0=None):
    return orc.md_run(pr, S, dt=1e-9, p0=p0, phi0=phi0, prm=FIXED, hstep=hstep, window=1,
                      trace=True)


def test_energy_drift_bounded_and_scales_as_h2(orc):
    inst = instances.sk_pm1(16, 3)
    pr = orc.Problem(inst.N, J=inst.dense)
    p0 = orc.initial_momenta(1, 0, inst.N)
    T = 400.0
    drifts = []
    for hstep in (0.4, 0.2):
        S = int(T / hstep)
        _, _, _, tr = _fixed_run(orc, pr, p0, hstep, S)
        drifts.append(np.max(np.abs(tr - tr[0])) / abs(tr[0]))
    assert drifts[0] < 5e-2
    ratio = drifts[0] / drifts[1]
    assert 3.0 < ratio < 5.5  # O(h^2): halving h quarters the energy error


def test_time_reversal(orc):
    inst = instances.with_integer_field(instances.sk_pm1(12, 8), 1, 2)
    pr = orc.Problem(inst.N, J=inst.dense, h=inst.h)
    p0 = orc.initial_momenta(5, 0, inst.N)
    phi0 = orc.initial_flux_random(5, 0, inst.N) * 4
    hstep, S = 0.3, 500
    phiS, pS_half, _ = orc.md_run(pr, S, dt=1e-9, p0=p0, phi0=phi0, prm=FIXED, hstep=hstep,
                                  window=1)
    # complete the last half kick to get p at the integer step S, then reverse
    pS = pS_half - 0.5 * hstep * orc.force(pr, 0.0, phiS, prm=FIXED)
    phiB, pB_half, _ = orc.md_run(pr, S, dt=1e-9, p0=-pS, phi0=phiS, prm=FIXED, hstep=hstep,
                                  window=1)
    pB = pB_half - 0.5 * hstep * orc.force(pr, 0.0, phiB, prm=FIXED)
    assert np.max(np.abs(phiB - phi0)) < 1e-10
    assert np.max(np.abs(-pB - p0)) < 1e-10


def test_second_order_convergence(orc):
    """Global error of the leapfrog at fixed end time falls as h^2 (Methods)."""
    inst = instances.sk_pm1(10, 4)
    pr = orc.Problem(inst.N, J=inst.dense)
    p0 = orc.initial_momenta(2, 0, inst.N)
    T = 60.0
    ref, _, _ = orc.md_run(pr, int(T / 0.0125), dt=1e-9, p0=p0, prm=FIXED, hstep=0.0125, window=1)
    errs = []
    for hstep in (0.2, 0.1):
        phi, _, _ = orc.md_run(pr, int(T / hstep), dt=1e-9, p0=p0, prm=FIXED, hstep=hstep, window=1)
        errs.append(np.max(np.abs(phi - ref)))
    assert 3.0 < errs[0] / errs[1] < 5.5


def test_beta_zero_decouples_spins(orc):
    inst = instances.sk_pm1(8, 1)
    prm = (0.02, 1.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    pr = orc.Problem(inst.N, J=inst.dense)
    p0 = orc.initial_momenta(9, 0, inst.N)
    phi, p, _ = orc.md_run(pr, 300, p0=p0, prm=prm)
    single = orc.Problem(1, J=np.zeros((1, 1)))
    for i in range(inst.N):
        phi1, p1, _ = orc.md_run(single, 300, p0=p0[i:i + 1], prm=prm)
        assert phi1[0] == phi[i] and p1[0] == p[i]


def test_window_mean_definition(orc):
    """With W = 1 the window mean is phi^(S); with W >= S it averages phi^(1..S)."""
    inst = instances.sk_pm1(6, 2)
    pr = orc.Problem(inst.N, J=inst.dense)
    p0 = orc.initial_momenta(4, 0, inst.N)
    phis = [orc.md_run(pr, s, dt=1 / 40, p0=p0, window=1)[0] for s in range(1, 11)]
    # dt fixed so the s-step runs are prefixes of one trajectory
    _, _, pbar = orc.md_run(pr, 10, dt=1 / 40, p0=p0, window=100)
    assert np.allclose(pbar, np.mean(phis, axis=0), rtol=0, atol=1e-15)
    _, _, pbar4 = orc.md_run(pr, 10, dt=1 / 40, p0=p0, window=4)
    assert np.allclose(pbar4, np.mean(phis[6:], axis=0), rtol=0, atol=1e-15)


def test_first_half_kick_with_zero_flux_keeps_momenta(orc):
    """phi(0) = 0 and S = 1: p^(1/2) = p^(0) exactly (V'(0) = 0, field 0)."""
    inst = instances.sk_pm1(20, 6)
    pr = orc.Problem(inst.N, J=inst.dense)
    p0 = orc.initial_momenta(1, 3, inst.N)
    phi, p, _ = orc.md_run(pr, 1, p0=p0)
    alpha_half, _ = orc.schedule(0.5)
    assert np.array_equal(p, p0)
    assert np.allclose(phi, alpha_half * p0, rtol=1e-15)


def test_replica_driver_equals_single_runs(orc):
    """The OpenMP replica driver (the CPU baseline and reference arm) runs each
    replica's trajectory on its own: the same bits as md_run per replica, at one
    thread and at several, from paper and from random initial fluxes."""
    inst = instances.with_integer_field(instances.er_pm1(90, 0.1, 7), 2, 8)
    pr = orc.Problem.from_instance(inst)
    R, S = 5, 60
    p0 = np.stack([orc.initial_momenta(11, r, inst.N) for r in range(R)])
    phi0 = np.stack([orc.initial_flux_random(11, r, inst.N) for r in range(R)])
    for start in (np.zeros_like(p0), phi0):
        runs = [orc.md_run_replicas(pr, S, start, p0, threads=t) for t in (1, 4)]
        for r in range(R):
            one = orc.md_run(pr, S, phi0=start[r], p0=p0[r])
            for t in range(2):
                for k in range(3):
                    assert np.array_equal(runs[t][k][r], one[k]), (r, t, k)


def test_table_schedule_hand_value(orc):
    """The TABLE kind's index conventions (alpha at k = 2m for the kick and 2m + 1 for
    the drift, beta at m), against three steps worked by hand in exact fractions."""
    want = {r[0]: [int(r[1]) / int(r[2]), int(r[3]) / int(r[4])]
            for r in _rows("table_schedule_3step.txt")}
    ta = np.array([1 / 2, 1 / 4, 1 / 8, 1 / 2, 1 / 4, 1 / 16, 1.0])
    tb = np.array([1.0, 1 / 2, 1 / 4, 1 / 8])
    pr = orc.Problem(2, J=np.array([[0.0, -1.0], [-1.0, 0.0]]))
    phi, p, pbar = orc.md_run(pr, 3, dt=1.0, p0=np.array([1.0, 0.5]), kind=orc.TABLE, M=2,
                              window=2, table_alpha=ta, table_beta=tb)
    assert phi.tolist() == want["phi"]
    assert p.tolist() == want["p"]
    assert pbar.tolist() == want["phibar"]


def test_table_sampled_from_paper_schedule_reproduces_paper_run(orc):
    """A table holding the paper's polynomials on the half-step grid (alpha at
    tau = k dt / 2, beta at tau = m dt) gives the PAPER-kind trajectory bitwise."""
    inst = instances.with_integer_field(instances.er_pm1(60, 0.1, 4), 1, 2)
    pr = orc.Problem.from_instance(inst)
    S, dt = 150, 1.0 / 150
    ta = np.array([orc.schedule(0.5 * k * dt)[0] for k in range(2 * S + 1)])
    tb = np.array([orc.schedule(m * dt)[1] for m in range(S + 1)])
    p0 = orc.initial_momenta(5, 0, inst.N)
    a = orc.md_run(pr, S, dt=dt, p0=p0, window=40)
    b = orc.md_run(pr, S, dt=dt, p0=p0, window=40, kind=orc.TABLE, table_alpha=ta,
                   table_beta=tb)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # a table that differs from the paper's at one half-step index changes the run
    ta2 = ta.copy()
    ta2[2 * 70 + 1] *= 1.5
    c = orc.md_run(pr, S, dt=dt, p0=p0, window=40, kind=orc.TABLE, table_alpha=ta2,
                   table_beta=tb)
    assert not np.array_equal(a[0], c[0])


@pytest.mark.parametrize("field", [False, True])
def test_dense_batch_oracle_equals_per_replica_oracle(orc, field):
    """The batched dense form (one FP64 matrix product per step for all replicas)
    follows the per-replica C routine to rounding: same schedule indices, half
    first kick, window and field term."""
    inst = instances.uniform_sg(90, 3) if field else instances.sk_pm1(90, 3)
    pr = orc.Problem.from_instance(inst)
    R, S = 5, 300
    p0 = np.stack([orc.initial_momenta(9, r, inst.N) for r in range(R)])
    phi0 = np.stack([orc.initial_flux_random(9, r, inst.N) for r in range(R)])
    a = orc.md_run_dense_batch(pr, S, phi0, p0, dt=1.0 / 400, window=30)
    b = orc.md_run_replicas(pr, S, phi0, p0, dt=1.0 / 400, window=30)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-9 * max(1.0, np.max(np.abs(y)))
