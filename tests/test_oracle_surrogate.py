"""CPU pins of the oracle's surrogate-gate routines (features of a trajectory prefix
and the confidence readout; the paper has no learned part, so these are pinned by
reductions to the paper's routines and by invariants):
  * one segment: the features reduce to (phi, p, L(phi), 0, phibar, 0) of one md_run
  * Z2 at h = 0: negating the initial momenta negates phi, p, mean L and phibar and
    leaves var L and the flip fraction unchanged (bitwise: the dynamics is odd)
  * z-scored columns have mean 0 and variance 1 (or are 0 when constant)
  * sigma(z_f) = 1: the readout is the method's readout applied to z_s
  * z_s = 0: every frozen spin counts 1/2 expected error
"""
import numpy as np
import pytest

from paper_2004_03972_gb300 import instances


def _pr(orc, inst):
    return orc.Problem.from_instance(inst)


def test_segment_lengths(orc):
    assert orc.segment_lengths(103, 5) == [21, 21, 21, 20, 20]
    assert sum(orc.segment_lengths(1000, 7)) == 1000
    assert orc.segment_lengths(4, 4) == [1, 1, 1, 1]


def test_one_segment_reduces_to_md_run(orc):
    inst = instances.er_pm1(60, 0.1, 3)
    pr = _pr(orc, inst)
    p0 = orc.initial_momenta(9, 0, inst.N)
    f = orc.surrogate_features_raw(pr, 37, 1, p0, dt=1e-3, window=10)
    phi, p, pbar = orc.md_run(pr, 37, dt=1e-3, p0=p0, window=10)
    J = inst.to_dense()
    np.testing.assert_array_equal(f[:, 0], phi)
    np.testing.assert_array_equal(f[:, 1], p)
    np.testing.assert_allclose(f[:, 2], J @ phi, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(f[:, 3], 0.0)
    np.testing.assert_array_equal(f[:, 4], pbar)
    np.testing.assert_array_equal(f[:, 5], 0.0)


def test_segment_samples_are_prefix_states(orc):
    """mean L and var L over three segment ends equal those of the three states
    computed by separate runs of 10, 20 and 30 steps; the flip fraction counts sign
    changes between them."""
    inst = instances.torus_pm1(6, 7, 1)
    pr = _pr(orc, inst)
    p0 = orc.initial_momenta(4, 2, inst.N)
    f = orc.surrogate_features_raw(pr, 30, 3, p0, dt=1e-2, window=100)
    J = inst.to_dense()
    states = [orc.md_run(pr, m, dt=1e-2, p0=p0)[0] for m in (10, 20, 30)]
    L = np.array([J @ s for s in states])
    np.testing.assert_allclose(f[:, 2], L.mean(0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(f[:, 3], L.var(0), rtol=1e-9, atol=1e-14)
    sg = np.where(np.array(states) >= 0, 1, -1)
    np.testing.assert_array_equal(f[:, 5], (sg[1:] != sg[:-1]).sum(0) / 2)
    # the last window covers the last segment only (10 steps): not the same as 30 steps
    pb10 = orc.md_run(pr, 30, dt=1e-2, p0=p0, window=10)[2]
    np.testing.assert_array_equal(f[:, 4], pb10)


def test_z2_covariance(orc):
    inst = instances.er_pm1(50, 0.12, 8)
    pr = _pr(orc, inst)
    p0 = orc.initial_momenta(2, 1, inst.N)
    a = orc.surrogate_features_raw(pr, 400, 8, p0, dt=2e-3, window=7)
    b = orc.surrogate_features_raw(pr, 400, 8, -p0, dt=2e-3, window=7)
    for k in (0, 1, 2, 4):
        np.testing.assert_array_equal(b[:, k], -a[:, k])
    np.testing.assert_array_equal(b[:, 3], a[:, 3])
    # sgn(0) = +1 breaks the symmetry only for a flux that is exactly zero
    nz = np.all(a[:, [0]] != 0, axis=1)
    np.testing.assert_array_equal(b[nz, 5], a[nz, 5])
    assert a[:, 5].max() > 0          # the prefix does see sign changes


def test_zscore_moments(orc):
    rng = np.random.default_rng(0)
    f = rng.normal(size=(500, 6)) * [1, 2, 3, 4, 5, 6] + [0, 1, -2, 3, 7, 0]
    f[:, 5] = 0.25
    z = orc.zscore(f)
    np.testing.assert_allclose(z[:, :5].mean(0), 0, atol=1e-12)
    np.testing.assert_allclose(z[:, :5].var(0), 1, rtol=1e-12)
    np.testing.assert_array_equal(z[:, 5], 0)


def test_readout_reduces_to_method_readout(orc):
    rng = np.random.default_rng(5)
    zs = rng.normal(size=300)
    logits = np.stack([np.full(300, 60.0), zs], axis=1)     # sigma(z_f) = 1 in FP64
    s, f, _, _ = orc.surrogate_readout(logits, 17, 1.0)
    # |2 sigma(z) - 1| = tanh(|z| / 2) is increasing in |z|: the same order as |z_s|
    rs, rf = orc.readout(zs, 17)
    np.testing.assert_array_equal(s, rs)
    np.testing.assert_array_equal(f, rf)


def test_readout_expected_errors(orc):
    logits = np.zeros((40, 2))
    s, f, acc, E = orc.surrogate_readout(logits, 6, 16.9)
    assert np.all(s == 1) and f.sum() == 34
    assert E == 17.0 and not acc
    assert orc.surrogate_readout(logits, 6, 17.0)[2]
    big = np.tile([[30.0, 40.0]], (40, 1))
    assert orc.surrogate_readout(big, 0, 1e-12)[3] < 1e-12
