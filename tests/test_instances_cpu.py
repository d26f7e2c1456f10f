"""CPU checks of the seeded instance generators (the one module the CUDA path and
the oracle share; it holds none of the method's arithmetic): every ensemble has
the structure its description states, and a seed fixes the instance."""
import numpy as np
import pytest

from paper_2004_03972_gb300 import instances


def _csr_checks(inst):
    """Symmetric, no diagonal, no repeated column, rows sorted; returns the dense J."""
    rp, col, val = inst.to_csr()
    assert rp[0] == 0 and rp[-1] == col.shape[0] == val.shape[0]
    for i in range(inst.N):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0), i          # sorted, no duplicates
        assert not np.any(c == i), i              # no diagonal
    J = inst.to_dense()
    assert np.array_equal(J, J.T)
    return J


@pytest.mark.parametrize("N", [5, 40])
def test_sk(N):
    inst = instances.sk_pm1(N, 3)
    J = inst.dense
    off = ~np.eye(N, dtype=bool)
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    assert set(np.unique(J[off])) == {-1.0, 1.0}
    assert inst.nnz == N * (N - 1)


def test_er_edge_count_and_weights():
    N, p = 800, 0.06
    inst = instances.er_pm1(N, p, 1200)
    J = _csr_checks(inst)
    assert set(np.unique(inst.val)) == {-1.0, 1.0}
    m, pairs = inst.nnz // 2, N * (N - 1) // 2
    mean, sd = pairs * p, np.sqrt(pairs * p * (1 - p))
    assert abs(m - mean) < 5 * sd                  # binomial edge count
    assert inst.nnz == 38322                      # the ER800 benchmark instance
    assert abs(np.mean(inst.val)) < 5 / np.sqrt(inst.nnz)
    assert np.count_nonzero(J) == inst.nnz


def test_er_mean_degree():
    inst = instances.er_mean_degree_pm1(3000, 8.0, 5)
    _csr_checks(inst)
    deg = np.diff(inst.row_ptr)
    pairs = 3000 * 2999 // 2
    p = 8.0 / 2999
    assert abs(inst.nnz // 2 - pairs * p) < 5 * np.sqrt(pairs * p * (1 - p))
    assert deg.min() >= 0 and abs(deg.mean() - 8.0) < 0.3


@pytest.mark.parametrize("N", [50, 301, 5000])
def test_regular3(N):
    inst = instances.regular3_pm1(N, 6)
    assert inst.N % 2 == 0 and inst.N in (N, N + 1)
    _csr_checks(inst)
    assert np.all(np.diff(inst.row_ptr) == 3)
    assert set(np.unique(inst.val)) <= {-1.0, 1.0}


@pytest.mark.parametrize("Lx,Ly", [(3, 3), (7, 8), (20, 15)])
def test_torus(Lx, Ly):
    inst = instances.torus_pm1(Lx, Ly, 2)
    J = _csr_checks(inst)
    assert np.all(np.diff(inst.row_ptr) == 4)
    for y in range(Ly):
        for x in range(Lx):
            i = y * Lx + x
            nb = {y * Lx + (x + 1) % Lx, y * Lx + (x - 1) % Lx,
                  ((y + 1) % Ly) * Lx + x, ((y - 1) % Ly) * Lx + x}
            assert set(np.flatnonzero(J[i])) == nb, (x, y)
    with pytest.raises(ValueError):
        instances.torus_pm1(2, 5, 1)


def test_uniform_sg():
    inst = instances.uniform_sg(300, 7)
    J, h = inst.dense, inst.h
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    assert np.all(np.abs(J) <= 1) and np.all(np.abs(h) <= 2)
    assert np.array_equal(J.astype(np.float32).astype(np.float64), J)   # exact in FP32
    assert np.array_equal(h.astype(np.float32).astype(np.float64), h)
    off = J[np.triu_indices(300, 1)]
    assert abs(off.mean()) < 5 * np.sqrt(1 / 3 / off.size)               # U[-1, 1]: var 1/3


def test_integer_field():
    inst = instances.with_integer_field(instances.er_pm1(200, 0.05, 2), 3, 4)
    assert np.all(inst.h == np.round(inst.h)) and np.abs(inst.h).max() <= 3
    assert set(np.unique(inst.h)) == {-3.0, -2.0, -1.0, 0.0, 1.0, 2.0, 3.0}


def test_uneven_batch_structure():
    batch = instances.uneven_batch(24, 200, 5000, 1400)
    assert len(batch) == 24
    for k, inst in enumerate(batch):
        deg = np.diff(inst.row_ptr)
        if k % 2 == 0:
            assert inst.meta["kind"] == "regular3" and np.all(deg == 3)
            assert 200 <= inst.N <= 5001
        else:
            assert inst.meta["kind"] == "torus" and np.all(deg == 4)
            assert 150 <= inst.N <= 5200                  # rounded to an Lx x Ly grid


def test_seed_fixes_the_instance():
    a, b = instances.er_pm1(300, 0.05, 9), instances.er_pm1(300, 0.05, 9)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)
    c = instances.er_pm1(300, 0.05, 10)
    assert not (a.col.shape == c.col.shape and np.array_equal(a.col, c.col))
    assert np.array_equal(instances.uniform_sg(50, 3).dense, instances.uniform_sg(50, 3).dense)
