"""Seeded synthetic problem instances (inputs only; none of the method's arithmetic).

Both the CUDA library's tests and the CPU oracle take their couplings from
here.  The paper's workloads are random ensembles described in words, so
every instance is drawn from the stated distribution with a numpy PCG64
generator seeded by the caller:

* ``sk_pm1``      -- all-to-all K_N with bimodal weights J_ij = +-1, zero
                     diagonal, h = 0 (the K2000 MAX-CUT ensemble, Results
                     "HQA for MAX-CUT problem"; Methods "MAX-CUT and Ising
                     spin-glass").
* ``er_pm1``      -- Erdos-Renyi G(N, p) with +-1 weights, stored as CSR.
* ``regular3_pm1``-- random 3-regular graph (pairing model with rejection).
* ``torus_pm1``   -- Lx x Ly periodic grid, +-1 weights.
* ``uniform_sg``  -- J_ij ~ U[-1, 1], h_i ~ U[-2, 2] (the spin-glass
                     ensemble of Results "HQA for Ising spin-glass problem");
                     real-valued, so the integer energy path does not apply.

All couplings are symmetric with an empty diagonal.  CSR rows are sorted by
column.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    name: str
    N: int
    dense: np.ndarray | None = None      # float64 [N, N] or None
    row_ptr: np.ndarray | None = None    # int64 [N + 1]
    col: np.ndarray | None = None        # int32 [nnz]
    val: np.ndarray | None = None        # float32 [nnz]
    h: np.ndarray | None = None          # float64 [N] or None (h = 0)
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        if self.row_ptr is not None:
            return int(self.row_ptr[-1])
        return int(np.count_nonzero(self.dense))

    def to_dense(self) -> np.ndarray:
        if self.dense is not None:
            return self.dense
        J = np.zeros((self.N, self.N), np.float64)
        rows = np.repeat(np.arange(self.N), np.diff(self.row_ptr))
        J[rows, self.col] = self.val
        return J

    def to_csr(self):
        if self.row_ptr is not None:
            return self.row_ptr, self.col, self.val
        return dense_to_csr(self.dense)


def dense_to_csr(J: np.ndarray):
    N = J.shape[0]
    nz = J != 0
    np.fill_diagonal(nz, False)
    counts = nz.sum(axis=1)
    row_ptr = np.zeros(N + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    rows, cols = np.nonzero(nz)
    return row_ptr, cols.astype(np.int32), J[rows, cols].astype(np.float32)


def _edges_to_csr(N: int, i: np.ndarray, j: np.ndarray, w: np.ndarray):
    """Undirected edge list (i != j, no duplicates) -> symmetric CSR sorted by column."""
    rows = np.concatenate([i, j])
    cols = np.concatenate([j, i])
    vals = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(N + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=N), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals.astype(np.float32)


def _pm1(rng, size):
    return np.where(rng.integers(0, 2, size=size) == 1, 1.0, -1.0)


def sk_pm1(N: int, seed: int) -> Instance:
    rng = np.random.Generator(np.random.PCG64(seed))
    upper = np.triu(_pm1(rng, (N, N)), k=1)
    J = upper + upper.T
    return Instance(f"sk_pm1_N{N}_s{seed}", N, dense=J, meta={"kind": "sk", "seed": seed})


def er_pm1(N: int, p: float, seed: int) -> Instance:
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(N, k=1)
    keep = rng.random(iu.shape[0]) < p
    i, j = iu[keep], ju[keep]
    w = _pm1(rng, i.shape[0])
    row_ptr, col, val = _edges_to_csr(N, i, j, w)
    return Instance(f"er_pm1_N{N}_p{p}_s{seed}", N, row_ptr=row_ptr, col=col, val=val,
                    meta={"kind": "er", "p": p, "seed": seed})


def er_mean_degree_pm1(N: int, mean_degree: float, seed: int) -> Instance:
    """G(N, p) with p = d/(N-1), drawn edge-by-edge without an N^2 table (large N)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = mean_degree / (N - 1)
    m_total = N * (N - 1) // 2
    m = rng.binomial(m_total, p)
    # sample m distinct unordered pairs uniformly
    chosen = set()
    out_i, out_j = [], []
    while len(out_i) < m:
        k = m - len(out_i)
        a = rng.integers(0, N, size=2 * k)
        b = rng.integers(0, N, size=2 * k)
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            key = (x, y) if x < y else (y, x)
            if key in chosen:
                continue
            chosen.add(key)
            out_i.append(key[0])
            out_j.append(key[1])
            if len(out_i) == m:
                break
    i = np.asarray(out_i, np.int64)
    j = np.asarray(out_j, np.int64)
    w = _pm1(rng, i.shape[0])
    row_ptr, col, val = _edges_to_csr(N, i, j, w)
    return Instance(f"er_pm1_N{N}_d{mean_degree}_s{seed}", N, row_ptr=row_ptr, col=col, val=val,
                    meta={"kind": "er", "mean_degree": mean_degree, "seed": seed})


def regular3_pm1(N: int, seed: int) -> Instance:
    """Random 3-regular simple graph by the pairing (configuration) model with rejection."""
    if N % 2:
        N += 1
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(10000):
        stubs = rng.permutation(np.repeat(np.arange(N), 3))
        a, b = stubs[0::2], stubs[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo.astype(np.int64) * N + hi
        if np.unique(key).shape[0] != key.shape[0]:
            continue
        w = _pm1(rng, lo.shape[0])
        row_ptr, col, val = _edges_to_csr(N, lo, hi, w)
        return Instance(f"reg3_pm1_N{N}_s{seed}", N, row_ptr=row_ptr, col=col, val=val,
                        meta={"kind": "regular3", "seed": seed})
    raise RuntimeError("pairing model did not produce a simple graph")


def torus_pm1(Lx: int, Ly: int, seed: int) -> Instance:
    if Lx < 3 or Ly < 3:
        raise ValueError("torus sides must be >= 3")
    rng = np.random.Generator(np.random.PCG64(seed))
    N = Lx * Ly
    idx = np.arange(N).reshape(Ly, Lx)
    right = np.roll(idx, -1, axis=1)
    down = np.roll(idx, -1, axis=0)
    i = np.concatenate([idx.ravel(), idx.ravel()])
    j = np.concatenate([right.ravel(), down.ravel()])
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    w = _pm1(rng, lo.shape[0])
    row_ptr, col, val = _edges_to_csr(N, lo, hi, w)
    return Instance(f"torus_pm1_{Lx}x{Ly}_s{seed}", N, row_ptr=row_ptr, col=col, val=val,
                    meta={"kind": "torus", "seed": seed})


def torus_for_n(N: int, seed: int) -> Instance:
    Lx = max(3, int(round(np.sqrt(N))))
    Ly = max(3, int(round(N / Lx)))
    return torus_pm1(Lx, Ly, seed)


def uniform_sg(N: int, seed: int) -> Instance:
    """Fully connected spin glass, J_ij ~ U[-1, 1] (i < j, symmetric), h_i ~ U[-2, 2].
    Values are rounded to FP32, the precision the library takes them in, so that
    every consumer sees the same instance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    upper = np.triu(rng.uniform(-1.0, 1.0, size=(N, N)).astype(np.float32).astype(np.float64), k=1)
    J = upper + upper.T
    h = rng.uniform(-2.0, 2.0, size=N).astype(np.float32).astype(np.float64)
    return Instance(f"uniform_sg_N{N}_s{seed}", N, dense=J, h=h, meta={"kind": "uniform_sg"})


def with_integer_field(inst: Instance, hmax: int, seed: int) -> Instance:
    """Copy of ``inst`` with an integer field h_i uniform in [-hmax, hmax]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = rng.integers(-hmax, hmax + 1, size=inst.N).astype(np.float64)
    return Instance(inst.name + f"_h{hmax}", inst.N, inst.dense, inst.row_ptr, inst.col, inst.val,
                    h, dict(inst.meta))


def uneven_batch(count: int, n_lo: int, n_hi: int, seed: int):
    """Half random 3-regular, half 2-D tori, N uniform in [n_lo, n_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.integers(n_lo, n_hi + 1, size=count)
    out = []
    for k, N in enumerate(Ns.tolist()):
        s = seed * 1000 + k
        out.append(regular3_pm1(N, s) if k % 2 == 0 else torus_for_n(N, s))
    return out
