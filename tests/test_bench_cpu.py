"""Host logic of bench.py that feeds the JSON line, checked without a GPU: the
committed ncu traffic table and its source-hash guard, the kernel keys it is
looked up by, the equal-cut bootstrap, and the launch count per step."""
import json
import os
import types

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the library's kernel selectors (include/hqa.h), as bench.py reads them from the binding
HQA = types.SimpleNamespace(KERNEL_AUTO=0, KERNEL_SCALAR=1, KERNEL_VECTOR=2, KERNEL_DENSE=3,
                            KERNEL_LOWDEG=4, KERNEL_STREAM=5)


def test_committed_traffic_entries_resolve_while_their_sources_are_unchanged():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        table = json.load(f)
    assert table, "the traffic table is empty"
    for key, ent in table.items():
        assert "--clock-control none" in ent["capture"] or ent["capture"].startswith("ncu --set full"), key
        srcs = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
        shas = ent["source_sha"] if isinstance(ent["source_sha"], list) else [ent["source_sha"]]
        unchanged = all(bench._src_sha(os.path.join(ROOT, "paper_2004_03972_gb300", "csrc", s)) == h
                        for s, h in zip(srcs, shas))
        got = bench.ncu_traffic(key)
        assert got == (ent["dram_bytes_per_launch"] if unchanged else None), key


def test_traffic_is_null_once_a_source_changed(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        key = next(iter(json.load(f)))
    monkeypatch.setattr(bench, "_src_sha", lambda path: "0000000000000000")
    assert bench.ncu_traffic(key) is None
    assert bench.ncu_traffic("no_such_kernel@nowhere") is None


@pytest.mark.parametrize("prec,key", [
    ("PREC_FP16X2", "k_dense_md<128,*,2,*,*,true,*,*,*>"),
    ("PREC_FP16", "k_dense_md<128,*,1,*,*,true,*,*,*>"),
    ("PREC_BF16X2", "k_dense_md<128,*,2,*,*,false,*,*,*>"),
    ("PREC_BF16", "k_dense_md<128,*,1,*,*,false,*,*,*>"),
    ("PREC_FP32", "k_dense_simt<1>"),
])
def test_dense_kernel_keys(prec, key):
    plan = {"kernel": HQA.KERNEL_DENSE, "replicas_per_block": 256}
    assert bench.kernel_name(HQA, plan, prec) == key


def test_sparse_kernel_keys():
    assert bench.kernel_name(HQA, {"kernel": HQA.KERNEL_VECTOR, "replicas_per_block": 8},
                             "PREC_BF16") == "k_sparse_md_vec<8,true>"
    assert bench.kernel_name(HQA, {"kernel": HQA.KERNEL_SCALAR, "replicas_per_block": 4},
                             "PREC_FP32") == "k_sparse_md<4,false>"
    assert bench.kernel_name(HQA, {"kernel": HQA.KERNEL_STREAM, "replicas_per_block": 8},
                             "PREC_BF16") == "k_sparse_stream<true>"


def test_equal_cut_interval():
    rng = np.random.default_rng(3)
    a = rng.integers(1900, 2000, 1024)
    lo, hi = bench.median_diff_ci(a, a.copy())
    assert lo <= 0 <= hi                                  # the same sample: equal median
    lo, hi = bench.median_diff_ci(a + 40, a)
    assert lo > 0 and abs((lo + hi) / 2 - 40) <= 5        # a shifted sample: the shift, not 0
    assert bench.bootstrap_halfwidth(a) >= 0
    assert bench.bootstrap_halfwidth(np.full(64, 7)) == 0


def test_launches_per_step():
    plain = {"one_at_a_time": False, "prec_name": "PREC_FP16X2"}
    dense = {"kernel": HQA.KERNEL_DENSE, "chunks": 2}
    # two chunks x (init, MD, output), readout, energy, sub-solve (prep, min, arg, walk, assemble, energy)
    assert bench.launches_per_step(HQA, dense, plain, None, 10000, False, False, 1) == 14
    fp32 = {"one_at_a_time": False, "prec_name": "PREC_FP32"}
    assert bench.launches_per_step(HQA, dense, fp32, None, 100, False, False, 1) == 102 + 8
    sparse = {"kernel": HQA.KERNEL_VECTOR}
    assert bench.launches_per_step(HQA, sparse, plain, None, 5000, True, False, 1) == 3
    one = {"one_at_a_time": True, "prec_name": "PREC_FP32"}
    assert bench.launches_per_step(HQA, sparse, one, None, 5000, True, False, 64) == 192


def test_whole_job_rate_single_rank():
    # units per rank-step x steps x ranks / time
    assert bench.whole_job_rate(1e9, 10, 1, 2.0) == pytest.approx(5e9)
