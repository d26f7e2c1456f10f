"""CUDA-graph capture and the autotuner, through the C ABI.

A captured sequence (MD run, readout, energy, exact sub-solve) replays to the
same results as the eager calls, bitwise; a capture whose calls were not
prepared by an identical eager call fails cleanly (HQA_ERR_UNSUPPORTED, no
graph) and leaves the stream usable.  The autotuner picks the fastest
candidate it timed, and hqa_run with open options then uses that shape and
gives the same results as with the shape named explicitly."""
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


def _outs(R, N, Rr):
    dev = torch.device("cuda")
    return {"phi": torch.empty(R, N, device=dev), "p": torch.empty(R, N, device=dev),
            "phibar": torch.empty(R, N, device=dev),
            "spins": torch.empty(R, N, dtype=torch.int8, device=dev),
            "frozen": torch.empty(R, N, dtype=torch.uint8, device=dev),
            "energy": torch.empty(Rr, dtype=torch.int64, device=dev),
            "cut": torch.empty(Rr, dtype=torch.int64, device=dev),
            "tally": torch.empty(Rr, 2, dtype=torch.int32, device=dev)}


def _scramble(d):
    for t in d.values():
        t.fill_(7)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replays_run_readout_energy_subsolve(hqa, prec):
    inst = instances.er_pm1(800, 0.06, 1200)
    ctx = hqa.Context.from_instance(inst)
    R, S, n = 64, 300, 12
    sched = hqa.schedule()
    sched.n_ambivalent = n
    st = torch.cuda.Stream()
    out = _outs(R, inst.N, R)
    sub = (torch.empty(R, inst.N, dtype=torch.int8, device="cuda"),
           torch.empty(R, dtype=torch.int64, device="cuda"))

    def step():
        ctx.run(S, R, seed=3, sched=sched, precision=prec, out=out, stream=st)
        ctx.solve_sub(out["spins"], out["frozen"], n, stream=st, out=sub)

    step()
    st.synchronize()
    ref = {k: v.clone() for k, v in out.items()}
    ref_sub = tuple(t.clone() for t in sub)
    with hqa.capture(st) as cap:
        step()
    for _ in range(2):
        _scramble(out)
        sub[0].fill_(0)
        sub[1].fill_(0)
        cap.graph.launch(st)
        st.synchronize()
        for k in out:
            assert torch.equal(out[k], ref[k]), k
        assert torch.equal(sub[0], ref_sub[0]) and torch.equal(sub[1], ref_sub[1])
    cap.graph.close()
    ctx.sync(st)


def test_graph_replays_uneven_batch(hqa):
    members = [hqa.Context.from_instance(i) for i in instances.uneven_batch(6, 200, 1500, 5)]
    b = hqa.Context.batch(members)
    R, S = 16, 200
    st = torch.cuda.Stream()
    out = _outs(R, b.N, R * len(members))
    b.run(S, R, seed=1, out=out, stream=st)
    st.synchronize()
    ref = {k: v.clone() for k, v in out.items()}
    with hqa.capture(st) as cap:
        b.run(S, R, seed=1, out=out, stream=st)
    _scramble(out)
    cap.graph.launch(st)
    st.synchronize()
    for k in out:
        assert torch.equal(out[k], ref[k]), k


def test_unprepared_capture_fails_cleanly(hqa):
    inst = instances.torus_pm1(20, 20, 3)
    ctx = hqa.Context.from_instance(inst)
    R, S = 8, 100
    st = torch.cuda.Stream()
    out = _outs(R, inst.N, R)
    with pytest.raises(hqa.HQAError) as ei:
        with hqa.capture(st):
            ctx.run(S, R, out=out, stream=st)     # nothing prepared: the schedule upload
    assert ei.value.status == 6                    # HQA_ERR_UNSUPPORTED
    with pytest.raises(hqa.HQAError):
        with hqa.capture(st):
            ctx.sync(st)                           # a synchronisation is not capturable
    ctx.run(S, R, out=out, stream=st)              # the stream works eagerly afterwards
    st.synchronize()
    ctx.sync(st)
    assert torch.isfinite(out["phi"]).all()


@pytest.mark.parametrize("prec", [0, 1, 3, 4])
@pytest.mark.parametrize("n", [256, 300])
def test_dense_md_graph_replay(hqa, prec, n):
    """The dense MD replays from a graph with the results of an eager run, bitwise:
    the persistent tcgen05 kernel as a 2-CTA cluster node (N = 256: two row tiles,
    one CTA pair) or as a cooperative kernel node (N = 300: three row tiles, one
    CTA each), and the per-step FP32 CUDA-core launches."""
    inst = instances.sk_pm1(n, 7)
    ctx = hqa.Context.from_instance(inst)
    R, S = 128, 50
    st = torch.cuda.Stream()
    kw = dict(precision=prec, kernel=hqa.KERNEL_DENSE, stream=st, seed=3)
    ref = ctx.run(S, R, **kw, outputs=("phi", "p", "phibar", "cut"))
    out = _outs(R, inst.N, R)
    ctx.run(S, R, **kw, out=out)                   # prepares plan, table and workspaces
    st.synchronize()
    with hqa.capture(st) as cap:
        ctx.run(S, R, **kw, out=out)
    for v in out.values():
        v.zero_()
    for _ in range(2):
        cap.graph.launch(st)
    st.synchronize()
    ctx.sync(st)
    for k in ("phi", "p", "phibar", "cut"):
        assert torch.equal(out[k], ref[k]), k


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_sparse(hqa, prec):
    inst = instances.er_pm1(800, 0.06, 1200)
    ctx = hqa.Context.from_instance(inst)
    R = 256
    best, rows = ctx.autotune(R, precision=prec, probe_steps=32)
    ok = [r for r in rows if r[2] > 0]
    assert len(ok) >= 3
    fastest = min(ok, key=lambda r: r[2])
    assert (best["kernel"], best["replicas_per_block"]) == fastest[:2]
    plan = ctx.plan(R, precision=prec)
    assert (plan["kernel"], plan["replicas_per_block"]) == fastest[:2]
    a = ctx.run(200, R, seed=4, precision=prec, outputs=("phi", "p", "cut"))
    b = ctx.run(200, R, seed=4, precision=prec, outputs=("phi", "p", "cut"),
                kernel=best["kernel"], replicas_per_block=best["replicas_per_block"])
    ctx.sync()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_autotune_batch_and_errors(hqa):
    members = [hqa.Context.from_instance(i) for i in instances.uneven_batch(8, 200, 3000, 6)]
    b = hqa.Context.batch(members)
    R = 32
    best, rows = b.autotune(R, probe_steps=16)
    ok = [r for r in rows if r[2] > 0]
    assert ok and {r[0] for r in rows} == {hqa.KERNEL_SCALAR, hqa.KERNEL_LOWDEG}
    fastest = min(ok, key=lambda r: r[2])
    assert (best["kernel"], best["replicas_per_block"]) == (fastest[0], fastest[1])
    x = b.run(100, R, seed=2, outputs=("phi", "cut"))
    y = b.run(100, R, seed=2, outputs=("phi", "cut"), kernel=best["kernel"],
              replicas_per_block=best["replicas_per_block"])
    b.sync()
    assert torch.equal(x["phi"], y["phi"]) and torch.equal(x["cut"], y["cut"])
    with pytest.raises(hqa.HQAError):
        b.autotune(R, probe_steps=0)


def test_stale_graph_is_refused(hqa):
    """A graph whose context re-uploaded its schedule table (another step count) or
    was destroyed is refused instead of replaying dangling device pointers."""
    inst = instances.torus_pm1(16, 16, 4)
    ctx = hqa.Context.from_instance(inst)
    R = 8
    st = torch.cuda.Stream()
    out = _outs(R, inst.N, R)
    ctx.run(300, R, out=out, stream=st)
    with hqa.capture(st) as cap:
        ctx.run(300, R, out=out, stream=st)
    cap.graph.launch(st)
    st.synchronize()
    ctx.run(100, R, out=out, stream=st)            # new schedule table
    with pytest.raises(hqa.HQAError) as ei:
        cap.graph.launch(st)
    assert ei.value.status == 1
    ctx.run(300, R, out=out, stream=st)
    with hqa.capture(st) as cap2:
        ctx.run(300, R, out=out, stream=st)
    cap2.graph.launch(st)
    st.synchronize()
    ctx.close()
    with pytest.raises(hqa.HQAError):
        cap2.graph.launch(st)
