"""Failure detection on the GPU without a fault: every wait of the persistent dense
kernel is bounded.  A wait on a flag that nothing sets (hqa_arm_wait_check) runs out
after its limit, the kernel leaves, hqa_sync reports HQA_ERR_TIMEOUT, and the context
stays usable: the next run is bitwise a fresh context's."""
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


@pytest.mark.parametrize("n", [256, 300])   # a CTA pair (two row tiles) / one CTA per row tile
def test_unset_flag_times_out_and_context_recovers(hqa, n):
    inst = instances.sk_pm1(n, 17)
    ctx = hqa.Context.from_instance(inst)
    R, S = 128, 60
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.arm_wait_check(flag, 5, 50_000_000)                 # 50 ms
    ctx.run(S, R, seed=2, precision=hqa.PREC_BF16, outputs=("phi",))
    with pytest.raises(hqa.HQAError) as ei:
        ctx.sync()
    assert ei.value.status == 8                              # HQA_ERR_TIMEOUT
    again = ctx.run(S, R, seed=2, precision=hqa.PREC_BF16, outputs=("phi", "p"))
    ctx.sync()
    fresh = hqa.Context.from_instance(inst)
    ref = fresh.run(S, R, seed=2, precision=hqa.PREC_BF16, outputs=("phi", "p"))
    fresh.sync()
    assert torch.equal(again["phi"], ref["phi"]) and torch.equal(again["p"], ref["p"])


def test_set_flag_changes_nothing(hqa):
    inst = instances.sk_pm1(256, 17)
    ctx = hqa.Context.from_instance(inst)
    flag = torch.ones(1, dtype=torch.int32, device="cuda")
    ctx.arm_wait_check(flag, 5, 50_000_000)
    a = ctx.run(60, 128, seed=3, precision=hqa.PREC_BF16, outputs=("phi",))
    ctx.sync()
    b = ctx.run(60, 128, seed=3, precision=hqa.PREC_BF16, outputs=("phi",))
    ctx.sync()
    assert torch.equal(a["phi"], b["phi"])


def test_arming_needs_a_dense_context(hqa):
    ctx = hqa.Context.from_instance(instances.er_pm1(100, 0.1, 1))
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(hqa.HQAError):
        ctx.arm_wait_check(flag, 1, 1000)
