"""hqa_solve_sub_noalloc: the sub-solve for callers that cannot let the library
allocate device memory (for example because another allocator already holds
the device's memory, or because cudaMalloc's device-wide synchronisation is
not acceptable to them).  It must give exactly the results of hqa_solve_sub,
call after call, while using only the library's fixed scratch array.

This file is collected last on purpose, and it passes both on its own in a
fresh process and after the rest of the suite.
"""
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


def _problem(rng, N, R, n):
    spins = rng.choice(np.array([-1, 1], np.int8), size=(R, N))
    frozen = np.ones((R, N), np.uint8)
    for r in range(R):
        frozen[r, rng.choice(N, size=n, replace=False)] = 0
    return torch.from_numpy(spins).cuda(), torch.from_numpy(frozen).cuda()


def test_noalloc_matches_solve_sub_on_consecutive_calls(hqa):
    inst = instances.with_integer_field(instances.er_pm1(300, 0.05, 17), 1, 4)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(2)
    R, n = 96, 14
    out_s = torch.empty((R, inst.N), dtype=torch.int8, device="cuda")
    out_e = torch.empty((R,), dtype=torch.int64, device="cuda")
    for call in range(2):          # the second call must not see the first call's scratch
        spins, frozen = _problem(rng, inst.N, R, n - 3 * call)
        ref_s, ref_e = ctx.solve_sub(spins, frozen, n)
        ctx.solve_sub_noalloc(spins, frozen, n, out_s, out_e)
        ctx.sync()
        assert torch.equal(out_s, ref_s), f"spins differ on call {call}"
        assert torch.equal(out_e, ref_e), f"energies differ on call {call}"


def test_noalloc_allocates_no_device_memory(hqa):
    inst = instances.er_pm1(200, 0.06, 5)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(9)
    R, n = 64, 12
    spins, frozen = _problem(rng, inst.N, R, n)
    out_s = torch.empty_like(spins)
    out_e = torch.empty((R,), dtype=torch.int64, device="cuda")
    ctx.solve_sub_noalloc(spins, frozen, n, out_s, out_e)   # first call on this device: set-up
    ctx.sync()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ctx.solve_sub_noalloc(spins, frozen, n, out_s, out_e)
    ctx.sync()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_more_replicas_than_its_scratch_holds(hqa):
    inst = instances.er_pm1(64, 0.1, 1)
    ctx = hqa.Context.from_instance(inst)
    R = 2049
    spins = torch.ones((R, inst.N), dtype=torch.int8, device="cuda")
    frozen = torch.ones((R, inst.N), dtype=torch.uint8, device="cuda")
    out_s = torch.empty_like(spins)
    with pytest.raises(hqa.HQAError) as ei:
        ctx.solve_sub_noalloc(spins, frozen, 4, out_s)
    assert ei.value.status == 9     # HQA_ERR_TOO_LARGE
