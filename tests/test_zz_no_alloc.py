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


def test_noalloc_matches_the_oracle(hqa, orc):
    """Against the CPU definition of the reduced problem, not only the other entry point."""
    inst = instances.er_pm1(180, 0.07, 23)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(11)
    R, n = 6, 13
    spins, frozen = _problem(rng, inst.N, R, n)
    out_s = torch.empty_like(spins)
    out_e = torch.empty((R,), dtype=torch.int64, device="cuda")
    ctx.solve_sub_noalloc(spins, frozen, n, out_s, out_e)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    s_h, f_h = spins.cpu().numpy(), frozen.cpu().numpy()
    for r in range(R):
        want_s, want_e, _, _ = orc.subsolve(pr, s_h[r], f_h[r])
        assert np.array_equal(out_s[r].cpu().numpy(), want_s)
        assert int(out_e[r]) == want_e


def test_noalloc_statuses_follow_solve_sub(hqa):
    """The same request gets the same status from both entry points: a real-valued
    context (UNSUPPORTED), a batch context (UNSUPPORTED) and n beyond 30 (TOO_LARGE)."""
    def status(fn, *a):
        try:
            fn(*a)
        except hqa.HQAError as e:
            return e.status
        return 0

    real = hqa.Context.from_instance(instances.uniform_sg(64, 3))
    unit = hqa.Context.from_instance(instances.er_pm1(64, 0.1, 2))
    batch = hqa.Context.batch([unit])
    for ctx, n in ((real, 4), (batch, 4), (unit, 31)):
        R = 8
        spins = torch.ones((R, ctx.N), dtype=torch.int8, device="cuda")
        frozen = torch.ones((R, ctx.N), dtype=torch.uint8, device="cuda")
        out_s = torch.empty_like(spins)
        out_e = torch.empty((R,), dtype=torch.int64, device="cuda")
        a = status(ctx.solve_sub, spins, frozen, n)
        b = status(ctx.solve_sub_noalloc, spins, frozen, n, out_s, out_e)
        assert a == b != 0


def test_noalloc_binding_rejects_wrong_buffers(hqa):
    """The binding checks the caller's buffers before the library writes through them."""
    inst = instances.er_pm1(64, 0.1, 8)
    ctx = hqa.Context.from_instance(inst)
    R, N = 4, inst.N
    spins = torch.ones((R, N), dtype=torch.int8, device="cuda")
    frozen = torch.ones((R, N), dtype=torch.uint8, device="cuda")
    good_s = torch.empty_like(spins)
    good_e = torch.empty((R,), dtype=torch.int64, device="cuda")
    bad = [
        (spins, frozen, torch.empty((R - 1, N), dtype=torch.int8, device="cuda"), good_e),
        (spins, frozen, good_s, torch.empty((R,), dtype=torch.int32, device="cuda")),
        (spins, frozen, good_s, torch.empty((R - 1,), dtype=torch.int64, device="cuda")),
        (spins, frozen.to(torch.int8), good_s, good_e),
        (spins, frozen, torch.empty((N, R), dtype=torch.int8, device="cuda").t(), good_e),
        (spins, frozen, torch.empty((R, N), dtype=torch.int8), good_e),
    ]
    for s, f, o, e in bad:
        with pytest.raises(ValueError):
            ctx.solve_sub_noalloc(s, f, 4, o, e)
