"""The streaming sparse kernel (operand and state in global memory, one grid
barrier per step) against the FP64 oracle: fields and states after 100 steps
(FP32 within 1e-5, BF16 within 1e-2, as for the resident kernels), ragged
replica counts, resume and Z2 symmetry bitwise, and the sizes the resident
kernels cannot hold (AUTO falls back to it instead of HQA_ERR_TOO_LARGE).
Methods, "Leapfrog algorithm"."""
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


def _close(gpu, ref, tol, scale=None):
    s = np.max(np.abs(ref)) if scale is None else max(scale, np.max(np.abs(ref)))
    return np.max(np.abs(gpu - ref)) <= tol * s


@pytest.mark.parametrize("R", [1, 37, 256])
@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-2)])
def test_stream_field(hqa, orc, R, prec, tol):
    inst = instances.with_integer_field(instances.er_mean_degree_pm1(3000, 8.0, 71), 2, 5)
    ctx = hqa.Context.from_instance(inst)
    phi = np.random.default_rng(R).uniform(-1.5, 1.5, size=(R, inst.N)).astype(np.float32)
    L = ctx.local_field(torch.from_numpy(phi).cuda(), precision=prec, kernel=hqa.KERNEL_STREAM)
    ctx.sync()
    L = L.cpu().numpy().astype(np.float64)
    pr = orc.Problem.from_instance(inst)
    rp, col, val = inst.row_ptr, inst.col, inst.val
    for r in sorted({0, R // 2, R - 1}):
        x = phi[r].astype(np.float64)
        ref = orc.beta_field(pr, x)
        scale = np.array([np.abs(val[rp[i]:rp[i + 1]]) @ np.abs(x[col[rp[i]:rp[i + 1]]])
                          for i in range(inst.N)]) + 2 * np.abs(inst.h) * np.abs(x)
        assert np.max(np.abs(L[r] - ref) / (np.abs(ref) + scale + 1e-30)) <= tol


@pytest.mark.parametrize("N,R", [(2000, 45), (20000, 256)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-2)])
def test_stream_states_after_100_steps(hqa, orc, N, R, prec, tol):
    inst = instances.er_mean_degree_pm1(N, 8.0, 900 + N)
    ctx = hqa.Context.from_instance(inst)
    out = ctx.run(100, R, seed=17, dt=1e-4, precision=prec, kernel=hqa.KERNEL_STREAM,
                  outputs=("phi", "p", "phibar"))
    ctx.sync()
    assert ctx.plan(R, precision=prec, kernel=hqa.KERNEL_STREAM)["kernel"] == hqa.KERNEL_STREAM
    pr = orc.Problem.from_instance(inst)
    for r in sorted({0, R - 1}):
        ophi, op, opbar = orc.md_run(pr, 100, dt=1e-4, p0=orc.initial_momenta(17, r, N))
        assert _close(out["phi"][r].cpu().numpy(), ophi, tol)
        assert _close(out["p"][r].cpu().numpy(), op, tol, scale=1.0)
        assert _close(out["phibar"][r].cpu().numpy(), opbar, tol, scale=np.max(np.abs(ophi)))


@pytest.mark.parametrize("prec", [0, 1])
def test_stream_resume_and_z2_bitwise(hqa, prec):
    inst = instances.er_mean_degree_pm1(5000, 8.0, 5)
    ctx = hqa.Context.from_instance(inst)
    R, S = 40, 300
    kw = dict(precision=prec, kernel=hqa.KERNEL_STREAM, dt=1.0 / S)
    full = ctx.run(S, R, seed=3, outputs=("phi", "p"), **kw)
    half = ctx.run(120, R, seed=3, outputs=("phi", "p"), **kw)
    rest = ctx.run(S - 120, R, init=hqa.INIT_GIVEN, phi0=half["phi"], p0=half["p"],
                   start_step=120, outputs=("phi", "p"), **kw)
    g = torch.Generator().manual_seed(2)
    p0 = (torch.randint(0, 2, (R, inst.N), generator=g) * 2 - 1).float().cuda()
    z = torch.zeros(R, inst.N, device="cuda")
    a = ctx.run(S, R, init=hqa.INIT_GIVEN, phi0=z, p0=p0, outputs=("phi", "p"), **kw)
    b = ctx.run(S, R, init=hqa.INIT_GIVEN, phi0=z, p0=-p0, outputs=("phi", "p"), **kw)
    ctx.sync()
    for k in ("phi", "p"):
        assert torch.equal(full[k], rest[k]), k
        assert torch.equal(a[k], -b[k]), k


def test_auto_streams_what_the_resident_kernels_cannot_hold(hqa, orc):
    """ER N = 40000, mean degree 8: one replica's FP32 operand (2 x 160 KB) exceeds
    shared memory, so the resident kernels answer HQA_ERR_TOO_LARGE and AUTO runs the
    streaming kernel."""
    inst = instances.er_mean_degree_pm1(40000, 8.0, 6)
    ctx = hqa.Context.from_instance(inst)
    with pytest.raises(hqa.HQAError) as ei:
        ctx.run(10, 2, kernel=hqa.KERNEL_SCALAR, outputs=("phi",))
    assert ei.value.status == 9
    assert ctx.plan(2)["kernel"] == hqa.KERNEL_STREAM
    out = ctx.run(50, 2, seed=8, dt=1e-4, outputs=("phi", "p", "phibar", "spins", "cut"))
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in (0, 1):
        ophi, op, _ = orc.md_run(pr, 50, dt=1e-4, p0=orc.initial_momenta(8, r, inst.N))
        assert _close(out["phi"][r].cpu().numpy(), ophi, 1e-5)
        assert int(out["cut"][r]) == orc.cut_int(pr, out["spins"][r].cpu().numpy())
