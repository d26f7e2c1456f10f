"""GPU parity of the HQA-MD path against the FP64 CPU oracle, through the C ABI.

Tolerances (from the arithmetic):
  local field, per element  e_i = |L_gpu - L_ref| / (|L_ref| + sum_j |J_ij| |phi_j|)
                            <= 1e-5 (FP32 operand), <= 1e-2 (BF16 operand)
  states after <= 100 steps max_i |x_gpu - x_ref| / scale_x <= 1e-5 (FP32), 1e-2 (BF16), with
                            scale_phi = max_i |phi_ref|, scale_p = max(max_i |p_ref|, max_i |p(0)|):
                            p swings through zero every half oscillation, so its error is
                            measured on the momentum scale of the trajectory (|p(0)| = 1)
  integer work (momenta draw, readout on equal inputs, energies, cuts) bit-exact.
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


def _inst(name):
    if name == "er800":
        return instances.er_pm1(800, 0.06, 1200)
    if name == "sk100":
        return instances.sk_pm1(100, 1100)
    if name == "er_h":
        return instances.with_integer_field(instances.er_pm1(300, 0.05, 5), 2, 9)
    if name == "reg3":
        return instances.regular3_pm1(1001, 4)
    if name == "torus":
        return instances.torus_pm1(13, 11, 2)
    raise KeyError(name)


def _abs_scale(inst, phi):
    J = np.abs(inst.to_dense())
    return np.abs(phi) @ J.T      # [R, N]: sum_j |J_ij| |phi_j|


@pytest.mark.parametrize("name", ["er800", "sk100", "er_h", "reg3", "torus"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-2)])
@pytest.mark.parametrize("R,rb,kernel", [(1, 0, 0), (37, 1, 1), (37, 8, 2), (45, 16, 2),
                                         (70, 32, 2), (37, 4, 0)])
def test_local_field(hqa, orc, name, prec, tol, R, rb, kernel):
    inst = _inst(name)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(R)
    phi = rng.uniform(-1.5, 1.5, size=(R, inst.N)).astype(np.float32)
    if kernel == hqa.KERNEL_VECTOR and rb < (8 if prec else 4):
        pytest.skip("vector kernel needs a full 16-byte vector per lane")
    try:
        L = ctx.local_field(torch.from_numpy(phi).cuda(), precision=prec, replicas_per_block=rb,
                            kernel=kernel)
    except hqa.HQAError as e:
        if e.status == 6 and kernel == hqa.KERNEL_VECTOR:
            pytest.skip("vector kernel's shared-memory image does not fit at this blocking")
        raise
    ctx.sync()
    L = L.cpu().numpy().astype(np.float64)
    pr = orc.Problem.from_instance(inst)
    ref = np.stack([orc.beta_field(pr, phi[r].astype(np.float64)) for r in range(R)])
    scale = _abs_scale(inst, phi.astype(np.float64))
    if inst.h is not None:
        scale += 2 * np.abs(inst.h) * np.abs(phi)
    e = np.abs(L - ref) / (np.abs(ref) + scale + 1e-30)
    assert e.max() <= tol


def test_initial_momenta_bit_exact(hqa, orc):
    inst = _inst("er800")
    ctx = hqa.Context.from_instance(inst)
    R = 19
    out = ctx.run(1, R, seed=1234567, outputs=("phi", "p"))
    ctx.sync()
    p = out["p"].cpu().numpy()
    for r in range(R):
        assert np.array_equal(p[r], orc.initial_momenta(1234567, r, inst.N).astype(np.float32))


def test_random_flux_init_bit_exact(hqa, orc):
    inst = _inst("torus")
    ctx = hqa.Context.from_instance(inst)
    # zero schedule: alpha = beta = 0, so phi^(1) = phi^(0) and p^(1/2) = p^(0)
    sched = hqa.schedule(alpha_f=0.0, beta_f=0.0)
    out = ctx.run(1, 5, seed=99, sched=sched, init=hqa.INIT_RANDOM_FLUX, outputs=("phi", "p"))
    ctx.sync()
    phi = out["phi"].cpu().numpy()
    for r in range(5):
        assert np.array_equal(phi[r], orc.initial_flux_random(99, r, inst.N).astype(np.float32))


def _states_close(gpu, ref, tol, scale=None):
    scale = np.max(np.abs(ref)) if scale is None else max(scale, np.max(np.abs(ref)))
    return np.max(np.abs(gpu - ref)) <= tol * scale


@pytest.mark.parametrize("name", ["er800", "sk100", "er_h", "reg3"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-2)])
@pytest.mark.parametrize("kernel", [1, 2])
def test_states_after_100_steps(hqa, orc, name, prec, tol, kernel):
    inst = _inst(name)
    ctx = hqa.Context.from_instance(inst)
    R, S, seed, dt = 45, 100, 77, 1.0 / 5000
    out = ctx.run(S, R, seed=seed, dt=dt, precision=prec, outputs=("phi", "p", "phibar"),
                  kernel=kernel, replicas_per_block=8)
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    phi, p, pbar = (out[k].cpu().numpy().astype(np.float64) for k in ("phi", "p", "phibar"))
    for r in range(0, R, 11):
        p0 = orc.initial_momenta(seed, r, inst.N)
        ophi, op, opbar = orc.md_run(pr, S, dt=dt, p0=p0)
        assert _states_close(phi[r], ophi, tol)
        assert _states_close(p[r], op, tol, scale=np.max(np.abs(p0)))
        assert _states_close(pbar[r], opbar, tol, scale=np.max(np.abs(ophi)))


@pytest.mark.parametrize("rb,kernel,prec", [(1, 1, 0), (2, 1, 0), (4, 1, 0), (8, 1, 0), (16, 1, 0),
                                            (32, 1, 0), (4, 2, 0), (8, 2, 0), (16, 2, 0),
                                            (32, 2, 0), (8, 2, 1), (16, 2, 1), (32, 2, 1)])
def test_every_replica_blocking_matches(hqa, orc, rb, kernel, prec):
    """Same run with each replicas-per-block choice and kernel variant (covers ragged
    last blocks)."""
    inst = _inst("er_h")
    ctx = hqa.Context.from_instance(inst)
    R, S, dt = 21, 60, 1.0 / 700
    out = ctx.run(S, R, seed=5, dt=dt, replicas_per_block=rb, init=hqa.INIT_RANDOM_FLUX,
                  outputs=("phi", "p"), kernel=kernel, precision=prec)
    tol = 1e-5 if prec == 0 else 1e-2
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in (0, R - 1):
        ophi, op, _ = orc.md_run(pr, S, dt=dt, p0=orc.initial_momenta(5, r, inst.N),
                                 phi0=orc.initial_flux_random(5, r, inst.N))
        assert _states_close(out["phi"][r].cpu().numpy(), ophi, tol)
        assert _states_close(out["p"][r].cpu().numpy(), op, tol, scale=1.0)


def test_linear_gamma_and_table_schedules(hqa, orc):
    inst = _inst("sk100")
    ctx = hqa.Context.from_instance(inst)
    pr = orc.Problem.from_instance(inst)
    S = 80
    out = ctx.run(S, 3, seed=8, sched=hqa.schedule(kind=hqa.SCHED_LINEAR_GAMMA), outputs=("phi",))
    ctx.sync()
    ophi, _, _ = orc.md_run(pr, S, p0=orc.initial_momenta(8, 2, 100), kind=orc.LINEAR_GAMMA)
    assert _states_close(out["phi"][2].cpu().numpy(), ophi, 1e-5)
    # explicit tables: alpha on the half-step grid, beta on the integer grid
    ta = 0.02 + 0.01 * np.cos(np.arange(2 * S + 1) * 0.1)
    tb = 0.03 * np.linspace(0.1, 1, S + 1)
    out = ctx.run(S, 3, seed=8, table=(ta, tb), outputs=("phi",))
    ctx.sync()
    ophi, _, _ = orc.md_run(pr, S, p0=orc.initial_momenta(8, 1, 100), kind=orc.TABLE,
                            table_alpha=ta, table_beta=tb)
    assert _states_close(out["phi"][1].cpu().numpy(), ophi, 1e-5)


def test_potential_exponents(hqa, orc):
    inst = _inst("er_h")
    ctx = hqa.Context.from_instance(inst)
    pr = orc.Problem.from_instance(inst)
    for M in (2, 4, 8):
        out = ctx.run(50, 2, seed=3, sched=hqa.schedule(M=M), dt=1 / 500, outputs=("phi",))
        ctx.sync()
        ophi, _, _ = orc.md_run(pr, 50, dt=1 / 500, p0=orc.initial_momenta(3, 1, inst.N), M=M)
        assert _states_close(out["phi"][1].cpu().numpy(), ophi, 1e-5)


@pytest.mark.parametrize("kernel,prec", [(1, 0), (2, 0), (2, 1)])
def test_z2_symmetry_bitwise(hqa, kernel, prec):
    """h = 0: negating p(0) negates the whole trajectory exactly (odd-symmetric rounding)."""
    inst = _inst("er800")
    ctx = hqa.Context.from_instance(inst)
    R, S = 64, 500
    g = torch.Generator().manual_seed(0)
    p0 = (torch.randint(0, 2, (R, inst.N), generator=g) * 2 - 1).float().cuda()
    phi0 = torch.zeros(R, inst.N, device="cuda")
    kw = dict(init=hqa.INIT_GIVEN, phi0=phi0, outputs=("phi", "p", "phibar"), kernel=kernel,
              precision=prec, replicas_per_block=8)
    a = ctx.run(S, R, p0=p0, **kw)
    b = ctx.run(S, R, p0=-p0, **kw)
    ctx.sync()
    for k in ("phi", "p", "phibar"):
        assert torch.equal(a[k], -b[k])


def test_readout_bit_exact(hqa, orc):
    inst = _inst("er800")
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(4)
    R = 9
    phibar = np.round(rng.normal(size=(R, inst.N)), 3).astype(np.float32)   # ties
    phibar[0, :5] = 0.0
    for n in (0, 1, 24, 799, 800, 1000):
        s, f, t = ctx.readout(torch.from_numpy(phibar).cuda(), n)
        ctx.sync()
        for r in range(R):
            os_, of = orc.readout(phibar[r].astype(np.float64), n)
            assert np.array_equal(s[r].cpu().numpy(), os_)
            assert np.array_equal(f[r].cpu().numpy(), of)
            nn = min(max(n, 0), inst.N)
            assert t[r].tolist() == [inst.N - nn, nn]


@pytest.mark.parametrize("name", ["er800", "sk100", "er_h", "torus"])
def test_energy_and_cut_bit_exact(hqa, orc, name):
    inst = _inst(name)
    ctx = hqa.Context.from_instance(inst)
    rng = np.random.default_rng(7)
    R = 33
    s = rng.choice(np.array([-1, 1], np.int8), size=(R, inst.N))
    s[0] = 1
    e, c = ctx.energy(torch.from_numpy(s).cuda())
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    for r in range(R):
        assert int(e[r]) == orc.energy_int(pr, s[r])
        if inst.h is None:
            assert int(c[r]) == orc.cut_int(pr, s[r])


def test_run_pipeline_consistency(hqa, orc):
    """Spins, masks, tallies and energies from hqa_run agree with the oracle's
    readout of the GPU's own window means, and with the oracle's energy."""
    inst = _inst("er800")
    ctx = hqa.Context.from_instance(inst)
    R, n = 40, 24
    out = ctx.run(300, R, seed=11, sched=hqa.schedule(n_ambivalent=n))
    ctx.sync()
    pr = orc.Problem.from_instance(inst)
    pbar = out["phibar"].cpu().numpy().astype(np.float64)
    for r in range(R):
        s, f = orc.readout(pbar[r], n)
        assert np.array_equal(out["spins"][r].cpu().numpy(), s)
        assert np.array_equal(out["frozen"][r].cpu().numpy(), f)
        assert int(out["energy"][r]) == orc.energy_int(pr, s)
        assert int(out["cut"][r]) == orc.cut_int(pr, s)
    assert torch.all(out["tally"][:, 0] == inst.N - n) and torch.all(out["tally"][:, 1] == n)


def test_rejects_bad_arguments(hqa):
    inst = _inst("sk100")
    ctx = hqa.Context.from_instance(inst)
    with pytest.raises(hqa.HQAError):
        ctx.run(0, 4)
    with pytest.raises(hqa.HQAError):
        ctx.run(10, 4, sched=hqa.schedule(M=5))
    with pytest.raises(hqa.HQAError):
        ctx.run(10, 4, replicas_per_block=3)
    J = inst.dense.copy()
    J[0, 1] = 5
    with pytest.raises(hqa.HQAError) as ei:
        hqa.Context.from_dense(J)
    assert ei.value.status == 2
    J = inst.dense.copy()
    J[3, 4] = J[4, 3] = np.nan
    with pytest.raises(hqa.HQAError) as ei:
        hqa.Context.from_dense(J)
    assert ei.value.status == 3


def test_nonfinite_trajectory_is_latched(hqa):
    """A huge step makes the phi^6 force overflow; the run reports HQA_ERR_NONFINITE."""
    inst = _inst("sk100")
    ctx = hqa.Context.from_instance(inst)
    ctx.run(200, 2, sched=hqa.schedule(hstep=60.0), outputs=("phi",))
    with pytest.raises(hqa.HQAError) as ei:
        ctx.sync()
    assert ei.value.status == 7
    ctx.run(10, 2, outputs=("phi",))
    ctx.sync()   # the status was cleared


@pytest.mark.parametrize("kernel,prec,name", [(1, 0, "er_h"), (2, 0, "er800"), (2, 1, "er800"),
                                              (3, 1, "sk100")])
def test_resume_is_bitwise(hqa, kernel, prec, name):
    """Checkpoint/resume: 2 x 300 steps with the state carried over equals 600 steps."""
    inst = _inst(name)
    ctx = hqa.Context.from_instance(inst)
    R, S, dt = 40, 300, 1 / 1000
    kw = dict(dt=dt, precision=prec, kernel=kernel, outputs=("phi", "p"))
    if kernel != 3:
        kw["replicas_per_block"] = 8
    full = ctx.run(2 * S, R, seed=6, **kw)
    a = ctx.run(S, R, seed=6, **kw)
    b = ctx.run(S, R, init=hqa.INIT_GIVEN, phi0=a["phi"], p0=a["p"], start_step=S, **kw)
    ctx.sync()
    assert torch.equal(full["phi"], b["phi"]) and torch.equal(full["p"], b["p"])


@pytest.fixture(scope="module")
def er20k(orc):
    """The largest size of the surrogate-gated workload: ER N = 20000, mean degree 8, +-1,
    with the oracle's 100-step states of replicas 0 and 255 (dt = 1e-4)."""
    inst = instances.er_mean_degree_pm1(20000, 8.0, 21500)
    pr = orc.Problem.from_instance(inst)
    ref = {r: orc.md_run(pr, 100, dt=1e-4, p0=orc.initial_momenta(13, r, inst.N))
           for r in (0, 255)}
    return inst, ref


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-2)])
def test_states_after_100_steps_er20000(hqa, er20k, prec, tol):
    """States at the size and replica count the surrogate-gated workload runs (256
    replicas, the launch shape the library picks for it)."""
    inst, ref = er20k
    ctx = hqa.Context.from_instance(inst)
    out = ctx.run(100, 256, seed=13, dt=1e-4, precision=prec, outputs=("phi", "p", "phibar"))
    ctx.sync()
    for r, (ophi, op, opbar) in ref.items():
        assert _states_close(out["phi"][r].cpu().numpy(), ophi, tol)
        assert _states_close(out["p"][r].cpu().numpy(), op, tol, scale=1.0)
        assert _states_close(out["phibar"][r].cpu().numpy(), opbar, tol,
                             scale=np.max(np.abs(ophi)))
