"""FP64 Hamiltonian diagnostic on the GPU (H_MD, Results Eq. (3)).

Parity: for given FP32 states the GPU value agrees with the FP64 oracle to
1e-6 of the Hamiltonian's absolute scale
  alpha sum (p^2/2 + |phi|^M) + beta/2 sum |phi| (sum_j |J_ij| |phi_j| + 2 |h| |phi|),
the bound of a sum whose only rounding is the FP32 local field (1e-7 relative
on that scale) and FP64 accumulation.
Conservation at a fixed schedule (alpha, beta constant): the leapfrog drift of
H_MD over a fixed time T falls as h^2 (ratio 4 +- 1 when h halves) and equals
the oracle's drift to 1e-4 absolute (FP32 trajectories)."""
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


def _scale(inst, tau, phi, p, orc, M=6):
    a, b = orc.schedule(tau)
    J = np.abs(inst.to_dense())
    h = np.zeros(inst.N) if inst.h is None else np.abs(inst.h)
    ap = np.abs(phi)
    return a * np.sum(0.5 * p * p + ap ** M) + 0.5 * b * np.sum(ap * (J @ ap + 2 * h * ap))


@pytest.mark.parametrize("name", ["er_h", "torus", "sk"])
@pytest.mark.parametrize("half", [False, True])
def test_hmd_matches_oracle(hqa, orc, name, half):
    inst = {"er_h": instances.with_integer_field(instances.er_pm1(300, 0.05, 5), 2, 9),
            "torus": instances.torus_pm1(13, 11, 2),
            "sk": instances.sk_pm1(120, 3)}[name]
    ctx = hqa.Context.from_instance(inst)
    R = 6
    rng = np.random.default_rng(1)
    phi = rng.uniform(-1.3, 1.3, size=(R, inst.N)).astype(np.float32)
    p = rng.uniform(-1, 1, size=(R, inst.N)).astype(np.float32)
    pr = orc.Problem.from_instance(inst)
    for tau in (0.0, 0.37, 1.0):
        out = ctx.hmd(torch.from_numpy(phi).cuda(), torch.from_numpy(p).cuda(), tau,
                      half_kick=half).cpu().numpy()
        for r in range(R):
            x, q = phi[r].astype(np.float64), p[r].astype(np.float64)
            if half:
                q = q - 0.5 * orc.force(pr, tau, x)
            ref = orc.hmd(pr, tau, x, q)
            assert abs(out[r] - ref) <= 1e-6 * _scale(inst, tau, x, q, orc), (tau, r)


def test_drift_scales_as_h_squared(hqa, orc):
    inst = instances.er_pm1(300, 0.05, 5)
    ctx = hqa.Context.from_instance(inst)
    pr = orc.Problem.from_instance(inst)
    R, T, seed = 8, 50.0, 3
    prm = (0.03, 1.0, 0.0, 0.08, 1.0, 0.0, 0.032)     # alpha = 0.03, beta = 0.08 for all tau
    drift = {}
    for h in (1.0, 0.5, 0.25):
        S = int(T / h)
        sched = hqa.schedule(alpha_f=prm[0], rho1=1.0, rho2=0.0, beta_f=prm[3], kappa1=1.0,
                             kappa2=0.0, hstep=h)
        out = ctx.run(S, R, seed=seed, sched=sched, dt=1.0 / S, outputs=("phi", "p"))
        H1 = ctx.hmd(out["phi"], out["p"], 1.0, sched=sched, half_kick=True).cpu().numpy()
        H0 = 0.03 * inst.N / 2                          # phi = 0, p = +-1
        drift[h] = H1 - H0
        p0 = orc.initial_momenta(seed, 0, inst.N)
        tr = orc.md_run(pr, S, dt=1.0 / S, p0=p0, prm=prm, hstep=h, trace=True)[3]
        assert abs(drift[h][0] - (tr[-1] - tr[0])) <= 1e-4 + 1e-3 * abs(tr[-1] - tr[0])
    for r in range(R):
        for a, b in ((1.0, 0.5), (0.5, 0.25)):
            assert 3.0 <= drift[a][r] / drift[b][r] <= 5.0, (r, a, drift[a][r], drift[b][r])


def test_hmd_rejects(hqa):
    inst = instances.torus_pm1(5, 5, 1)
    ctx = hqa.Context.from_instance(inst)
    phi = torch.zeros(2, inst.N, device="cuda")
    s = hqa.schedule()
    s.kind = hqa.SCHED_TABLE
    with pytest.raises(hqa.HQAError):
        ctx.hmd(phi, phi, 0.5, sched=s)
    with pytest.raises(hqa.HQAError):
        ctx.hmd(phi, phi, float("nan"))
