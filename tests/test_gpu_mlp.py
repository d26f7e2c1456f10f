"""GPU MLP kernels (surrogate gate) against the FP64 oracle.

FP32: logits and the loss gradient agree with the oracle to 1e-5 (normwise,
relative to the largest entry); BF16 (rounded weights, inputs, activations):
logits within 2e-2 of the oracle's logit scale.  AdamW is checked against its
update formula, and a short training run must reduce the loss."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hqa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2004_03972_gb300 import build, hqa as H
    build.build()
    return H


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 6)).astype(np.float32)
    y = (rng.random((n, 2)) < 0.4).astype(np.float32)
    return x, y


@pytest.mark.parametrize("n", [1, 77, 1000, 20011])
def test_forward_and_gradient_fp32(hqa, orc, n):
    w = hqa.MLP.init_params(3)
    mlp = hqa.MLP(w)
    x, y = _data(n, n)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    z = mlp.forward(xg).cpu().numpy().astype(np.float64)
    g, loss = mlp.grad(xg, yg)
    torch.cuda.synchronize()
    l_ref, g_ref, z_ref = orc.mlp_loss_grad(x.astype(np.float64), y.astype(np.float64),
                                           w.astype(np.float64))
    assert np.max(np.abs(z - z_ref)) <= 1e-5 * max(1.0, np.max(np.abs(z_ref)))
    gg = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gg - g_ref)) <= 1e-5 * np.max(np.abs(g_ref))
    assert float(loss) == pytest.approx(l_ref, rel=1e-5)


def test_forward_and_gradient_bf16(hqa, orc):
    w = hqa.MLP.init_params(4)
    mlp = hqa.MLP(w)
    x, y = _data(5000, 1)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    z = mlp.forward(xg, precision=hqa.PREC_BF16).cpu().numpy().astype(np.float64)
    g, _ = mlp.grad(xg, yg, precision=hqa.PREC_BF16)
    torch.cuda.synchronize()
    _, g_ref, z_ref = orc.mlp_loss_grad(x.astype(np.float64), y.astype(np.float64),
                                       w.astype(np.float64))
    assert np.max(np.abs(z - z_ref)) <= 2e-2 * max(1.0, np.max(np.abs(z_ref)))
    gg = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gg - g_ref)) <= 5e-2 * np.max(np.abs(g_ref))


def test_adamw_step_matches_oracle(hqa, orc):
    w = hqa.MLP.init_params(5)
    mlp = hqa.MLP(w)
    rng = np.random.default_rng(2)
    gs = [rng.normal(size=hqa.MLP_PARAMS).astype(np.float32) for _ in range(3)]
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.99, 1e-6, 1e-3
    refs = orc.adamw(w.astype(np.float64), gs, lr, b1, b2, eps, wd)
    for g, ref in zip(gs, refs):
        mlp.adamw(torch.from_numpy(g).cuda(), lr, b1, b2, eps, wd)
        torch.cuda.synchronize()
        # FP32 update of O(1) weights by O(lr) steps: a few ulp of the weight
        assert np.max(np.abs(mlp.params() - ref)) <= 1e-5


def test_training_reduces_loss(hqa):
    """A learnable rule (label 0 = x0 > 0, label 1 = x1 + x2 > 0): the loss falls."""
    rng = np.random.default_rng(7)
    x = rng.normal(size=(8192, 6)).astype(np.float32)
    y = np.stack([x[:, 0] > 0, x[:, 1] + x[:, 2] > 0], axis=1).astype(np.float32)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    mlp = hqa.MLP(hqa.MLP.init_params(1))
    _, l0 = mlp.grad(xg, yg)
    first = float(l0)
    for _ in range(200):
        g, loss = mlp.grad(xg, yg)
        mlp.adamw(g, lr=3e-3)
    torch.cuda.synchronize()
    assert float(loss) < 0.25 * first
    z = mlp.forward(xg).cpu().numpy()
    acc = np.mean((z > 0) == (y > 0.5))
    assert acc > 0.95
