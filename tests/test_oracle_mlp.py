"""CPU pins of the oracle's surrogate MLP (6 -> 64 -> 64 -> 2, ReLU, two sigmoid
outputs with binary cross-entropy): the analytic gradient equals central finite
differences of the loss, and a network whose hidden layers are silenced has a
loss known in closed form."""
import math

import numpy as np
import pytest


def _params(rng, scale=0.4):
    from oracle.oracle import MLP_P
    return rng.normal(scale=scale, size=MLP_P)


def test_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(40, 6))
    y = (rng.random((40, 2)) < 0.5).astype(np.float64)
    w = _params(rng)
    loss, g, _ = orc.mlp_loss_grad(x, y, w)
    eps = 1e-6
    idx = np.concatenate([rng.choice(orc.MLP_P, 200, replace=False),
                          np.arange(orc.MLP_P - 130, orc.MLP_P)])   # all of W3, b3
    for p in idx:
        wp, wm = w.copy(), w.copy()
        wp[p] += eps
        wm[p] -= eps
        fd = (orc.mlp_loss_grad(x, y, wp, False)[0] - orc.mlp_loss_grad(x, y, wm, False)[0]) / (2 * eps)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, np.abs(g).max()), p


def test_silent_hidden_layers_closed_form(orc):
    """W2 = 0, b2 = 0: h2 = 0, so the logits are b3 for every input and the loss is
    sum_o [softplus(b3_o) - mean(y_o) b3_o]."""
    rng = np.random.default_rng(1)
    w = _params(rng)
    H, IN = orc.MLP_H, orc.MLP_IN
    o2 = H * IN + H
    w[o2:o2 + H * H + H] = 0.0
    b3 = np.array([0.7, -1.3])
    w[-2:] = b3
    x = rng.normal(size=(25, 6))
    y = (rng.random((25, 2)) < 0.3).astype(np.float64)
    loss, g, z = orc.mlp_loss_grad(x, y, w)
    sp = [math.log1p(math.exp(v)) for v in b3]
    want = sum(sp[o] - y[:, o].mean() * b3[o] for o in range(2))
    assert loss == pytest.approx(want, rel=1e-13)
    assert np.allclose(z, b3, rtol=0, atol=1e-15)
    sig = 1 / (1 + np.exp(-b3))
    assert np.allclose(g[-2:], sig - y.mean(axis=0), rtol=1e-12)
    # silent layers pass no gradient back: only b3 moves
    assert np.all(g[:-2] == 0.0)


def test_adamw_constant_gradient_closed_form(orc):
    """With the same gradient g at every step the bias-corrected moments are exactly
    g and g^2, so without decay each step moves w by lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    w0 = rng.normal(size=300)
    g = rng.normal(size=300)
    g[:5] = [0.0, 1e-9, -1e-9, 4.0, -4.0]
    lr, eps = 1e-2, 1e-6
    ws = orc.adamw(w0, [g] * 7, lr, 0.9, 0.99, eps, 0.0)
    for t, w in enumerate(ws, 1):
        want = w0 - t * lr * g / (np.abs(g) + eps)
        assert np.max(np.abs(w - want)) <= 1e-12


def test_adamw_decay_only_closed_form(orc):
    """A zero gradient leaves the moments at zero: each step scales w by (1 - lr wd)."""
    w0 = np.linspace(-2.0, 3.0, 41)
    lr, wd = 0.05, 0.2
    ws = orc.adamw(w0, [np.zeros_like(w0)] * 5, lr, 0.9, 0.999, 1e-8, wd)
    for t, w in enumerate(ws, 1):
        assert np.allclose(w, w0 * (1 - lr * wd) ** t, rtol=1e-14, atol=0)


def test_adamw_first_step_is_sign_like(orc):
    """Step 1: mhat = g and vhat = g^2 whatever b1, b2; decay acts on the old w."""
    rng = np.random.default_rng(4)
    w0, g = rng.normal(size=50), rng.normal(size=50)
    lr, eps, wd = 3e-3, 1e-8, 0.1
    (w1,) = orc.adamw(w0, [g], lr, 0.5, 0.75, eps, wd)
    assert np.allclose(w1, w0 - lr * (g / (np.abs(g) + eps) + wd * w0), rtol=0, atol=1e-15)
