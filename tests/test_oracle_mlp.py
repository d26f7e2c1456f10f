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
