"""Pins of the oracle's importance network.

* Backpropagation against central finite differences of the loss (a
  different computation of the same derivative), every parameter group.
* Special cases with closed forms: zero hidden weights give
  f = b3 + sum_k W3_k SiLU(b2_k); SiLU(0) = 0 and SiLU'(0) = 1/2 fix the
  gradient of a zero network exactly.
* Adam: the first step moves every parameter by lr * sign(g) (bias
  correction makes m/sqrt(v) = g/|g|).
* A few hundred Adam steps fit a smooth 1-D target (the loss falls by more
  than 100x).
"""
import math

import numpy as np

from oracle import oracle as O

H = 64


def _params(n_in, rng, scale=0.3):
    return rng.normal(0.0, scale, O.mlp_param_count(n_in, H))


def _split(p, n_in):
    i = 0
    out = []
    for shape in ((H, n_in), (H,), (H, H), (H,), (H,), (1,)):
        k = int(np.prod(shape))
        out.append(p[i:i + k].reshape(shape))
        i += k
    return out


def test_param_count():
    assert O.mlp_param_count(8, H) == 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(1)
    n_in, n = 8, 20
    p = _params(n_in, rng)
    X = rng.uniform(-1, 1, (n, n_in))
    y = rng.normal(0, 1, n)
    w = rng.uniform(0.5, 2.0, n)
    loss, g = O.mlp_loss_grad(p, X, y, w)
    idx = np.concatenate([rng.choice(np.arange(0, 512), 12, replace=False),      # W1
                          np.arange(512, 520),                                   # b1
                          rng.choice(np.arange(576, 576 + 4096), 12, replace=False),  # W2
                          np.arange(4672, 4680),                                 # b2
                          np.arange(4736, 4744),                                 # W3
                          [p.size - 1]])                                         # b3
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (O.mlp_loss_grad(pp, X, y, w)[0] - O.mlp_loss_grad(pm, X, y, w)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_zero_hidden_weights_closed_form():
    rng = np.random.default_rng(2)
    n_in = 5
    p = np.zeros(O.mlp_param_count(n_in, H))
    W1, b1, W2, b2, W3, b3 = _split(p, n_in)
    b2[:] = rng.normal(0, 1, H)
    W3[:] = rng.normal(0, 1, H)
    b3[:] = 0.7
    X = rng.uniform(-1, 1, (4, n_in))
    silu = lambda z: z / (1 + np.exp(-z))
    expect = 0.7 + np.dot(W3, silu(b2))
    np.testing.assert_allclose(O.mlp_forward(p, X), expect, rtol=1e-14)


def test_zero_network_gradient_closed_form():
    # all parameters zero: f = 0, h1 = h2 = 0, dsilu(0) = 1/2
    n_in, n = 3, 6
    rng = np.random.default_rng(3)
    p = np.zeros(O.mlp_param_count(n_in, H))
    X = rng.uniform(-1, 1, (n, n_in))
    y = rng.normal(0, 1, n)
    w = np.ones(n)
    loss, g = O.mlp_loss_grad(p, X, y, w)
    assert loss == np.mean(y ** 2)
    gW1, gb1, gW2, gb2, gW3, gb3 = _split(g, n_in)
    assert abs(gb3[0] - np.sum(2 * (0 - y)) / n) <= 1e-14 * abs(gb3[0])
    assert np.all(gW3 == 0) and np.all(gW2 == 0) and np.all(gb2 == 0) and np.all(gW1 == 0)


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(4)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    p0 = p.copy()
    m, v = np.zeros(50), np.zeros(50)
    O.adam_step(p, m, v, g, 1, lr=1e-2, eps=0.0)
    np.testing.assert_allclose(p0 - p, 1e-2 * np.sign(g), rtol=1e-12)


def test_adam_fits_a_smooth_target():
    rng = np.random.default_rng(5)
    n_in = 2
    X = np.stack([np.linspace(-1, 1, 64), np.ones(64)], axis=1)
    y = np.sin(2.5 * X[:, 0]) - 3.0 * X[:, 0]
    w = np.ones(64)
    p = _params(n_in, rng, 0.2)
    m, v = np.zeros_like(p), np.zeros_like(p)
    l0 = O.mlp_loss_grad(p, X, y, w)[0]
    for t in range(1, 401):
        loss, g = O.mlp_loss_grad(p, X, y, w)
        O.adam_step(p, m, v, g, t, lr=1e-2)
    assert loss < l0 / 100, (l0, loss)
    assert math.isfinite(loss)
