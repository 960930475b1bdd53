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
* The BF16-operand mode (the precision fixed for the network) equals an
  independent numpy emulation that rounds the same operands to BF16, and
  the first-order bound of that rounding (orc_mlp_error_bounds) holds for it
  against the FP64 definition, element by element.
"""
import math

import pytest

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


def _bf16(a):
    """Values rounded to BF16 (through FP32; round to nearest, ties to even)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _emulate_bf16(p, X, y, w, n_in):
    """Forward and backward with every matrix-product operand rounded to BF16
    (x, W1, h1, W2, dL/dz2, dL/dz1), everything else in FP64."""
    W1, b1, W2, b2, W3, b3 = _split(p, n_in)
    Xr, W1r, W2r = _bf16(X), _bf16(W1), _bf16(W2)
    z1 = Xr @ W1r.T + b1
    h1r = _bf16(_silu(z1))
    z2 = h1r @ W2r.T + b2
    h2 = _silu(z2)
    f = h2 @ W3 + b3[0]
    dy = 2.0 * w * (f - y) / w.sum()
    d2r = _bf16(dy[:, None] * W3[None, :] * _dsilu(z2))
    d1r = _bf16((d2r @ W2r) * _dsilu(z1))
    g = np.concatenate([(d1r.T @ Xr).ravel(), d1r.sum(0), (d2r.T @ h1r).ravel(), d2r.sum(0),
                        dy @ h2, [dy.sum()]])
    return f, g


def test_error_bounds_hold_for_a_bf16_emulation():
    rng = np.random.default_rng(21)
    for n_in, n in ((8, 500), (5, 1500), (16, 300)):
        p = _params(n_in, rng, 0.25)
        X = rng.uniform(-1, 1, (n, n_in))
        y = rng.normal(0, 1, n)
        w = rng.uniform(0.2, 1.0, n)
        w[rng.random(n) < 0.2] = 0.0
        f_ex = O.mlp_forward(p, X, H)
        _, g_ex = O.mlp_loss_grad(p, X, y, w, H)
        fb, gb, lb, gs, gm = O.mlp_error_bounds(p, X, y, w, H)
        f_em, g_em = _emulate_bf16(p, X, y, w, n_in)
        assert np.all(fb > 0) and np.all(gb > 0) and lb > 0
        # the oracle's BF16 mode is the emulation, up to FP64 summation order
        f16 = O.mlp_forward(p, X, H, bf16=True)
        _, g16 = O.mlp_loss_grad(p, X, y, w, H, bf16=True)
        assert np.all(np.abs(f16 - f_em) <= 1e-12 * fb)
        assert np.all(np.abs(g16 - g_em) <= 1e-12 * gs)
        # first order: the emulated deviation stays inside the bound everywhere
        assert np.all(np.abs(f_em - f_ex) <= fb), np.max(np.abs(f_em - f_ex) / fb)
        assert np.all(np.abs(g_em - g_ex) <= gb), np.max(np.abs(g_em - g_ex) / gb)
        # and the bound is not vacuous: the rounding comes within 1000x of it
        assert np.max(np.abs(g_em - g_ex) / gb) > 1e-3
        # term statistics: |g| <= sum |terms|, max term <= sum
        assert np.all(np.abs(g_ex) <= gs * (1 + 1e-12)) and np.all(gm <= gs)


def test_training_loop_equals_a_numpy_adam_over_minibatches():
    """orc_mlp_train against Adam written out here in numpy (m, v, bias
    correction with the step count from 1) over the same minibatches of
    consecutive samples, the last one shorter, with the oracle's gradient of
    each minibatch; also in the BF16-operand mode."""
    rng = np.random.default_rng(8)
    n_in, n, batch, epochs, lr = 6, 700, 256, 3, 3e-3
    p0 = _params(n_in, rng, 0.3)
    X = rng.uniform(-1, 1, (n, n_in))
    y = rng.normal(0, 1, n)
    w = rng.uniform(0.1, 1.0, n)
    for bf16 in (False, True):
        p = p0.copy()
        m, v = np.zeros_like(p), np.zeros_like(p)
        t, losses = 0, []
        for ep in range(epochs):
            ls = []
            for f0 in range(0, n, batch):
                sl = slice(f0, min(n, f0 + batch))
                loss, g = O.mlp_loss_grad(p, X[sl], y[sl], w[sl], H, bf16=bf16)
                t += 1
                m = 0.9 * m + 0.1 * g
                v = 0.999 * v + 0.001 * g * g
                p = p - lr * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
                ls.append(loss)
            losses.append(np.mean(ls))
        q, lf, ll = O.mlp_train(p0, X, y, w, epochs, batch, lr, H, bf16=bf16)
        np.testing.assert_allclose(q, p, rtol=1e-12, atol=1e-14)
        assert lf == pytest.approx(losses[0], rel=1e-12) and ll == pytest.approx(losses[-1], rel=1e-12)
        assert ll < lf
