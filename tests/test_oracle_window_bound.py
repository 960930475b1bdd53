"""The oracle's bound on the warp-batched window evaluation
(orc_mlp_window_bound), pinned against an independent simulation of that
arithmetic in numpy: binary16 operands W1, W2, W3, inputs and activations
(numpy's float16 rounding), FP32 sums,
activations round(h + h t) with h = round(z / 2) and t = tanh(h) moved by
+-eps_t, inputs moved by +-x_abs.  Every simulated output must stay inside the
bound; with the tanh errors alone, signed to push the output one way, the
simulation must stay inside the bound's tanh part and reach a good part of
it, so a bound that drops a term or a factor would fail."""
import numpy as np

from oracle import oracle as O

EPS_T, U, XA = 2.0 ** -9, 2.0 ** -11, 2.0 ** -22


def _net(n_in, H, seed, sd):
    npar = O.mlp_param_count(n_in, H)
    return np.random.default_rng(seed).normal(0.0, sd, npar)


def _split(p, n_in, H):
    W1 = p[:H * n_in].reshape(H, n_in)
    b1 = p[H * n_in:H * n_in + H]
    o = H * n_in + H
    W2 = p[o:o + H * H].reshape(H, H)
    b2 = p[o + H * H:o + H * H + H]
    W3 = p[o + H * H + H:o + H * H + 2 * H]
    return W1, b1, W2, b2, W3, p[-1]


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _act(z, r, exact=False):
    """round(h + h t), h = round(z / 2), t = tanh(h) + r eps_t (binary16);
    exact: no rounding (the tanh error alone)."""
    rnd = (lambda v: v) if exact else (lambda v: v.astype(np.float16).astype(np.float64))
    h = rnd(0.5 * z)
    t = np.tanh(h) + r * EPS_T
    return rnd(h + h * t)


def _simulate(p, X, n_in, H, r1, r2, rx, exact=False):
    W1, b1, W2, b2, W3, b3 = _split(p, n_in, H)
    ft = np.float64 if exact else np.float32
    half = (lambda v: v) if exact else (lambda v: v.astype(np.float16))
    W1h, W2h = half(W1).astype(ft), half(W2).astype(ft)
    xh = half(X + rx * XA).astype(ft)
    z1 = (xh @ W1h.T + b1.astype(ft)).astype(np.float64)
    s1 = _act(z1, r1, exact).astype(ft)
    z2 = (s1 @ W2h.T + b2.astype(ft)).astype(np.float64)
    s2 = _act(z2, r2, exact).astype(ft)
    return (s2 @ half(W3).astype(ft) + ft(b3)).astype(np.float64)


def _exact(p, X, n_in, H):
    W1, b1, W2, b2, W3, b3 = _split(p, n_in, H)
    z1 = X @ W1.T + b1
    z2 = _silu(z1) @ W2.T + b2
    return _silu(z2) @ W3 + b3, z1, z2


def test_bound_is_the_definition_of_the_exact_output():
    """The bound is centred on the oracle's exact network (mlp_forward)."""
    n_in, H = 11, 64
    p = _net(n_in, H, 1, 0.2)
    X = np.random.default_rng(2).uniform(-1, 1, (50, n_in))
    y, _, _ = _exact(p, X, n_in, H)
    np.testing.assert_allclose(O.mlp_forward(p, X, hidden=H), y, rtol=1e-12, atol=1e-12)


def test_simulated_evaluation_stays_inside_the_bound():
    for n_in, H, sd in ((11, 64, 0.3), (3, 24, 0.6), (20, 16, 0.5)):
        p = _net(n_in, H, n_in + H, sd)
        rng = np.random.default_rng(H)
        X = rng.uniform(-1, 1, (400, n_in))
        X[:, 4:] = 0.0
        if n_in > 4:
            X[np.arange(400), 4 + rng.integers(0, n_in - 4, 400)] = 1.0
        y, z1, z2 = _exact(p, X, n_in, H)
        b = O.mlp_window_bound(p, X, hidden=H, u=U, eps_t=EPS_T, x_abs=XA)
        assert np.all(b > 0)
        for trial in range(4):
            sg = lambda shape: rng.choice([-1.0, 1.0], shape)
            ys = _simulate(p, X, n_in, H, sg(z1.shape), sg(z2.shape), sg(X.shape))
            assert np.all(np.abs(ys - y) <= b), np.max(np.abs(ys - y) / b)
        # worst-case signs for the tanh errors: t moved towards the sign of dy/dt
        W1, b1, W2, b2, W3, b3 = _split(p, n_in, H)
        h1 = 0.5 * z1
        h2 = 0.5 * z2
        r2 = np.sign(W3[None, :] * h2)
        dy_ds1 = (W3[None, :] * _dsilu(z2)) @ W2            # dy / d(layer-1 activation)
        r1 = np.sign(dy_ds1 * h1)
        ys = _simulate(p, X, n_in, H, r1, r2, np.zeros_like(X))
        assert np.all(np.abs(ys - y) <= b), np.max(np.abs(ys - y) / b)
        # the tanh error alone (exact arithmetic otherwise) against the bound's
        # tanh part: inside it, and pushed to a good part of it (the rest is
        # the triangle inequality over layer 2's paths, which the first-order
        # bound takes)
        ye = _simulate(p, X, n_in, H, r1, r2, np.zeros_like(X), exact=True)
        tanh_only = O.mlp_window_bound(p, X, hidden=H, u=0.0, eps_t=EPS_T, x_abs=0.0)
        assert np.all(np.abs(ye - y) <= tanh_only * (1 + 1e-6) + 1e-12)
        assert np.median((ye - y) / tanh_only) > 0.2, np.median((ye - y) / tanh_only)


def test_planted_mistakes_are_caught():
    """Mistakes planted in the simulation -- layer 2's weights transposed (a
    fragment laid out the wrong way), two inputs swapped (a row written in the
    wrong order) -- leave the bound for most samples."""
    n_in, H = 11, 64
    p = _net(n_in, H, 5, 0.3)
    X = np.random.default_rng(6).uniform(-1, 1, (300, n_in))
    y, z1, z2 = _exact(p, X, n_in, H)
    b = O.mlp_window_bound(p, X, hidden=H, u=U, eps_t=EPS_T, x_abs=XA)
    zeros = (np.zeros_like(z1), np.zeros_like(z2), np.zeros_like(X))
    q = p.copy()
    o = H * n_in + H
    q[o:o + H * H] = p[o:o + H * H].reshape(H, H).T.ravel()
    ys = _simulate(q, X, n_in, H, *zeros)
    assert np.mean(np.abs(ys - y) > b) > 0.5
    ys = _simulate(p, X[:, [1, 0] + list(range(2, n_in))], n_in, H, *zeros)
    assert np.mean(np.abs(ys - y) > b) > 0.5
