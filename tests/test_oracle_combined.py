"""Pins of the oracle's combined track-length/collision estimator (R14; no value
here comes from the CUDA path).

* the combination itself, on synthetic batch series: the coefficient and the
  variance are the minimum over a fine grid on [0, 1] of the sample variance
  of a x + (1 - a) y (brute force, no formula retyped), for correlated,
  anticorrelated and independent series and where the unconstrained optimum
  lies outside [0, 1] (clipped: the end of the interval); special cases:
  identical series (a = 1/2, the single-series error), a constant second
  series (a = 0, zero error), a bin scored by one batch only (perfectly
  correlated estimators: a clipped end, not an estimate of zero);
* one run scoring both: its two halves equal, bit for bit, the sums of the
  track-length-only and collision-only runs with the same seed (the same
  histories), and the summed products equal those rebuilt from separate runs
  of every batch's histories; the region scalar equals the brute-force
  combination of those per-batch region sums;
* closed form, infinite medium: the track length of a history is the
  collision score plus independent noise (per history L = K / St plus the
  spread of K exponential flights), so the best combination is the collision
  estimator: a -> 0 and the combined error equals the collision error.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W


def _sums(x, y, nv):
    """Batch sums from batch values x_b = B s_b / (N V)."""
    B = len(x)
    sx, sy = np.asarray(x) * nv / B, np.asarray(y) * nv / B
    return [np.array([v]) for v in (sx.sum(), (sx * sx).sum(), sy.sum(), (sy * sy).sum(),
                                    (sx * sy).sum())]


def _brute(x, y, lo=0.0, hi=1.0, n=100_001):
    """Grid minimum over a of the sample variance of the mean of a x + (1-a) y."""
    a = np.linspace(lo, hi, n)
    z = a[:, None] * x[None, :] + (1.0 - a[:, None]) * y[None, :]
    var = z.var(axis=1, ddof=1) / len(x)
    k = int(np.argmin(var))
    return a[k], z[k].mean(), var[k], (hi - lo) / (n - 1)


@pytest.mark.parametrize("case", ["positive", "negative", "outside", "independent"])
def test_combination_is_the_grid_minimum(case):
    rng = np.random.default_rng({"positive": 1, "negative": 2, "outside": 3, "independent": 4}[case])
    B = 40
    u, e = rng.normal(size=B), rng.normal(size=B)
    x = 10.0 + u
    y = {"positive": 10.0 + 0.6 * u + 0.5 * e,
         "negative": 10.0 - 0.7 * u + 0.4 * e,
         "outside": 10.0 + 2.0 * u + 0.05 * e,      # unconstrained optimum near 2
         "independent": 10.0 + 1.3 * e}[case]
    N, vol = 4000, 2.5
    alpha = np.zeros(1)
    m, r = O.combine(*_sums(x, y, N * vol), N, B, vol, alpha=alpha)
    a_b, m_b, v_b, da = _brute(x, y)
    assert abs(alpha[0] - a_b) <= da
    assert m[0] == pytest.approx(m_b, rel=1e-9, abs=abs(x.mean() - y.mean()) * da)
    assert (m[0] * r[0]) ** 2 == pytest.approx(v_b, rel=1e-6)
    # never worse than either estimator alone
    assert (m[0] * r[0]) ** 2 <= min(x.var(ddof=1), y.var(ddof=1)) / B * (1 + 1e-12)
    if case == "outside":
        assert alpha[0] == 1.0


def test_combination_special_cases():
    rng = np.random.default_rng(7)
    B, N, vol = 25, 2500, 1.0
    x = 3.0 + rng.normal(size=B)
    # identical series: any a gives the same variance; a = 1/2 by the rule
    alpha = np.zeros(1)
    m, r = O.combine(*_sums(x, x, N * vol), N, B, vol, alpha=alpha)
    assert alpha[0] == 0.5
    assert m[0] == pytest.approx(x.mean(), rel=1e-12)
    assert r[0] == pytest.approx(x.std(ddof=1) / math.sqrt(B) / x.mean(), rel=1e-9)
    # a constant second series (N V = B, so batch sums equal batch values)
    one = np.ones(B)
    m, r = O.combine(*_sums(x, one, B), B, B, 1.0, alpha=alpha)
    assert abs(alpha[0]) < 1e-12
    assert m[0] == pytest.approx(1.0, rel=1e-12)
    assert r[0] < 1e-6
    # one scoring batch: y = (Y / X) x exactly; the unclipped optimum would be
    # a = Y / (Y - X) and the estimate zero
    X, Y = 6.0, 4.0
    x1, y1 = np.zeros(B), np.zeros(B)
    x1[3], y1[3] = X, Y
    m, r = O.combine(*_sums(x1, y1, B), B, B, 1.0, alpha=alpha)
    assert alpha[0] == 0.0                       # Y / (Y - X) = -2, clipped
    assert m[0] == pytest.approx(Y / B, rel=1e-12)
    assert r[0] == pytest.approx(y1.std(ddof=1) / math.sqrt(B) / y1.mean(), rel=1e-9)


def _td_box():
    """A small 3-D multigroup time-dependent problem with vacuum faces."""
    G = 2
    mat = np.zeros((3, 4, 5), np.uint8)
    mat[:, 1:3, 2:4] = 1
    st = [[1.0, 1.5], [0.4, 2.5]]
    c = [[0.6, 0.5], [0.9, 0.3]]
    P = np.array([[[0.3, 0.7], [0.1, 0.9]], [[0.5, 0.5], [0.2, 0.8]]])
    return W.box("combined_box", (5, 4, 3), (1.0, 1.0, 1.0), mat, st, c, P, [2.0, 0.5],
                 (1.0, 1.0, 0.5), (3.0, 3.0, 2.5), np.linspace(0.0, 4.0, 5), (2, 1, 0), (5, 3, 3),
                 src_pdf=[0.7, 0.3])


def test_combined_run_halves_are_the_single_estimator_runs():
    prob = _td_box()
    N, B = 6000, 12
    cb = O.run(prob, N, seed=5, batches=B, estimator=O.EST_COMBINED, threads=3)
    tl = O.run(prob, N, seed=5, batches=B, estimator=O.EST_TRACK, threads=3)
    ce = O.run(prob, N, seed=5, batches=B, estimator=O.EST_COLLISION, threads=3)
    assert cb["counts"] == tl["counts"] == ce["counts"]
    assert np.array_equal(cb["sum1"][0], tl["sum1"]) and np.array_equal(cb["sum2"][0], tl["sum2"])
    assert np.array_equal(cb["sum1"][1], ce["sum1"]) and np.array_equal(cb["sum2"][1], ce["sum2"])
    # the combined estimate per bin is the combination of the two halves
    assert np.all(np.isfinite(cb["mean"])) and np.all(cb["relerr"] >= 0)
    scored = (tl["sum1"] > 0) & (ce["sum1"] > 0)
    assert scored.sum() > 100


def test_summed_products_from_separate_batch_runs():
    prob = _td_box()
    N, B = 2000, 4                      # 500 histories per batch
    cb = O.run(prob, N, seed=8, batches=B, estimator=O.EST_COMBINED, threads=2)
    T, Cc = [], []
    for b in range(B):
        part = O.run(prob, N // B, seed=8, offset=b * (N // B), batches=2,
                     estimator=O.EST_COMBINED, threads=1)
        T.append(part["sum1"][0])
        Cc.append(part["sum1"][1])
    T, Cc = np.array(T), np.array(Cc)
    np.testing.assert_allclose(cb["sum12"], (T * Cc).sum(axis=0), rtol=1e-11, atol=1e-300)
    np.testing.assert_allclose(cb["sum2"][0], (T * T).sum(axis=0), rtol=1e-11, atol=1e-300)
    # region scalar (cells i in [2, 5), j in [1, 3), all k) from the per-batch
    # sums, by brute force
    nv = N * 1.0
    reg = (slice(None), slice(None), slice(1, 3), slice(2, 5))
    x, y = B * T[reg].sum(axis=(1, 2, 3, 4, 5)) / nv, B * Cc[reg].sum(axis=(1, 2, 3, 4, 5)) / nv
    a_b, m_b, v_b, da = _brute(x, y)
    m, r = cb["scalar"]
    assert abs(cb["scalar_alpha"] - a_b) <= 2 * da
    assert m == pytest.approx(m_b, rel=1e-9, abs=abs(x.mean() - y.mean()) * 2 * da)
    assert (m * r) ** 2 == pytest.approx(v_b, rel=1e-5)


def test_infinite_medium_combination_is_the_collision_estimator():
    st, ss = 1.0, 0.8
    sa = st - ss
    n, width = (2, 2, 2), (1.0, 1.0, 1.0)
    mat = np.zeros(n, np.uint8)
    prob = W.box("inf_medium", n, width, mat, [[st]], [[ss / st]], np.eye(1)[None], (1.0,),
                 (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), None, (0, 0, 0), n, bc=(W.BC_REFLECT,) * 6)
    N, B = 400_000, 400
    cb = O.run(prob, N, seed=31, batches=B, estimator=O.EST_COMBINED)
    ce = O.run(prob, N, seed=31, batches=B, estimator=O.EST_COLLISION)
    tl = O.run(prob, N, seed=31, batches=B, estimator=O.EST_TRACK)
    m, r = cb["scalar"]
    var_c = ss / (sa ** 2 * st)          # collision score per history
    var_l = 1.0 / sa ** 2                # path length ~ Exponential(Sa)
    assert abs(m - 1.0 / sa) < 4.0 * math.sqrt(var_c / N)
    # a -> 0: the regression of the collision score on (L - C) has slope 0;
    # its standard error over B batches is sqrt(var_c / ((var_l - var_c) B))
    assert abs(cb["scalar_alpha"]) < 4.0 * math.sqrt(var_c / ((var_l - var_c) * B))
    assert r == pytest.approx(ce["scalar"][1], rel=0.05)
    assert r <= min(ce["scalar"][1], tl["scalar"][1]) * (1 + 1e-12)
    assert tl["scalar"][1] > 1.05 * ce["scalar"][1]   # the collision estimator is the better one


def test_combined_estimator_validated():
    prob = _td_box()
    with pytest.raises(ValueError):
        O.run(prob, 100, seed=1, batches=4, estimator=-1)
