"""Pins of the oracle's collision estimator and implicit capture (no value here
comes from the CUDA path).

* collision estimator (every collision scores w / sigma_t into the bin of the
  arriving particle):
  - exact: with unit weights every collision adds exactly 1/sigma_t, so the
    summed tally equals (number of collisions) / sigma_t, and choosing the
    estimator changes no history (identical event counts);
  - pure absorber beam: the score of bin i is 1/sigma_t with probability
    p_i = e^{-St x_i} - e^{-St x_i+1}, so mean and variance are exact;
  - infinite medium: K collisions per history, K ~ Geometric(Sa/St), so the
    total score K/St has mean 1/Sa and variance Ss/(Sa^2 St) exactly;
  - infinite medium pulse: expected score per time bin equals the time
    integral of the flux, (e^{-v Sa t_j} - e^{-v Sa t_j+1}) / Sa;
  - multigroup (asymmetric transfer, per-group sigma_t): the linear solve
    (diag St - S^T) phi = q; scoring with the post-collision group fails it.
* implicit capture (weight times sigma_s/sigma_t at every collision, roulette
  below a cutoff):
  - pure absorber: the weight drops to zero at the first collision, so the
    run is the analog one exactly (tallies and counts);
  - infinite medium pulse with a cutoff no weight reaches: every history is
    censused, source weight = absorbed + censused weight to rounding, and the
    time-bin flux keeps its closed form;
  - infinite medium steady state with the roulette active: unbiased flux 1/Sa;
  - multigroup with both options: the linear solve again (the weight factor
    of the group the particle collides in; the new group's factor fails it).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W


def _inf_box(st, ss, G=1, transfer=None, speed=(1.0,), edges=None, src_pdf=None):
    if transfer is None:
        transfer = np.tile(np.eye(G), (1, 1, 1))
    n, width = (2, 2, 2), (1.0, 1.0, 1.0)
    mat = np.zeros((2, 2, 2), np.uint8)
    return W.box("inf_medium", n, width, mat, [list(np.atleast_1d(st))],
                 [list(np.atleast_1d(ss) / np.atleast_1d(st))], transfer, speed,
                 (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), edges, (0, 0, 0), n, bc=(W.BC_REFLECT,) * 6,
                 src_pdf=src_pdf)


def test_collision_estimator_scores_one_over_sigma_t_per_collision():
    st, ss = 2.0, 1.6          # 1/st = 0.5 exactly; sums of halves are exact
    prob = _inf_box(st, ss)
    N = 20_000
    tl = O.run(prob, N, seed=41, batches=20)
    ce = O.run(prob, N, seed=41, batches=20, estimator=O.EST_COLLISION)
    assert ce["counts"] == tl["counts"]           # the estimator changes no history
    assert ce["sum1"].sum() == ce["counts"]["collisions"] / st
    assert tl["sum1"].sum() != ce["sum1"].sum()   # the two estimators differ per run


def test_collision_estimator_pure_absorber_beam():
    L, nb, st = 5.0, 25, 1.0
    prob = W.slab("absorber_beam", L, nb, np.zeros(nb), [[st]], [[0.0]], src=(0.0, 0.0),
                  kind=W.SRC_BEAM, direction=(1.0, 0.0, 0.0))
    N = 200_000
    res = O.run(prob, N, seed=3, batches=40, estimator=O.EST_COLLISION)
    dx = L / nb
    x = np.arange(nb) * dx
    p = np.exp(-st * x) - np.exp(-st * (x + dx))
    mean = p / st / dx
    sig = np.sqrt(p * (1 - p) / N) / st / dx
    z = (res["mean"].reshape(-1) - mean) / sig
    assert np.all(np.abs(z) < 4.5), np.abs(z).max()
    # the same histories as the track-length run
    tl = O.run(prob, N, seed=3, batches=40)
    assert tl["counts"] == res["counts"]


def test_collision_estimator_infinite_medium_geometric_law():
    st, ss = 1.0, 0.8
    sa = st - ss
    prob = _inf_box(st, ss)
    N = 100_000
    res = O.run(prob, N, seed=5, batches=50, estimator=O.EST_COLLISION)
    m, r = res["scalar"]                 # total score per history (V_cell = 1)
    var = ss / (sa ** 2 * st)
    assert abs(m - 1.0 / sa) < 4.0 * math.sqrt(var / N)
    assert r == pytest.approx(math.sqrt(var) / (1.0 / sa) / math.sqrt(N), rel=0.4)
    assert res["counts"]["absorbed"] == N


def test_collision_estimator_pulse_time_bins():
    st, ss, v = 1.0, 0.7, 2.0
    sa = st - ss
    edges = np.array([0.0, 0.5, 1.0, 2.0, 3.0, 5.0])
    prob = _inf_box(st, ss, speed=(v,), edges=edges)
    N = 100_000
    res = O.run(prob, N, seed=9, batches=40, estimator=O.EST_COLLISION)
    tot = res["sum1"].sum(axis=(0, 1, 2, 3)) / N
    ref = (np.exp(-v * sa * edges[:-1]) - np.exp(-v * sa * edges[1:])) / sa
    # bound: score per history <= K/St with E[K^2] = (2 - p)/p^2, p = Sa/St
    p = sa / st
    sig = math.sqrt((2 - p) / p ** 2 / st ** 2 / N)
    assert np.all(np.abs(tot - ref) < 4.5 * sig), (tot, ref)


def _multigroup_data():
    st = np.array([1.0, 1.5, 2.0])
    c = np.array([0.6, 0.7, 0.5])
    P = np.array([[0.2, 0.5, 0.3],
                  [0.1, 0.3, 0.6],
                  [0.4, 0.0, 0.6]])
    q = np.array([0.5, 0.3, 0.2])
    return st, c, P, q


@pytest.mark.parametrize("implicit", [None, (0.05, 0.1)])
def test_collision_estimator_multigroup_steady(implicit):
    st, c, P, q = _multigroup_data()
    prob = _inf_box(st, st * c, G=3, transfer=P[None], speed=(1.0, 1.0, 1.0), src_pdf=q)
    N = 100_000
    res = O.run(prob, N, seed=21, batches=40, estimator=O.EST_COLLISION, implicit=implicit)
    S = (st * c)[:, None] * P
    phi = np.linalg.solve(np.diag(st) - S.T, q)
    tot = res["sum1"].sum(axis=(0, 1, 2, 4)) / N
    assert np.max(np.abs(tot - phi) / phi) < 0.025, (tot, phi)
    # weighting by the ratio of the group scattered into (a plausible slip)
    # or scoring after the group change would change phi by far more
    wrong = np.linalg.solve(np.diag(st) - (S * (c[None, :] / c[:, None])).T, q)
    assert np.max(np.abs(wrong - phi) / phi) > 0.08


def test_implicit_capture_pure_absorber_is_analog():
    L, nb, st = 5.0, 25, 1.0
    prob = W.slab("absorber_beam", L, nb, np.zeros(nb), [[st]], [[0.0]], src=(0.0, 0.0),
                  kind=W.SRC_BEAM, direction=(1.0, 0.0, 0.0))
    N = 50_000
    a = O.run(prob, N, seed=13, batches=20)
    b = O.run(prob, N, seed=13, batches=20, implicit=(0.25, 0.5))
    assert np.array_equal(a["sum1"], b["sum1"])
    assert a["counts"]["absorbed"] == b["counts"]["absorbed"]
    assert b["counts"]["roulette_killed"] == 0
    dx = L / nb
    x = np.arange(nb) * dx
    mean = (np.exp(-st * x) - np.exp(-st * (x + dx))) / st / dx
    assert np.max(np.abs(b["mean"].reshape(-1) - mean) / mean) < 0.05


def test_implicit_capture_pulse_weight_balance_and_time_bins():
    st, ss, v = 1.0, 0.7, 2.0
    sa = st - ss
    edges = np.array([0.0, 0.5, 1.0, 2.0, 3.0, 5.0])
    prob = _inf_box(st, ss, speed=(v,), edges=edges)
    N = 100_000
    res = O.run(prob, N, seed=9, batches=40, implicit=(1e-200, 1e-199))
    c = res["counts"]
    # nothing can end a history before the last census: no absorption kills
    assert c["absorbed"] == 0 and c["roulette_killed"] == 0 and c["censused"] == N
    # weight leaves only through absorption (implicit) and the last census
    assert c["w_source"] == N
    assert abs(c["w_absorbed"] + c["w_censused"] - N) < 1e-9 * N
    # the surviving weight is the survival probability e^{-v Sa T}
    assert abs(c["w_censused"] / N - math.exp(-v * sa * edges[-1])) < 1e-2
    tot = res["sum1"].sum(axis=(0, 1, 2, 3)) / N
    ref = (np.exp(-v * sa * edges[:-1]) - np.exp(-v * sa * edges[1:])) / sa
    # bound: weight <= 1, so a bin's score <= v * its width
    sig = v * np.diff(edges) / math.sqrt(N)
    assert np.all(np.abs(tot - ref) < 4.5 * sig), (tot, ref)


def test_implicit_capture_with_roulette_unbiased():
    st, ss = 1.0, 0.8
    sa = st - ss
    prob = _inf_box(st, ss)
    N = 100_000
    res = O.run(prob, N, seed=17, batches=50, implicit=(0.25, 0.5))
    c = res["counts"]
    assert c["roulette_killed"] > 0 and c["roulette_survived"] > 0
    assert c["absorbed"] == 0
    assert c["roulette_killed"] == N        # the only way a history ends here
    m, r = res["scalar"]
    assert abs(m - 1.0 / sa) < 4.0 * m * r
    assert r < 1.0 / math.sqrt(N)           # lower variance than analog (exactly 1/sqrt(N))


def test_estimator_options_validated():
    prob = _inf_box(1.0, 0.5)
    with pytest.raises(ValueError):
        O.run(prob, 100, seed=1, batches=4, implicit=(0.5, 0.25))
    with pytest.raises(ValueError):
        O.run(prob, 100, seed=1, batches=4, implicit=(0.0, 0.5))
    with pytest.raises(ValueError):
        O.run(prob, 100, seed=1, batches=4, estimator=3)
