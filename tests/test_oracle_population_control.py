"""Pins of the oracle's population control (a comb of the census bank at every
interior time edge; no value here comes from the CUDA path).

* the comb itself: teeth picks are in bank order; particle i gets floor or
  ceil of M w_i / W copies (systematic resampling); averaged over the comb
  offset its expected copy count is exactly M w_i / W;
* every comb keeps the bank's weight (W in = W out) and emits exactly M
  particles; the particle count balances: histories + combs' (out - in) =
  absorbed + leaked + censused + rouletted;
* identical particles (a beam in void): combing to the same count changes
  nothing, the tally equals the exact chords;
* infinite medium pulse: time-bin flux keeps its closed form
  (e^{-v Sa t_j} - e^{-v Sa t_j+1}) / Sa and the surviving weight is
  e^{-v Sa T}; the late bins get a smaller error than analog at equal N;
* multigroup time dependent (asymmetric transfer, per-group speeds): the
  matrix-exponential solution, so banked particles keep group and speed.
"""
import math

import numpy as np
import pytest
from scipy import linalg

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W


def test_comb_is_systematic_resampling():
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = int(rng.integers(1, 40))
        w = rng.uniform(0.0, 3.0, n) * (rng.uniform(size=n) < 0.8)
        w[0] += 0.1
        M = int(rng.integers(1, 60))
        xi = float(rng.uniform())
        sel = O.comb(w, M, xi)
        assert np.all(np.diff(sel) >= 0) and sel.min() >= 0 and sel.max() < n
        cnt = np.bincount(sel, minlength=n)
        share = M * w / w.sum()
        assert np.all(cnt >= np.floor(share - 1e-9)) and np.all(cnt <= np.ceil(share + 1e-9))
        assert np.all(cnt[w == 0] == 0)
    # averaged over the offset (midpoint rule), copies are M w_i / W exactly
    w = np.array([0.3, 1.7, 0.05, 2.2, 0.75])
    M, K = 7, 20000
    tot = np.zeros(5)
    for k in range(K):
        tot += np.bincount(O.comb(w, M, (k + 0.5) / K), minlength=5)
    np.testing.assert_allclose(tot / K, M * w / w.sum(), atol=2.0 / K)


def _inf_box(st, ss, G=1, transfer=None, speed=(1.0,), edges=None, src_pdf=None):
    if transfer is None:
        transfer = np.tile(np.eye(G), (1, 1, 1))
    mat = np.zeros((2, 2, 2), np.uint8)
    return W.box("inf_medium", (2, 2, 2), (1.0, 1.0, 1.0), mat, [list(np.atleast_1d(st))],
                 [list(np.atleast_1d(ss) / np.atleast_1d(st))], transfer, speed,
                 (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), edges, (0, 0, 0), (2, 2, 2),
                 bc=(W.BC_REFLECT,) * 6, src_pdf=src_pdf)


def balance_with_combs(c):
    return c["histories"] + c["pc_out"] - c["pc_in"] == (
        c["absorbed"] + c["leaked"] + c["censused"] + c["roulette_killed"])


def test_comb_conserves_weight_and_count():
    prob = W.c2_two_region()
    N, B, M = 20_000, 8, 1500
    res = O.run(prob, N, seed=3, batches=B, pc_target=M)
    c = res["counts"]
    assert c["pc_combs"] > 0 and c["pc_out"] == c["pc_combs"] * M
    assert c["w_pc_out"] == pytest.approx(c["w_pc_in"], rel=1e-12)
    assert balance_with_combs(c)


def test_comb_of_identical_particles_changes_nothing():
    # beam in void along x: every particle follows the same chord; combing
    # N identical unit-weight particles to N gives N unit-weight particles
    nb = 10
    edges = np.arange(0.0, 11.0, 1.0)           # speed 1: one cell per time bin
    prob = W.slab("void_beam", 10.0, nb, np.zeros(nb), [[0.0]], [[0.0]], src=(0.0, 0.0),
                  kind=W.SRC_BEAM, direction=(1.0, 0.0, 0.0), edges=edges)
    N, B = 400, 4
    a = O.run(prob, N, seed=1, batches=B)
    b = O.run(prob, N, seed=1, batches=B, pc_target=N // B)
    assert b["counts"]["pc_combs"] == B * 9
    np.testing.assert_allclose(b["sum1"], a["sum1"], rtol=1e-12)
    chord = np.zeros(prob.tally_shape)
    for i in range(nb):
        chord[0, 0, i, 0, i] = 1.0            # cell i is crossed during bin i
    np.testing.assert_allclose(a["mean"], chord, rtol=1e-12, atol=1e-12)


def test_population_control_pulse_unbiased_and_lower_late_error():
    st, ss, v = 1.0, 0.7, 2.0
    sa = st - ss
    edges = np.array([0.0, 0.5, 1.0, 2.0, 3.0, 5.0])
    prob = _inf_box(st, ss, speed=(v,), edges=edges)
    ref = (np.exp(-v * sa * edges[:-1]) - np.exp(-v * sa * edges[1:])) / sa
    # R independent replicas (each two combed simulations of 2500 histories)
    R, n = 24, 5000
    reps = {"pc": [], "analog": []}
    for r in range(R):
        for kind in reps:
            res = O.run(prob, n, seed=9, offset=r * n, batches=2,
                        pc_target=2500 if kind == "pc" else 0)
            reps[kind].append(res["sum1"].sum(axis=(0, 1, 2, 3)) / n)
            if kind == "pc":
                c = res["counts"]
                assert balance_with_combs(c) and c["pc_combs"] == 2 * 4
                assert c["w_pc_out"] == pytest.approx(c["w_pc_in"], rel=1e-12)
    pc, an = np.array(reps["pc"]), np.array(reps["analog"])
    se = pc.std(axis=0, ddof=1) / math.sqrt(R)
    z = (pc.mean(axis=0) - ref) / se
    assert np.all(np.abs(z) < 4.5), z
    # late bins: more, lighter particles than analog at the same N
    assert pc.std(axis=0, ddof=1)[-1] < 0.8 * an.std(axis=0, ddof=1)[-1]
    # the surviving (censused) weight is e^{-v Sa T}
    big = O.run(prob, 100_000, seed=4, batches=40, pc_target=2500)
    assert big["counts"]["w_censused"] / 100_000 == pytest.approx(
        math.exp(-v * sa * edges[-1]), rel=0.05)


def test_population_control_multigroup_time_dependent():
    st = np.array([1.0, 1.5, 2.0])
    c = np.array([0.6, 0.7, 0.5])
    P = np.array([[0.2, 0.5, 0.3],
                  [0.1, 0.3, 0.6],
                  [0.4, 0.0, 0.6]])
    q = np.array([0.5, 0.3, 0.2])
    v = np.array([3.0, 1.0, 0.5])
    edges = np.array([0.0, 0.4, 1.0, 2.0, 4.0])
    prob = _inf_box(st, st * c, G=3, transfer=P[None], speed=tuple(v), edges=edges, src_pdf=q)
    N = 100_000
    res = O.run(prob, N, seed=33, batches=40, pc_target=2500)
    S = (st * c)[:, None] * P
    A = (S.T - np.diag(st)) @ np.diag(v)
    Ainv = np.linalg.inv(A)
    ref = np.zeros((3, len(edges) - 1))
    for j in range(len(edges) - 1):
        ref[:, j] = v * (Ainv @ (linalg.expm(A * edges[j + 1]) - linalg.expm(A * edges[j])) @ q)
    tot = res["sum1"].sum(axis=(0, 1, 2)) / N
    big = ref > 0.02
    assert np.max(np.abs(tot[big] - ref[big]) / ref[big]) < 0.03, (tot, ref)
    assert balance_with_combs(res["counts"])


def test_population_control_options_validated():
    p = W.c2_two_region()
    with pytest.raises(ValueError):          # weight windows and a comb
        O.run(p, 100, 1, batches=4, pc_target=10, ww={"lower": np.ones(p.n_bins)})
    import dataclasses
    with pytest.raises(ValueError):          # a source past the first census edge
        O.run(dataclasses.replace(p, src_t1=1.0), 100, 1, batches=4, pc_target=10)
    with pytest.raises(ValueError):          # steady state: no census edges
        O.run(W.c1_slab(), 100, 1, batches=4, pc_target=10)
    with pytest.raises(ValueError):          # no per-history trace under a comb
        O.trace(p, 1, np.arange(3), pc_target=10)
