"""Pins of the oracle's per-event network windows (R15; no value here comes
from the CUDA path).

* inputs: the position and time inputs are the training's cell-centre and
  bin-centre values at those points, -1 and +1 at the mesh and time edges;
* reduction to the table (R9): a network whose output depends only on the
  group (no weight on position or time) gives, event for event, the run with
  the table of its values (identical tallies and counts);
* unbiasedness: spatially varying network windows leave the infinite-medium
  flux at its closed form 1 / Sigma_a, with splits and roulettes happening;
* a network over the position alone (3 inputs) is, event for event, the
  full-input network whose time and group weights are zero.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W


def _box(G=2, T=4):
    n, width = (4, 3, 2), (0.5, 1.0, 1.5)
    mat = np.zeros((2, 3, 4), np.uint8)
    P = np.tile(np.full((G, G), 1.0 / G), (1, 1, 1))
    edges = np.linspace(0.0, 4.0, T + 1) if T else None
    return W.box("net_box", n, width, mat, [[1.0] * G], [[0.8] * G], P, [1.0] * G,
                 (0.0, 0.0, 0.0), (2.0, 3.0, 3.0), edges, (0, 0, 0), n,
                 bc=(W.BC_REFLECT,) * 6, src_pdf=[1.0 / G] * G)


def test_inputs_at_centres_edges_and_bins():
    prob = _box()
    # cell (i, j, k) centre -> 2 (i + 0.5) / n - 1 on each axis; bin centre in time
    f = O.net_features(prob, 0.25 * 3, 0.5 * 1 + 1.0 * 1, 0.75 + 1.5 * 1, 1.5, 1, 1)
    assert f[0] == pytest.approx(2 * 1.5 / 4 - 1)
    assert f[1] == pytest.approx(2 * 1.5 / 3 - 1)
    assert f[2] == pytest.approx(2 * 1.5 / 2 - 1)
    assert f[3] == pytest.approx(2 * 1.5 / 4 - 1)
    assert list(f[4:]) == [0.0, 1.0]
    lo = O.net_features(prob, 0.0, 0.0, 0.0, 0.0, 0, 0)
    hi = O.net_features(prob, 2.0, 3.0, 3.0, 4.0, 3, 1)
    assert list(lo[:4]) == [-1.0, -1.0, -1.0, -1.0] and list(lo[4:]) == [1.0, 0.0]
    assert list(hi[:4]) == [1.0, 1.0, 1.0, 1.0]
    # inside a cell and a bin the inputs move continuously
    f = O.net_features(prob, 0.6, 1.2, 0.3, 1.25, 1, 0)
    assert f[0] == pytest.approx(2 * 0.6 / 2.0 - 1)
    assert f[1] == pytest.approx(2 * 1.2 / 3.0 - 1)
    assert f[2] == pytest.approx(2 * 0.3 / 3.0 - 1)
    assert f[3] == pytest.approx(2 * (1 + 0.25) / 4 - 1)
    steady = _box(T=0)
    assert O.net_features(steady, 1.0, 1.0, 1.0, 0.0, 0, 0)[3] == 0.0


def _net(n_in, H, rng, position_weight=1.0):
    npar = H * n_in + H + H * H + H + H + 1
    p = rng.normal(0.0, 0.5, npar)
    W1 = p[:H * n_in].reshape(H, n_in)
    W1[:, :4] *= position_weight          # 0: the output depends on the group only
    return p


def test_group_only_network_equals_its_table():
    prob = _box()
    G, T = 2, 4
    n_in, H = 4 + G, 8
    p = _net(n_in, H, np.random.default_rng(3), position_weight=0.0)
    net = {"net": p, "hidden": H, "shift": -0.5, "scale": 2.0, "top": 1.0, "floor": -3.0,
           "wl0": 0.6, "upper_ratio": 4.0, "survival_ratio": 2.0, "nmax": 8}
    # the table of the same windows: w_L(g) = wl0 exp(min(0, max(lp, floor) - top))
    wl = []
    for g in range(G):
        f = np.zeros(n_in)
        f[4 + g] = 1.0
        y = O.mlp_forward(p, f[None, :], hidden=H)[0]
        lp = max(y * 2.0 - 0.5, -3.0)
        wl.append(0.6 * np.exp(min(0.0, lp - 1.0)))
    cells = int(np.prod(prob.n))
    table = np.tile(np.repeat(np.array(wl), T), cells)
    tab = {"lower": table, "upper_ratio": 4.0, "survival_ratio": 2.0, "nmax": 8}
    a = O.run(prob, 4000, seed=5, batches=8, ww=net, threads=2)
    b = O.run(prob, 4000, seed=5, batches=8, ww=tab, threads=2)
    assert a["counts"] == b["counts"]
    assert a["counts"]["splits"] > 0 or a["counts"]["roulette_killed"] > 0
    np.testing.assert_allclose(a["sum1"], b["sum1"], rtol=1e-12, atol=0)


def test_varying_network_windows_are_unbiased():
    prob = _box(T=0)                      # steady infinite medium: flux 1 / Sigma_a per cell
    n_in, H = 6, 8
    p = _net(n_in, H, np.random.default_rng(11))
    net = {"net": p, "hidden": H, "shift": 0.0, "scale": 1.5, "top": 2.0, "floor": -4.0,
           "wl0": 0.5, "upper_ratio": 4.0, "survival_ratio": 2.0, "nmax": 8}
    res = O.run(prob, 40_000, seed=9, batches=40, ww=net)
    c = res["counts"]
    assert c["splits"] > 1000 and c["roulette_killed"] > 1000
    # region scalar: the sum of the 24 cells' fluxes, each 1 / (Sigma_a V_box)
    # with V_box = 2 x 3 x 3
    m, r = res["scalar"]
    ref = 24.0 / (0.2 * 18.0)
    assert abs(m - ref) < 4.0 * m * r, (m, ref, r)


def test_position_only_network_equals_full_network_without_time_and_group():
    prob = _box()
    G, H = 2, 8
    rng = np.random.default_rng(19)
    p3 = _net(3, H, rng)
    W1 = p3[:H * 3].reshape(H, 3)
    full = np.concatenate([np.concatenate([W1, np.zeros((H, 1 + G))], axis=1).ravel(),
                           p3[H * 3:]])
    consts = {"hidden": H, "shift": -0.3, "scale": 2.0, "top": 1.0, "floor": -3.0,
              "wl0": 0.6, "upper_ratio": 4.0, "survival_ratio": 2.0, "nmax": 8}
    f3 = O.net_features(prob, 0.6, 1.2, 0.3, 1.25, 1, 0, n_in=3)
    assert f3.shape == (3,)
    np.testing.assert_array_equal(f3, O.net_features(prob, 0.6, 1.2, 0.3, 1.25, 1, 0)[:3])
    a = O.run(prob, 4000, seed=7, batches=8, ww={"net": p3, "n_in": 3, **consts}, threads=2)
    b = O.run(prob, 4000, seed=7, batches=8, ww={"net": full, **consts}, threads=2)
    assert a["counts"] == b["counts"]
    assert a["counts"]["splits"] > 0 and a["counts"]["roulette_killed"] > 0
    np.testing.assert_allclose(a["sum1"], b["sum1"], rtol=1e-12, atol=0)
