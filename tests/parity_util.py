"""Comparison helpers of the GPU parity tests (FP64 event-exact records,
tallies to relative 1e-9, exact event counts) and a scaled-down channel
problem.  No test functions here."""
import numpy as np

from paper_2409_04668_b300 import workloads as W

REL_TALLY = 1e-9


def small_channel(n=12, G=7, T=8, seed=3):
    """A scaled-down copy of the channel problem: same materials, groups,
    speeds and time grid shape on an n^3 mesh."""
    full = W.c3_channel(seed)
    f = 60 // n
    mat = full.material[::f, ::f, ::f].copy()
    return W.box("channel_small", (n, n, n), (1.0 * f,) * 3, mat, full.sigma_t, full.sigma_s /
                 full.sigma_t, full.transfer, full.speed, (0.0,) * 3, (10.0,) * 3,
                 np.linspace(0.0, 1e-6, T + 1), (n // 2,) * 3, (n,) * 3)


def compare_records(gpu, orc, dim):
    assert np.array_equal(gpu["hid"], orc["hid"])
    for f in ("end", "g", "ctr", "n_seg", "n_col", "n_cross"):
        bad = np.nonzero(gpu[f] != orc[f])[0]
        assert bad.size == 0, (f, bad[:10], gpu[f][bad[:5]], orc[f][bad[:5]])
    axes = ("x", "t") if dim == 1 else ("x", "y", "z", "t")
    for f in axes:
        np.testing.assert_allclose(gpu[f], orc[f], rtol=1e-12, atol=1e-12 * (1 + np.abs(orc[f]).max()))
    np.testing.assert_allclose(gpu["w"], orc["w"], rtol=1e-12)


def compare_tallies(g, o):
    for key in ("sum1", "sum2"):
        a, b = g[key], o[key]
        scale = np.maximum(np.abs(b), 1e-300)
        rel = np.abs(a - b) / scale
        assert np.all((rel <= REL_TALLY) | (np.abs(a - b) <= 1e-300)), (key, rel.max())
    nz = o["mean"] != 0
    np.testing.assert_allclose(g["mean"][nz], o["mean"][nz], rtol=REL_TALLY)
    np.testing.assert_array_equal(g["mean"] == 0, o["mean"] == 0)
    np.testing.assert_allclose(g["relerr"], o["relerr"], rtol=1e-6, atol=1e-12)


COUNT_KEYS = ("histories", "segments", "collisions", "crossings", "census", "absorbed", "leaked",
              "censused", "splits", "children", "roulette_killed", "roulette_survived")


def allowed_exceedances(n_bins, dof, z=4.0, p_fail=1e-3):
    """The most bins that may show |z| > z by chance: the smallest k with
    P(X > k) < p_fail for X ~ Binomial(n_bins, p), p the two-sided tail of
    Student's t with `dof` degrees of freedom (a difference of two batch
    means whose spreads are estimated from `dof` + 1 batches each; Welch's
    combination has at least that many degrees of freedom, so the tail is
    not underestimated)."""
    from scipy import stats
    p = 2.0 * stats.t.sf(z, dof)
    k = 0
    while stats.binom.sf(k, n_bins, p) >= p_fail:
        k += 1
    return k


def fp32_bins_agree(g, o, batches, rel_max=0.25):
    """Per-bin statistical agreement of an FP32 run with an independent
    oracle run: over the bins both estimate well (relative error <= rel_max)
    |z| > 4 at most as often as chance allows (allowed_exceedances, with the
    smaller run's batch count); every bin the oracle estimates well is
    scored by the GPU.  Returns (exceedances, bins, allowed)."""
    gm, gr, om, orr = g["mean"], g["relerr"], o["mean"], o["relerr"]
    well_o = (om != 0) & (orr <= rel_max)
    assert np.all(gm[well_o] != 0), int((gm[well_o] == 0).sum())
    both = well_o & (gm != 0) & (gr <= rel_max)
    s = np.sqrt((gm * gr) ** 2 + (om * orr) ** 2)[both]
    z = (gm - om)[both] / s
    n = int((np.abs(z) > 4).sum())
    nb = int(both.sum())
    k = allowed_exceedances(nb, batches - 1)
    assert n <= k, (n, nb, k)
    return n, nb, k


def compare_counts(g, o):
    for k in COUNT_KEYS:
        assert g[k] == o[k], (k, g[k], o[k])
