"""Per-event network weight windows on the GPU against the oracle.

The lower bound of every window check comes from the importance network
evaluated at the particle (position, time, group), not from a table.  FP64
mode takes the same decisions as the oracle given the same FP32 parameters
(both evaluate in FP64 from them), so tallies agree bin by bin to 1e-9 and
event counts exactly; the FP32 modes evaluate the network in FP32 and are
checked against a closed form (an infinite medium's flux is 1 / Sigma_a
whatever the windows do, as long as they are unbiased).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W
from parity_util import compare_counts, compare_tallies, small_channel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def _params(n_in, H, seed, sd=0.5):
    """Random parameters, rounded to FP32 (what the GPU stores) for both sides."""
    npar = H * n_in + H + H * H + H + H + 1
    return np.random.default_rng(seed).normal(0.0, sd, npar).astype(np.float32)


def _consts(H, shift, scale, top, floor, wl0, up=5.0, surv=2.5, nmax=16):
    return dict(hidden=H, shift=shift, scale=scale, top=top, floor=floor, wl0=wl0,
                upper_ratio=up, survival_ratio=surv, nmax=nmax)


def _run_gpu(mcdc, prob, p, c, N, seed, B, precision, **opts):
    with mcdc.Problem(prob, precision=precision, tally_mode=mcdc.TALLY_GLOBAL, **opts) as P:
        P.set_network_windows(p, c["hidden"], c["shift"], c["scale"], c["top"], c["floor"],
                              c["wl0"], c["upper_ratio"], c["survival_ratio"], c["nmax"])
        s1, s2, mean, rel = (np.zeros(P.n_bins) for _ in range(4))
        stats, scal = P.run_ex(N, seed, batches=B, sum1=s1, sum2=s2, mean=mean, relerr=rel)
    g = {"sum1": s1.reshape(prob.tally_shape), "sum2": s2.reshape(prob.tally_shape),
         "mean": mean.reshape(prob.tally_shape), "relerr": rel.reshape(prob.tally_shape)}
    return g, stats, scal


def _oracle_ww(p, c):
    return {"net": p.astype(np.float64), **c}


@pytest.mark.parametrize("H,shift", [(8, -5.65), (64, 0.32)])
def test_fp64_channel_matches_oracle(mcdc, H, shift):
    """3-D, 7 groups, 8 time bins, leakage: 11 inputs, the widest hidden layer.
    Lower bounds up to 2 (above the source weight: roulettes) and down to
    2 e^-6 (splits)."""
    prob = small_channel()
    n_in = 4 + prob.sigma_t.shape[1]
    p = _params(n_in, H, seed=H, sd=0.5 if H == 8 else 0.2)
    c = _consts(H, shift=shift, scale=6.0, top=0.0, floor=-6.0, wl0=2.0)
    N, B = 20_000, 8
    g, stats, scal = _run_gpu(mcdc, prob, p, c, N, 17, B, mcdc.PREC_FP64)
    o = O.run(prob, N, seed=17, batches=B, ww=_oracle_ww(p, c))
    compare_tallies(g, o)
    compare_counts(stats, o["counts"])
    assert stats["splits"] > 100 and stats["roulette_killed"] > 100, stats


def test_fp64_slab_matches_oracle(mcdc):
    """1-D two-region slab (unbounded y and z: those inputs are 0), ragged batches."""
    prob = W.c2_two_region()
    n_in, H = 5, 16
    p = _params(n_in, H, seed=5)
    c = _consts(H, shift=-0.7, scale=6.0, top=0.0, floor=-6.0, wl0=2.0)
    N, B = 30_001, 7
    g, stats, scal = _run_gpu(mcdc, prob, p, c, N, 23, B, mcdc.PREC_FP64)
    o = O.run(prob, N, seed=23, batches=B, ww=_oracle_ww(p, c))
    compare_tallies(g, o)
    compare_counts(stats, o["counts"])
    assert stats["splits"] > 100 and stats["roulette_killed"] > 100, stats


def _infinite_box(G=2):
    n, width = (4, 3, 2), (0.5, 1.0, 1.5)
    mat = np.zeros((2, 3, 4), np.uint8)
    P = np.full((1, G, G), 1.0 / G)
    return W.box("net_box", n, width, mat, [[1.0] * G], [[0.8] * G], P, [1.0] * G,
                 (0.0, 0.0, 0.0), (2.0, 3.0, 3.0), None, (0, 0, 0), n,
                 bc=(W.BC_REFLECT,) * 6, src_pdf=[1.0 / G] * G)


@pytest.mark.parametrize("prec", ["fp32", "fp32_local", "fp64"])
def test_infinite_medium_flux_is_unbiased(mcdc, prec):
    """Strongly varying windows (splits and roulettes by the million) leave the
    region total at its closed form: 24 cells of flux 1 / (Sigma_a V_box)."""
    pr = {"fp32": mcdc.PREC_FP32, "fp32_local": mcdc.PREC_FP32_LOCAL,
          "fp64": mcdc.PREC_FP64}[prec]
    prob = _infinite_box()
    p = _params(6, 8, seed=11)
    c = _consts(8, shift=0.0, scale=1.5, top=2.0, floor=-4.0, wl0=0.5, up=4.0, surv=2.0, nmax=8)
    N = 1_000_000
    g, stats, scal = _run_gpu(mcdc, prob, p, c, N, 9, 40, pr)
    assert stats["splits"] > 100_000 and stats["roulette_killed"] > 100_000, stats
    m, r = scal
    ref = 24.0 / (0.2 * 18.0)
    print(prec, "region total", m, "closed form", ref, "relerr", r)
    assert abs(m - ref) < 4.0 * m * r, (m, ref, r)
    assert r < 2e-3


def test_switching_and_refusals(mcdc):
    """Turning the windows off restores the analog run event for event; the shared
    tally, population control and bad constants are refused."""
    prob = W.c2_two_region()
    p = _params(5, 8, seed=2)
    c = _consts(8, shift=0.0, scale=1.0, top=0.0, floor=-3.0, wl0=0.3)
    N = 50_000
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, tally_mode=mcdc.TALLY_GLOBAL) as P:
        a = np.zeros(P.n_bins)
        sa, _ = P.run_ex(N, 4, batches=4, sum1=a)
        P.set_network_windows(p, 8, c["shift"], c["scale"], c["top"], c["floor"], c["wl0"])
        w = np.zeros(P.n_bins)
        st, _ = P.run_ex(N, 4, batches=4, sum1=w)
        assert st["splits"] + st["roulette_killed"] > 0
        P.set_network_windows(None, 8, 0.0, 1.0, 0.0, -3.0, 0.3)
        b = np.zeros(P.n_bins)
        st, _ = P.run_ex(N, 4, batches=4, sum1=b)
        assert st["splits"] == 0 and st["roulette_killed"] == 0
        for k in ("segments", "collisions", "crossings", "census", "absorbed", "leaked",
                  "censused", "children"):
            assert st[k] == sa[k], k
        # the same events; the sums differ only in the order of the tally's atomic adds
        np.testing.assert_allclose(b, a, rtol=1e-12)
        assert np.abs(w - a).max() > 1e-6 * np.abs(a).max()
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, tally_mode=mcdc.TALLY_SHARED) as P:
        with pytest.raises(mcdc.MCDCError, match="global tally"):
            P.set_network_windows(p, 8, 0.0, 1.0, 0.0, -3.0, 0.3)
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32, tally_mode=mcdc.TALLY_GLOBAL,
                      pc_target=1000) as P:
        with pytest.raises(mcdc.MCDCError, match="population control"):
            P.set_network_windows(p, 8, 0.0, 1.0, 0.0, -3.0, 0.3)
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32, tally_mode=mcdc.TALLY_GLOBAL) as P:
        with pytest.raises(mcdc.MCDCError, match="hidden"):
            P.set_network_windows(p, 65, 0.0, 1.0, 0.0, -3.0, 0.3)
        with pytest.raises(mcdc.MCDCError, match="finite"):
            P.set_network_windows(p, 8, np.nan, 1.0, 0.0, -3.0, 0.3)


def test_network_kernels_take_their_own_launch_shape(mcdc):
    """The network instantiations run 384 threads per CTA whatever shape the
    autotuner chose for the analog kernel (their registers fit one such CTA
    per SM), fewer only when the caller asked for fewer; the caller's own
    CTAs per SM must fit.  Turning the windows off restores the analog shape."""
    prob = W.c2_two_region()
    p = _params(5, 8, seed=2)
    c = _consts(8, shift=0.0, scale=1.0, top=0.0, floor=-3.0, wl0=0.3)
    for kw, want in (({}, 384), ({"block_size": 512}, 384), ({"block_size": 256}, 256)):
        with mcdc.Problem(prob, precision=mcdc.PREC_FP32_LOCAL, tally_mode=mcdc.TALLY_GLOBAL,
                          **kw) as P:
            st0, _ = P.run_ex(20_000, 3, batches=4)
            P.set_network_windows(p, 8, c["shift"], c["scale"], c["top"], c["floor"], c["wl0"])
            st, _ = P.run_ex(20_000, 3, batches=4)
            assert st["block_size"] == want, (kw, st["block_size"])
            assert st["ctas_per_sm"] >= 1
            P.set_network_windows(None, 8, 0.0, 1.0, 0.0, -3.0, 0.3)
            st1, _ = P.run_ex(20_000, 3, batches=4)
            assert (st1["block_size"], st1["ctas_per_sm"]) == (st0["block_size"], st0["ctas_per_sm"])
            assert st1["segments"] == st0["segments"]
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32_LOCAL, tally_mode=mcdc.TALLY_GLOBAL,
                      block_size=256, ctas_per_sm=2) as P:
        st0, _ = P.run_ex(20_000, 3, batches=4)
        P.set_weight_windows(np.full(P.n_bins, 0.1), 5.0, 2.5, 16)   # w = 1 splits in two
        stw, _ = P.run_ex(20_000, 3, batches=4)
        with pytest.raises(mcdc.MCDCError, match="ctas_per_sm"):
            P.set_network_windows(p, 8, c["shift"], c["scale"], c["top"], c["floor"], c["wl0"])
        # the refused network left the table windows and their kernel in place
        st, _ = P.run_ex(20_000, 3, batches=4)
        assert (st["block_size"], st["ctas_per_sm"]) == (256, 2)
        for k in ("segments", "splits", "roulette_killed"):
            assert st[k] == stw[k], k
        assert stw["splits"] + stw["roulette_killed"] > 0 and st0["splits"] == 0


@pytest.mark.parametrize("time_resolved", [0, 1])
@pytest.mark.parametrize("prec", ["fp32", "fp32_local"])
def test_trained_network_per_event_is_unbiased(mcdc, time_resolved, prec):
    """The importance network trained on a pilot tally and evaluated at every
    window check (no baked table): the region total of the two-region slab
    (one group, 50 time bins) agrees with an independent analog run within the
    combined noise.  With the time fold (default) the windows come from a
    position network fitted to the folded table, which its windows at the
    cell centres must follow; time-resolved, from the trained network itself,
    whose windows split and roulette by the thousand."""
    prob = W.c2_two_region()
    pr = {"fp32": mcdc.PREC_FP32, "fp32_local": mcdc.PREC_FP32_LOCAL}[prec]
    with mcdc.Problem(prob, precision=pr, tally_mode=mcdc.TALLY_GLOBAL) as P:
        mean, rel = np.zeros(P.n_bins), np.zeros(P.n_bins)
        _, (m_a, r_a) = P.run_ex(4_000_000, 3, batches=32, mean=mean, relerr=rel)
        rep = P.train_importance(mean, rel, epochs=6, batch=16384, per_event=1,
                                 time_resolved=time_resolved)
        assert rep["steps"] > 0 and rep["bake_ms"] >= 0.0
        if time_resolved:
            assert rep["distill_steps"] == 0
        else:
            assert rep["distill_steps"] >= 8000 and rep["distill_loss"] < 0.01, rep
            table = P.get_weight_windows().reshape(prob.tally_shape)
            cells = table.reshape(prob.n[0], -1)[:, 0]     # the folded table: one value per cell
            xc = np.zeros((prob.n[0], 3))
            xc[:, 0] = prob.origin[0] + (np.arange(prob.n[0]) + 0.5) * prob.width[0]
            wl = P.network_window_lower(xc, np.full(prob.n[0], 0.5 * prob.edges[1]),
                                        np.zeros(prob.n[0], np.int32))
            dev = np.abs(np.log(wl) - np.log(cells))
            print(prec, "position network against the table: max |log ratio|", dev.max(),
                  "table range", cells.min(), cells.max())
            assert np.all(wl > 0) and dev.max() < 0.1, (dev.max(), np.argmax(dev))
        st, (m_w, r_w) = P.run_ex(2_000_000, 11, batches=32)
    if time_resolved:
        assert st["splits"] + st["roulette_killed"] > 1000, st
    se = np.hypot(m_a * r_a, m_w * r_w)
    print("analog", m_a, r_a, "per-event windows", m_w, r_w, "splits", st["splits"])
    assert abs(m_w - m_a) < 4.0 * se, (m_w, m_a, se)

def _states(prob, n, seed):
    """Random particle states inside the mesh: positions on the bounded axes (0
    on an unbounded one), times inside the census grid, groups."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 3))
    for a in range(3):
        if np.isfinite(prob.width[a]):
            lo = prob.origin[a]
            x[:, a] = rng.uniform(lo, lo + prob.n[a] * prob.width[a], n)
    e = prob.edges
    t = rng.uniform(e[0], e[-1], n) if e is not None else np.zeros(n)
    g = rng.integers(0, prob.sigma_t.shape[1], n).astype(np.int32)
    return x, t, g


def _oracle_lower(prob, p, n_in, H, c, x, t, g):
    """The oracle's inputs for each state, its log w_L from the exact network,
    and the first-order bound on the warp-batched evaluation's error in log w_L
    (binary16 operands, FP32 sums, SiLU through tanh.approx taken within 2^-9,
    FP32 inputs)."""
    e = prob.edges
    T = 0 if e is None else len(e) - 1
    tb = np.clip(np.searchsorted(e, t, side="right") - 1, 0, T - 1) if T else np.zeros(len(t), int)
    F = np.array([O.net_features(prob, *x[i], t[i], tb[i], g[i], n_in=n_in)
                  for i in range(len(t))]).reshape(len(t), n_in)
    pd = p.astype(np.float64)
    y = O.mlp_forward(pd, F, hidden=H)
    fb = O.mlp_window_bound(pd, F, hidden=H)

    def logw(v):
        lp = np.maximum(v * c["scale"] + c["shift"], c["floor"])
        return np.log(c["wl0"]) + np.minimum(0.0, lp - c["top"])
    return logw(y), fb * abs(c["scale"])


WINDOW_CASES = {
    # 3-D channel, 7 groups, 8 time bins: 11 inputs (two K steps), 64 hidden
    "channel_full": (small_channel, 11, 64, 0.2),
    # the same mesh, position-only network, 24 hidden (a partial n-tile)
    "channel_position": (small_channel, 3, 24, 0.5),
    # 1-D slab: unbounded y and z, steady state: 5 inputs, 16 hidden
    "slab": (W.c2_two_region, 5, 16, 0.5),
}


@pytest.mark.parametrize("case", sorted(WINDOW_CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_local"])
def test_window_lower_bounds_match_oracle(mcdc, case, prec):
    """The lower bound each window check applies, through the kernels' own
    evaluation, state by state: FP64 equals the oracle's FP64 network; the
    FP32 modes (tensor cores, 32 states per warp, binary16 operands, FP32
    sums, SiLU through tanh.approx) stay within the first-order bound of that
    arithmetic around the oracle's exact network.  1001 states (31 full warps
    and a ragged one), a single state and none."""
    make, n_in, H, sd = WINDOW_CASES[case]
    prob = make()
    p = _params(n_in, H, seed=n_in * 7 + H, sd=sd)
    # top far above the outputs and floor far below: log w_L follows y exactly
    c = _consts(H, shift=0.0, scale=1.0, top=30.0, floor=-60.0, wl0=2.0)
    pr = {"fp32": mcdc.PREC_FP32, "fp32_local": mcdc.PREC_FP32_LOCAL,
          "fp64": mcdc.PREC_FP64}[prec]
    x, t, g = _states(prob, 1001, seed=H)
    ly, bound = _oracle_lower(prob, p, n_in, H, c, x, t, g)
    with mcdc.Problem(prob, precision=pr, tally_mode=mcdc.TALLY_GLOBAL) as P:
        P.set_network_windows(p, H, c["shift"], c["scale"], c["top"], c["floor"], c["wl0"],
                              n_in=n_in)
        wl = P.network_window_lower(x, t, g)
        one = P.network_window_lower(x[:1], t[:1], g[:1])
        none = P.network_window_lower(x[:0], t[:0], g[:0])
        bad = P.network_window_lower(x[:2], t[:2], np.array([0, prob.sigma_t.shape[1]]))
    assert np.all(wl > 0) and none.size == 0
    assert one[0] == wl[0]
    assert np.isfinite(bad[0]) and np.isnan(bad[1])
    lw = np.log(wl)
    if prec == "fp64":
        np.testing.assert_allclose(lw, ly, rtol=0, atol=1e-12)
        return
    # + the FP32 window map (fast exponential): 1e-6 in log w_L
    tol = bound + 1e-6
    err = np.abs(lw - ly)
    print(prec, case, "max error / bound", np.max(err / tol), "median", np.median(err / tol))
    assert np.all(err <= tol), np.max(err / tol)
    # a wrong row (the neighbouring state's value) would not pass
    assert np.mean(np.abs(ly - np.roll(ly, 1)) > tol) > 0.8
