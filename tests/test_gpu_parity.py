"""GPU parity against the FP64 CPU oracle, through the C-ABI.

FP64 mode: every history's primary particle ends the same way, in the same
group, after the same number of flights, collisions, crossings and random
draws, at the same place and time (relative 1e-12); every tally bin's batch
sums agree to relative 1e-9.  FP32-split mode: bins agree statistically with
an independent oracle run (|z| < 4 on coarsened bins), the paired bias
against the FP64 twin is bounded, and particle balance is exact.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W
from parity_util import (COUNT_KEYS, REL_TALLY, compare_counts, compare_records, compare_tallies,
                         fp32_bins_agree, small_channel)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


@pytest.mark.parametrize("mode", ["shared", "global"])
def test_fp64_c1_slab_full_size(mcdc, mode):
    prob = W.c1_slab()
    N, B = 100_000, 32
    tm = mcdc.TALLY_SHARED if mode == "shared" else mcdc.TALLY_GLOBAL
    g = mcdc.run_numpy(prob, N, seed=1, batches=B, records=N, precision=mcdc.PREC_FP64,
                       tally_mode=tm)
    o = O.run(prob, N, seed=1, batches=B)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(prob, 1, np.arange(N)), dim=1)


@pytest.mark.parametrize("mode", ["shared", "global"])
def test_fp64_c2_two_region_ragged(mcdc, mode):
    prob = W.c2_two_region()
    N, B = 100_003, 10
    tm = mcdc.TALLY_SHARED if mode == "shared" else mcdc.TALLY_GLOBAL
    g = mcdc.run_numpy(prob, N, seed=7, offset=12345, batches=B, records=N,
                       precision=mcdc.PREC_FP64, tally_mode=tm, block_size=128,
                       bank_per_cta=160)
    o = O.run(prob, N, seed=7, offset=12345, batches=B)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(prob, 7, 12345 + np.arange(N)), dim=1)


@pytest.mark.parametrize("mode", ["shared", "global"])
def test_fp64_3d_channel_small(mcdc, mode):
    # the shared tally must fit one CTA's shared memory: 6^3 x 7 x 4 bins in FP64
    prob = small_channel() if mode == "global" else small_channel(n=6, T=4)
    N, B = 20_000, 8
    tm = mcdc.TALLY_SHARED if mode == "shared" else mcdc.TALLY_GLOBAL
    g = mcdc.run_numpy(prob, N, seed=3, batches=B, records=N, precision=mcdc.PREC_FP64,
                       tally_mode=tm)
    o = O.run(prob, N, seed=3, batches=B)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(prob, 3, np.arange(N)), dim=3)
    assert g["scalar"][0] == pytest.approx(o["scalar"][0], rel=REL_TALLY)


def test_fp64_batched_graph_replay_takes_each_calls_seed(mcdc):
    """The batched layer captures a run once per shape and replays it: two
    calls with different seeds each equal the oracle at their own seed
    (1e-9), and after one problem is destroyed and a different one of the
    same size takes its place, the next call equals the new problem's oracle
    run (the destroyed problem's plan is dropped, not replayed)."""
    probs, _ = W.c5_batch(n_problems=3, seed=23)
    small = []
    for p in probs:
        k = min(p.n[0], 10)
        small.append(W.box(p.name, (k, k, k), p.width, p.material[:k, :k, :k].copy(), p.sigma_t,
                           p.sigma_s / p.sigma_t, p.transfer, p.speed, (0.0,) * 3, (float(k),) * 3,
                           None, (0, 0, 0), (k, k, k)))
    hist, B = [3000, 2500, 2048], 4
    handles = [mcdc.Problem(p, precision=mcdc.PREC_FP64) for p in small]
    means = [np.zeros(h.n_bins) for h in handles]

    def check(seed, problems):
        stats, scal = mcdc.run_batched(handles, hist, seed, batches=B, means=means)
        assert stats["histories"] == sum(hist)
        for i, p in enumerate(problems):
            s = (seed + i * 0x9E3779B97F4A7C15) % (1 << 64)
            o = O.run(p, hist[i], seed=s, batches=B)
            got = means[i].reshape(p.tally_shape)
            nz = o["mean"] != 0
            np.testing.assert_allclose(got[nz], o["mean"][nz], rtol=REL_TALLY)
            np.testing.assert_array_equal(got == 0, o["mean"] == 0)

    try:
        check(101, small)
        check(202, small)                  # replay with another seed
        # a different problem of the same size in slot 1
        mat = small[1].material.copy()
        mat = mat[::-1].copy()
        other = W.box("other", small[1].n, small[1].width, mat, small[1].sigma_t,
                      small[1].sigma_s / small[1].sigma_t, small[1].transfer, small[1].speed,
                      (0.0,) * 3, tuple(float(v) for v in small[1].n), None, (0, 0, 0),
                      tuple(small[1].n))
        handles[1].close()
        handles[1] = mcdc.Problem(other, precision=mcdc.PREC_FP64)
        check(303, [small[0], other, small[2]])
    finally:
        for h in handles:
            h.close()


@pytest.mark.parametrize("cap", [-1, 4096])
def test_fp64_global_tally_one_launch_per_batch(mcdc, cap):
    """The global tally's per-batch path (a launch and a fold per batch),
    taken when the per-batch slices exceed their memory cap or cannot be
    allocated: forced here by a cap of 'never' and one of 4 KiB, it matches
    the oracle to 1e-9 (region scalar over the partial box of the far
    octant included), and a second run on the same problem gives the same
    sums."""
    prob = small_channel(n=10, T=6)
    N, B = 12_000, 6
    o = O.run(prob, N, seed=5, batches=B)
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, tally_mode=mcdc.TALLY_GLOBAL,
                      slice_bytes_max=cap) as P:
        for _ in range(2):
            s1, s2, mean, rel = (np.zeros(P.n_bins) for _ in range(4))
            stats, scal = P.run_ex(N, 5, batches=B, sum1=s1, sum2=s2, mean=mean, relerr=rel)
            g = {"sum1": s1.reshape(prob.tally_shape), "sum2": s2.reshape(prob.tally_shape),
                 "mean": mean.reshape(prob.tally_shape), "relerr": rel.reshape(prob.tally_shape)}
            compare_tallies(g, o)
            compare_counts(stats, o["counts"])
            assert scal[0] == pytest.approx(o["scalar"][0], rel=REL_TALLY)
            assert scal[1] == pytest.approx(o["scalar"][1], rel=1e-6)


def test_fp64_weight_windows_infinite_medium(mcdc):
    mat = np.zeros((2, 2, 4), np.uint8)
    prob = W.box("inf_ww", (4, 2, 2), (0.5, 1.0, 1.0), mat, [[1.0]], [[0.8]], np.ones((1, 1, 1)),
                 [1.0], (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), None, (0, 0, 0), (4, 2, 2),
                 bc=(W.BC_REFLECT,) * 6)
    lower = np.random.default_rng(7).uniform(0.05, 0.6, size=prob.n_bins)
    N, B = 20_000, 10
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, overflow_per_cta=8192) as P:
        P.set_weight_windows(lower, 5.0, 2.5, 16)
        s1, s2, mean, rel = (np.zeros(P.n_bins) for _ in range(4))
        stats, scal = P.run_ex(N, 13, batches=B, sum1=s1, sum2=s2, mean=mean, relerr=rel)
    o = O.run(prob, N, seed=13, batches=B,
              ww={"lower": lower, "upper_ratio": 5.0, "survival_ratio": 2.5, "nmax": 16})
    g = {"sum1": s1.reshape(prob.tally_shape), "sum2": s2.reshape(prob.tally_shape),
         "mean": mean.reshape(prob.tally_shape), "relerr": rel.reshape(prob.tally_shape)}
    compare_tallies(g, o)
    compare_counts(stats, o["counts"])
    assert stats["splits"] > 100 and stats["roulette_killed"] > 100


def test_fp64_weight_windows_global_tally_with_spill(mcdc):
    """Global tally, 64-slot warp stacks and strong splitting: children spill
    to the device-wide banks and run in later passes on other warps; each
    keeps its own random stream, so the tallies still match the oracle."""
    mat = np.zeros((2, 2, 4), np.uint8)
    prob = W.box("inf_ww", (4, 2, 2), (0.5, 1.0, 1.0), mat, [[1.0]], [[0.9]], np.ones((1, 1, 1)),
                 [1.0], (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), None, (0, 0, 0), (4, 2, 2),
                 bc=(W.BC_REFLECT,) * 6)
    lower = np.random.default_rng(9).uniform(0.002, 0.05, size=prob.n_bins)
    N, B = 4000, 4
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, tally_mode=mcdc.TALLY_GLOBAL,
                      overflow_per_cta=512) as P:
        P.set_weight_windows(lower, 5.0, 2.5, 16)
        s1, s2, mean, rel = (np.zeros(P.n_bins) for _ in range(4))
        stats, scal = P.run_ex(N, 21, batches=B, sum1=s1, sum2=s2, mean=mean, relerr=rel)
    o = O.run(prob, N, seed=21, batches=B,
              ww={"lower": lower, "upper_ratio": 5.0, "survival_ratio": 2.5, "nmax": 16})
    g = {"sum1": s1.reshape(prob.tally_shape), "sum2": s2.reshape(prob.tally_shape),
         "mean": mean.reshape(prob.tally_shape), "relerr": rel.reshape(prob.tally_shape)}
    compare_tallies(g, o)
    compare_counts(stats, o["counts"])
    assert stats["children"] > 64 * 8 * 148 * 2, stats["children"]   # more than the warp stacks hold


def test_fp64_batched_problems_match_independent_oracle_runs(mcdc):
    """Five random 3-D problems of different size and group count in one
    batched run: each problem's tally equals an oracle run of that problem
    with its own seed, to 1e-9."""
    probs, _ = W.c5_batch(n_problems=5, seed=17)
    small = []
    for i, p in enumerate(probs):        # keep the oracle fast: at most 12^3 cells
        k = min(p.n[0], 12)
        # two problems score a partial region box (the fold's cell test),
        # the others the whole mesh
        lo = {1: (k // 2, 0, 0), 3: (1, k // 3, k // 2)}.get(i, (0, 0, 0))
        hi = {3: (k - 1, k, k - 2)}.get(i, (k, k, k))
        small.append(W.box(p.name, (k, k, k), p.width, p.material[:k, :k, :k].copy(), p.sigma_t,
                           p.sigma_s / p.sigma_t, p.transfer, p.speed, (0.0,) * 3, (float(k),) * 3,
                           None, lo, hi))
    hist = [3000, 5000, 2048, 4001, 2500]
    seed, B = 99, 4
    handles = [mcdc.Problem(p, precision=mcdc.PREC_FP64) for p in small]
    means = [np.zeros(h.n_bins) for h in handles]
    rels = [np.zeros(h.n_bins) for h in handles]
    stats, scal = mcdc.run_batched(handles, hist, seed, batches=B, means=means, relerrs=rels)
    assert stats["histories"] == sum(hist)
    for i, p in enumerate(small):
        s = (seed + i * 0x9E3779B97F4A7C15) % (1 << 64)
        o = O.run(p, hist[i], seed=s, batches=B)
        nz = o["mean"] != 0
        got = means[i].reshape(p.tally_shape)
        np.testing.assert_allclose(got[nz], o["mean"][nz], rtol=REL_TALLY)
        np.testing.assert_array_equal(got == 0, o["mean"] == 0)
        np.testing.assert_allclose(rels[i].reshape(p.tally_shape), o["relerr"], rtol=1e-6, atol=1e-12)
        assert scal[i][0] == pytest.approx(o["scalar"][0], rel=REL_TALLY)
    for h in handles:
        h.close()


def _coarse(mean):
    """20 x 10 blocks of (space, time) bins of the two-region slab."""
    return mean[0, 0, :, 0, :].reshape(20, 10, 10, 5).sum(axis=(1, 3))


@pytest.mark.parametrize("prec", ["fp32", "fp32_local"])
def test_fp32_c2_statistical_and_paired_bias(mcdc, prec):
    P32 = mcdc.PREC_FP32 if prec == "fp32" else mcdc.PREC_FP32_LOCAL
    prob = W.c2_two_region()
    # (1) every bin against an independent oracle run: per-bin batch errors
    # are valid, so |z| > 4 may only occur about as often as chance allows
    N = 2_000_000
    g32 = mcdc.run_numpy(prob, N, seed=2, batches=40, precision=P32)
    o = O.run(prob, 1_000_000, seed=1, batches=40)
    c = g32["counts"]
    assert c["absorbed"] + c["leaked"] + c["censused"] == N
    n4, nbins, _ = fp32_bins_agree(g32, o, batches=40)
    print("per-bin |z| > 4:", n4, "of", nbins, "well-estimated bins")
    # (2) coarse bins: neighbouring bins share histories, so the error of a
    # block comes from 32 independent replicas of each precision (the FP64
    # path reproduces the oracle event for event, tested above)
    R, n = 32, 300_000
    reps = {}
    for pr in (P32, mcdc.PREC_FP64):
        with mcdc.Problem(prob, precision=pr) as P:
            rows = []
            for r in range(R):
                m = np.zeros(P.n_bins)
                P.run_ex(n, 5, offset=(r + 1) * 10_000_000 + (pr * 1000_000_000), batches=8,
                         mean=m, want_stats=False)
                rows.append(_coarse(m.reshape(prob.tally_shape)))
        reps[pr] = np.array(rows)
    a, b = reps[P32], reps[mcdc.PREC_FP64]
    se = np.sqrt(a.var(axis=0, ddof=1) / R + b.var(axis=0, ddof=1) / R)
    ok = se > 0
    z = (a.mean(axis=0) - b.mean(axis=0))[ok] / se[ok]
    print("coarse |z| max", float(np.abs(z).max()), "mean z", float(z.mean()))
    assert np.all(np.abs(z) < 5.0), np.abs(z).max()
    # (3) paired with its FP64 twin (same seed; sampling the distance to
    # collision every flight, so the same random numbers): the precision
    # bias of the region total stays far below the noise
    g32 = mcdc.run_numpy(prob, N, seed=2, batches=40, precision=P32, flight_sampling=1)
    g64 = mcdc.run_numpy(prob, N, seed=2, batches=40, precision=mcdc.PREC_FP64)
    bias = g32["scalar"][0] / g64["scalar"][0] - 1.0
    cb = _coarse(g32["mean"]) / np.maximum(_coarse(g64["mean"]), 1e-300) - 1.0
    print("paired FP32-FP64 bias of the total", bias, "noise", g64["scalar"][1],
          "coarse max |bias|", float(np.abs(cb[_coarse(g64["mean"]) > 0]).max()))
    assert abs(bias) < 0.2 * g64["scalar"][1], (bias, g64["scalar"][1])


@pytest.mark.parametrize("prec", ["fp32", "fp32_local"])
def test_fp32_modes_3d_channel(mcdc, prec):
    """3-D geometry of the FP32 modes: exact balance, the region total of a
    paired FP64 run (same random streams: distance sampled every flight)
    within a small fraction of the statistical error, and the default mode
    (optical depth carried) against an independent FP64 run."""
    P32 = mcdc.PREC_FP32 if prec == "fp32" else mcdc.PREC_FP32_LOCAL
    prob = small_channel()
    N = 400_000
    whole = ((0, 0, 0), prob.n)
    e = mcdc.run_numpy(prob, 4 * N, seed=9, batches=20, precision=P32, region=whole)
    d = mcdc.run_numpy(prob, N, seed=4, batches=20, precision=mcdc.PREC_FP64, region=whole)
    (me, re_), (md, rd) = e["scalar"], d["scalar"]
    assert abs(me - md) < 4.0 * np.hypot(me * re_, md * rd), (me, md)
    g = mcdc.run_numpy(prob, N, seed=4, batches=20, precision=P32, region=whole,
                       flight_sampling=1)
    c = g["counts"]
    assert c["absorbed"] + c["leaked"] + c["censused"] == N
    tot32, tot64 = g["sum1"].sum(), d["sum1"].sum()
    # total track length: relative error of the total is well below 1e-2 here
    assert abs(tot32 / tot64 - 1.0) < 2e-3, (tot32, tot64)
    bias = g["scalar"][0] / d["scalar"][0] - 1.0
    assert abs(bias) < 0.3 * d["scalar"][1], (bias, d["scalar"][1])


@pytest.mark.parametrize("prec", ["fp32", "fp32_local"])
def test_fp32_modes_reflecting_infinite_medium(mcdc, prec):
    """All faces reflecting, uniform source: every cell's flux is
    1 / (Sigma_a V_box) (the closed form the oracle is pinned to)."""
    P32 = mcdc.PREC_FP32 if prec == "fp32" else mcdc.PREC_FP32_LOCAL
    mat = np.zeros((3, 2, 4), np.uint8)
    n, w = (4, 2, 3), (0.5, 1.0, 0.7)
    ext = tuple(k * d for k, d in zip(n, w))
    prob = W.box("inf", n, w, mat, [[1.0]], [[0.8]], np.ones((1, 1, 1)),
                 [1.0], (0.0, 0.0, 0.0), ext, None, (0, 0, 0), n, bc=(W.BC_REFLECT,) * 6)
    N = 400_000
    g = mcdc.run_numpy(prob, N, seed=6, batches=40, precision=P32)
    ref = 1.0 / (0.2 * ext[0] * ext[1] * ext[2])
    m = g["mean"].reshape(-1)
    z = (m - ref) / (m * g["relerr"].reshape(-1))
    assert np.all(np.abs(z) < 4.5), z
    assert g["counts"]["absorbed"] == N


def test_edge_cases(mcdc):
    prob = W.c1_slab()
    # the smallest run: two histories, two batches
    g = mcdc.run_numpy(prob, 2, seed=5, batches=2, records=2, precision=mcdc.PREC_FP64)
    o = O.run(prob, 2, seed=5, batches=2)
    compare_tallies(g, o)
    compare_records(g["records"], O.trace(prob, 5, np.arange(2)), dim=1)
    # invalid run arguments are rejected
    with mcdc.Problem(prob) as P:
        with pytest.raises(mcdc.MCDCError):
            P.run_ex(0, 1)
        with pytest.raises(mcdc.MCDCError):
            P.run_ex(10, 1, batches=11)
        with pytest.raises(mcdc.MCDCError):
            P.run_ex(10, 1, batches=1)


def test_born_after_last_census(mcdc):
    prob = W.c2_two_region()
    import dataclasses
    late = dataclasses.replace(prob, src_t0=0.0, src_t1=40.0)   # half are born after t = 20
    N = 20_000
    g = mcdc.run_numpy(late, N, seed=9, batches=4, records=N, precision=mcdc.PREC_FP64)
    o = O.run(late, N, seed=9, batches=4)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(late, 9, np.arange(N)), dim=1)


def test_history_partition_invariance(mcdc):
    prob = W.c2_two_region()
    a = mcdc.run_numpy(prob, 40_000, seed=8, batches=4, precision=mcdc.PREC_FP64)
    b1 = mcdc.run_numpy(prob, 20_000, seed=8, offset=0, batches=2, precision=mcdc.PREC_FP64)
    b2 = mcdc.run_numpy(prob, 20_000, seed=8, offset=20_000, batches=2, precision=mcdc.PREC_FP64)
    np.testing.assert_allclose(a["sum1"], b1["sum1"] + b2["sum1"], rtol=1e-11, atol=1e-300)


def test_fp_full_size_c2_sampled_histories(mcdc):
    """The full 1e7-history two-region workload: FP32-split balance is exact,
    and in FP64 mode 2000 sampled histories match the oracle event for
    event."""
    prob = W.c2_two_region()
    N = 10_000_000
    g = mcdc.run_numpy(prob, N, seed=1, precision=mcdc.PREC_FP32)
    c = g["counts"]
    assert c["histories"] == N
    assert c["absorbed"] + c["leaked"] + c["censused"] == N
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64) as P:
        rec = np.zeros(N, dtype=mcdc.RECORD_DTYPE)
        stats, _ = P.run_ex(N, 1, records=rec)
    pick = np.sort(np.random.default_rng(0).choice(N, 2000, replace=False))
    compare_records(rec[pick], O.trace(prob, 1, pick), dim=1)
    assert stats["absorbed"] + stats["leaked"] + stats["censused"] == N


@pytest.mark.parametrize("prec", ["fp32", "fp32_local", "fp64"])
@pytest.mark.parametrize("sampling", [0, 1])
def test_uncollided_beam_through_void_gap_and_census(mcdc, prec, sampling):
    """Pure absorbers (sigma_t 0.8, then void, then 0.4) under a normal beam
    with census edges every 0.5 time units (speed 1): the track-length flux
    of every cell, summed over time bins, is the uncollided closed form
    int exp(-tau(x)) dx / width.  Pins the optical depth the FP32 modes carry
    across surfaces (including a change of sigma_t and a void, where it must
    not change) and census events."""
    P = {"fp32": mcdc.PREC_FP32, "fp32_local": mcdc.PREC_FP32_LOCAL,
         "fp64": mcdc.PREC_FP64}[prec]
    nc, L = 60, 12.0
    w = L / nc
    mats = np.array([0] * 15 + [1] * 15 + [2] * 30)
    prob = W.slab("void_gap_beam", L, nc, mats, [[0.8], [0.0], [0.4]], [[0.0], [0.0], [0.0]],
                  src=(0.0, 0.0), kind=W.SRC_BEAM, direction=(1.0, 0.0, 0.0),
                  edges=np.linspace(0.0, 13.0, 27))
    N = 2_000_000
    g = mcdc.run_numpy(prob, N, seed=3, batches=40, precision=P, flight_sampling=sampling)
    c = g["counts"]
    assert c["absorbed"] + c["leaked"] == N and c["census"] > 2 * N
    a = np.arange(nc) * w
    b = a + w
    ref = np.empty(nc)
    r1 = b <= 3.0 + 1e-12
    ref[r1] = (np.exp(-0.8 * a[r1]) - np.exp(-0.8 * b[r1])) / 0.8
    rv = (a >= 3.0 - 1e-12) & (b <= 6.0 + 1e-12)
    ref[rv] = np.exp(-2.4) * w
    r3 = a >= 6.0 - 1e-12
    ref[r3] = np.exp(-2.4) * (np.exp(-0.4 * (a[r3] - 6.0)) - np.exp(-0.4 * (b[r3] - 6.0))) / 0.4
    ref /= w
    s1 = g["sum1"].reshape(nc, -1).sum(axis=1) / (N * w)
    # error of the time-summed cell flux from the batch sums of its bins is
    # not available; bound it by the sum of the per-bin standard errors
    se = np.sqrt(((g["mean"] * g["relerr"]).reshape(nc, -1) ** 2).sum(axis=1)) * np.sqrt(2.0)
    z = (s1 - ref) / np.maximum(se, 1e-30)
    assert np.all(np.abs(z) < 4.5), (np.abs(z).max(), int(np.abs(z).argmax()))
    # the void cells: every history that reaches the gap crosses it whole
    np.testing.assert_allclose(s1[rv], np.exp(-2.4), rtol=6 * np.sqrt((1 - np.exp(-2.4)) / (np.exp(-2.4) * N)))


def _ww_boxes():
    """Three small 3-D problems of different sizes and materials, all faces
    reflecting (every history ends by absorption), each with its own table of
    lower bounds drawn so that both splits and roulettes happen."""
    out = []
    for k, (n, c, seed) in enumerate((((4, 2, 2), 0.8, 7), ((3, 3, 2), 0.7, 8), ((5, 2, 3), 0.85, 9))):
        mat = np.zeros((n[2], n[1], n[0]), np.uint8)
        w = (0.5, 1.0, 0.7)
        ext = tuple(a * b for a, b in zip(n, w))
        prob = W.box(f"ww_box{k}", n, w, mat, [[1.0]], [[c]], np.ones((1, 1, 1)), [1.0],
                     (0.0, 0.0, 0.0), ext, None, (0, 0, 0), n, bc=(W.BC_REFLECT,) * 6)
        lower = np.random.default_rng(seed).uniform(0.05, 0.6, size=prob.n_bins)
        out.append((prob, lower))
    return out


def test_fp64_batched_weight_windows_match_oracle(mcdc):
    """Table windows in a batched run: every problem splits and roulettes with
    its own table in the shared launch, its children staying in the warp that
    serves its work item, and equals the oracle at its own seed (1e-9, event
    counts summed over the problems exactly).  Turning the windows off makes
    the next call analog (the cached plan holds the problems' tables, so it
    must not be replayed)."""
    boxes = _ww_boxes()
    hist, seed, B = [6000, 5000, 4000], 31, 4
    handles = [mcdc.Problem(p, precision=mcdc.PREC_FP64) for p, _ in boxes]
    try:
        for h, (p, lower) in zip(handles, boxes):
            h.set_weight_windows(lower, 5.0, 2.5, 16)
        means = [np.zeros(h.n_bins) for h in handles]
        for windows in (True, False):
            stats, scal = mcdc.run_batched(handles, hist, seed, batches=B, means=means)
            tot = {k: 0 for k in COUNT_KEYS}
            for i, (p, lower) in enumerate(boxes):
                s = (seed + i * 0x9E3779B97F4A7C15) % (1 << 64)
                ww = ({"lower": lower, "upper_ratio": 5.0, "survival_ratio": 2.5, "nmax": 16}
                      if windows else None)
                o = O.run(p, hist[i], seed=s, batches=B, ww=ww)
                for k in COUNT_KEYS:
                    tot[k] += o["counts"][k]
                got = means[i].reshape(p.tally_shape)
                nz = o["mean"] != 0
                np.testing.assert_allclose(got[nz], o["mean"][nz], rtol=REL_TALLY)
                np.testing.assert_array_equal(got == 0, o["mean"] == 0)
            compare_counts(stats, tot)
            if windows:
                assert stats["splits"] > 100 and stats["roulette_killed"] > 100, stats
                assert stats["splits_dropped"] == 0
                for h in handles:
                    h.set_weight_windows(None, 0.0, 0.0, 0)
            else:
                assert stats["splits"] == 0 and stats["roulette_killed"] == 0
    finally:
        for h in handles:
            h.close()
