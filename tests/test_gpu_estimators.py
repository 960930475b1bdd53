"""GPU parity of the collision estimator and of implicit capture against the
FP64 CPU oracle, through the C-ABI.

FP64 mode: the same histories event for event (end, group, counter, flights,
collisions, crossings, position, time and weight of every primary), tallies
to relative 1e-9, exact event counts and weight sums to relative 1e-9, in the
shared and the global tally modes, in 1-D and 3-D, alone and with weight
windows.  FP32 modes: the region total against an independent oracle run
(|z| < 4) and exact history balance.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W
from parity_util import (REL_TALLY, compare_counts, compare_records, compare_tallies,
                         fp32_bins_agree, small_channel)

pytestmark = pytest.mark.gpu

IMPLICIT = (0.25, 0.5)
WEIGHT_KEYS = ("w_source", "w_absorbed", "w_leaked", "w_censused")


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def compare_weights(g, o):
    for k in WEIGHT_KEYS:
        assert g[k] == pytest.approx(o[k], rel=REL_TALLY, abs=1e-12), (k, g[k], o[k])


@pytest.mark.parametrize("mode", ["shared", "global"])
def test_fp64_collision_estimator_c2(mcdc, mode):
    prob = W.c2_two_region()
    N, B = 50_003, 10
    tm = mcdc.TALLY_SHARED if mode == "shared" else mcdc.TALLY_GLOBAL
    g = mcdc.run_numpy(prob, N, seed=7, offset=99, batches=B, records=N,
                       precision=mcdc.PREC_FP64, tally_mode=tm, estimator=mcdc.EST_COLLISION)
    o = O.run(prob, N, seed=7, offset=99, batches=B, estimator=O.EST_COLLISION)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(prob, 7, 99 + np.arange(N)), dim=1)
    assert g["scalar"][0] == pytest.approx(o["scalar"][0], rel=REL_TALLY)


@pytest.mark.parametrize("mode", ["shared", "global"])
def test_fp64_implicit_capture_c2(mcdc, mode):
    prob = W.c2_two_region()
    N, B = 50_003, 10
    tm = mcdc.TALLY_SHARED if mode == "shared" else mcdc.TALLY_GLOBAL
    g = mcdc.run_numpy(prob, N, seed=11, batches=B, records=N, precision=mcdc.PREC_FP64,
                       tally_mode=tm, implicit=IMPLICIT)
    o = O.run(prob, N, seed=11, batches=B, implicit=IMPLICIT)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_weights(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(prob, 11, np.arange(N), implicit=IMPLICIT), dim=1)
    c = g["counts"]
    assert c["roulette_killed"] > 1000 and c["roulette_survived"] > 1000


def test_fp64_both_options_3d_channel(mcdc):
    prob = small_channel()
    N, B = 20_000, 8
    g = mcdc.run_numpy(prob, N, seed=3, batches=B, records=N, precision=mcdc.PREC_FP64,
                       tally_mode=mcdc.TALLY_GLOBAL, estimator=mcdc.EST_COLLISION,
                       implicit=(0.1, 0.3))
    o = O.run(prob, N, seed=3, batches=B, estimator=O.EST_COLLISION, implicit=(0.1, 0.3))
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_weights(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(prob, 3, np.arange(N), implicit=(0.1, 0.3)), dim=3)


def test_fp64_implicit_capture_with_weight_windows(mcdc):
    mat = np.zeros((2, 2, 4), np.uint8)
    prob = W.box("inf_ww", (4, 2, 2), (0.5, 1.0, 1.0), mat, [[1.0]], [[0.8]], np.ones((1, 1, 1)),
                 [1.0], (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), None, (0, 0, 0), (4, 2, 2),
                 bc=(W.BC_REFLECT,) * 6)
    lower = np.random.default_rng(7).uniform(0.05, 0.6, size=prob.n_bins)
    N, B = 20_000, 10
    ww = {"lower": lower, "upper_ratio": 5.0, "survival_ratio": 2.5, "nmax": 16}
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, overflow_per_cta=8192,
                      estimator=mcdc.EST_COLLISION, implicit=(0.02, 0.04)) as P:
        P.set_weight_windows(lower, 5.0, 2.5, 16)
        s1, s2, mean, rel = (np.zeros(P.n_bins) for _ in range(4))
        stats, _ = P.run_ex(N, 13, batches=B, sum1=s1, sum2=s2, mean=mean, relerr=rel)
    o = O.run(prob, N, seed=13, batches=B, ww=ww, estimator=O.EST_COLLISION,
              implicit=(0.02, 0.04))
    shp = prob.tally_shape
    g = {"sum1": s1.reshape(shp), "sum2": s2.reshape(shp), "mean": mean.reshape(shp),
         "relerr": rel.reshape(shp)}
    compare_tallies(g, o)
    compare_counts(stats, o["counts"])
    compare_weights(stats, o["counts"])
    assert stats["splits"] > 100


@pytest.mark.parametrize("prec", ["fp32", "fp32_local"])
@pytest.mark.parametrize("opts", ["collision", "implicit"])
def test_fp32_options_statistical(mcdc, prec, opts):
    P32 = mcdc.PREC_FP32 if prec == "fp32" else mcdc.PREC_FP32_LOCAL
    prob = W.c2_two_region()
    kw_g = {"estimator": mcdc.EST_COLLISION} if opts == "collision" else {"implicit": IMPLICIT}
    kw_o = {"estimator": O.EST_COLLISION} if opts == "collision" else {"implicit": IMPLICIT}
    N = 2_000_000
    g = mcdc.run_numpy(prob, N, seed=2, batches=40, precision=P32, **kw_g)
    o = O.run(prob, 400_000, seed=1, batches=40, **kw_o)
    c = g["counts"]
    assert c["absorbed"] + c["leaked"] + c["censused"] + c["roulette_killed"] == N
    (mg, rg), (mo, ro) = g["scalar"], o["scalar"]
    z = (mg - mo) / np.hypot(mg * rg, mo * ro)
    assert abs(z) < 4.0, (mg, mo, z)
    # every well-estimated bin: |z| > 4 only about as often as chance allows
    fp32_bins_agree(g, o, batches=40)


def test_batched_runs_take_the_collision_estimator_and_refuse_implicit_capture(mcdc):
    probs = [W.c1_slab(), W.c2_two_region()]
    handles = [mcdc.Problem(p, precision=mcdc.PREC_FP64, estimator=mcdc.EST_COLLISION)
               for p in probs]
    hist, seed, B = [30_000, 20_000], 5, 8
    means = [np.zeros(h.n_bins) for h in handles]
    stats, scal = mcdc.run_batched(handles, hist, seed, batches=B, means=means)
    for i, p in enumerate(probs):
        s = (seed + i * 0x9E3779B97F4A7C15) % (1 << 64)      # problem i's own seed
        o = O.run(p, hist[i], seed=s, batches=B, estimator=O.EST_COLLISION)
        nz = o["mean"] != 0
        got = means[i].reshape(p.tally_shape)
        np.testing.assert_allclose(got[nz], o["mean"][nz], rtol=REL_TALLY)
        np.testing.assert_array_equal(got == 0, o["mean"] == 0)
    for h in handles:
        h.close()
    with mcdc.Problem(W.c1_slab(), precision=mcdc.PREC_FP64, implicit=IMPLICIT) as h:
        with pytest.raises(mcdc.MCDCError):
            mcdc.run_batched([h], [1000], seed, batches=4, means=[np.zeros(h.n_bins)])
