"""GPU parity of the combined track-length/collision estimator against the FP64
CPU oracle, through the C-ABI.

FP64 mode: both halves of the tally, squared sums and the summed products to
relative 1e-9, exact event counts, the per-estimator means and errors to
relative 1e-9 (against the oracle's track-length-only and collision-only runs
of the same histories), and the combined mean, error and coefficient within
the rounding of the sums amplified by the conditioning of the coefficient;
in the shared and global tally modes, in 3-D and 1-D, with weight windows,
implicit capture and population control.  FP32 split: the combined region
scalar against an oracle run (|z| < 4).  Refusals: batched and
allocation-free runs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W
from parity_util import REL_TALLY, compare_counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def td_box():
    mat = np.zeros((3, 4, 5), np.uint8)
    mat[:, 1:3, 2:4] = 1
    st = [[1.0, 1.5], [0.4, 2.5]]
    c = [[0.6, 0.5], [0.9, 0.3]]
    P = np.array([[[0.3, 0.7], [0.1, 0.9]], [[0.5, 0.5], [0.2, 0.8]]])
    return W.box("combined_box", (5, 4, 3), (1.0, 1.0, 1.0), mat, st, c, P, [2.0, 0.5],
                 (1.0, 1.0, 0.5), (3.0, 3.0, 2.5), np.linspace(0.0, 4.0, 5), (2, 1, 0), (5, 3, 3),
                 src_pdf=[0.7, 0.3])


# Scores are positive, so a bin's batch sum over n scores, added in any order,
# is within n x 2^-53 of the exact sum relative; n stays below 1e4 here.
DELTA = 1e-11


def _close(a, b, rtol):
    return np.abs(a - b) <= rtol * np.maximum(np.abs(b), 1e-300) + 1e-300


def _sensitivity(o, N, B, vol, h=1e-7):
    """Per bin, the first-order change of the oracle's combined mean, relative
    error and coefficient when each of its five sums moves by a relative h,
    summed over the five (finite differences through the oracle)."""
    nb = o["sum12"].size
    sums = [o["sum1"][0].ravel(), o["sum2"][0].ravel(), o["sum1"][1].ravel(),
            o["sum2"][1].ravel(), o["sum12"].ravel()]
    a0 = np.zeros(nb)
    m0, r0 = O.combine(*sums, N, B, vol, alpha=a0)
    sm, sr, sa = np.zeros(nb), np.zeros(nb), np.zeros(nb)
    for i in range(5):
        q = list(sums)
        q[i] = q[i] * (1.0 + h)
        ai = np.zeros(nb)
        mi, ri = O.combine(*q, N, B, vol, alpha=ai)
        sm += np.abs(mi - m0) / h
        sr += np.abs(ri - r0) / h
        sa += np.abs(ai - a0) / h
    shp = o["mean"].shape
    return sm.reshape(shp), sr.reshape(shp), sa.reshape(shp)


def check_combined(g, o, tl, ce, N, B, vol=1.0):
    for key in ("sum1", "sum2", "sum12"):
        assert np.all(_close(g[key], o[key], DELTA)), key
    compare_counts(g["counts"], o["counts"])
    # per-estimator moments: the single-estimator runs of the same histories
    parts = g["parts"]
    for e, ref in ((0, tl), (1, ce)):
        np.testing.assert_allclose(parts[2 * e], ref["mean"], rtol=REL_TALLY, atol=1e-300)
        np.testing.assert_allclose(parts[2 * e + 1], ref["relerr"], rtol=1e-6, atol=1e-12)
    # combined: the sums' rounding (DELTA) through the combination's sensitivity
    sm, sr, sa = _sensitivity(o, N, B, vol)
    for got, ref, sens in ((g["mean"], o["mean"], sm), (g["relerr"], o["relerr"], sr),
                           (parts[4], o["alpha"], sa)):
        tol = 10.0 * DELTA * sens + 1e-13 * np.abs(ref) + 1e-300
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5])
    # most scored bins are well conditioned (the check above is not vacuous)
    scored = o["sum1"][0] > 0
    assert (sm[scored] * DELTA < 1e-6 * np.abs(o["mean"][scored])).mean() > 0.9
    # region scalar: combined and the two parts
    (mg, rg), (mo, ro) = g["scalar"], o["scalar"]
    assert mg == pytest.approx(mo, rel=1e-7)
    assert rg == pytest.approx(ro, rel=1e-5)
    sp = g["scalar_parts"]
    assert sp[0] == pytest.approx(tl["scalar"][0], rel=REL_TALLY)
    assert sp[2] == pytest.approx(ce["scalar"][0], rel=REL_TALLY)
    assert sp[1] == pytest.approx(tl["scalar"][1], rel=1e-6)
    assert sp[3] == pytest.approx(ce["scalar"][1], rel=1e-6)
    assert sp[4] == pytest.approx(o["scalar_alpha"], rel=1e-6, abs=1e-9)
    assert rg <= min(sp[1], sp[3]) * (1 + 1e-9)


def oracle_three(prob, N, seed, B, **kw):
    o = O.run(prob, N, seed=seed, batches=B, estimator=O.EST_COMBINED, **kw)
    tl = O.run(prob, N, seed=seed, batches=B, estimator=O.EST_TRACK, **kw)
    ce = O.run(prob, N, seed=seed, batches=B, estimator=O.EST_COLLISION, **kw)
    return o, tl, ce


@pytest.mark.parametrize("mode", ["shared", "global"])
def test_fp64_combined_3d(mcdc, mode):
    prob = td_box()
    N, B = 40_001, 16
    tm = mcdc.TALLY_SHARED if mode == "shared" else mcdc.TALLY_GLOBAL
    g = mcdc.run_numpy(prob, N, seed=5, batches=B, precision=mcdc.PREC_FP64, tally_mode=tm,
                       estimator=mcdc.EST_COMBINED)
    check_combined(g, *oracle_three(prob, N, 5, B), N, B)


def test_fp64_combined_slab_global(mcdc):
    prob = W.c2_two_region()
    N, B = 30_000, 10
    g = mcdc.run_numpy(prob, N, seed=9, batches=B, precision=mcdc.PREC_FP64,
                       tally_mode=mcdc.TALLY_GLOBAL, estimator=mcdc.EST_COMBINED)
    check_combined(g, *oracle_three(prob, N, 9, B), N, B)


def test_fp64_combined_with_implicit_capture(mcdc):
    prob = td_box()
    N, B = 30_000, 12
    imp = (0.1, 0.3)
    g = mcdc.run_numpy(prob, N, seed=3, batches=B, precision=mcdc.PREC_FP64,
                       tally_mode=mcdc.TALLY_GLOBAL, estimator=mcdc.EST_COMBINED, implicit=imp)
    check_combined(g, *oracle_three(prob, N, 3, B, implicit=imp), N, B)


def test_fp64_combined_with_population_control(mcdc):
    prob = td_box()
    prob = W.box("combined_box_pc", prob.n, prob.width, prob.material, prob.sigma_t,
                 prob.sigma_s / prob.sigma_t, prob.transfer, prob.speed, prob.src_lo, prob.src_hi,
                 prob.edges, prob.region_lo, prob.region_hi, src_pdf=prob.src_pdf,
                 src_t=(0.0, 0.5))
    N, B, M = 20_000, 8, 2000
    g = mcdc.run_numpy(prob, N, seed=4, batches=B, precision=mcdc.PREC_FP64,
                       tally_mode=mcdc.TALLY_GLOBAL, estimator=mcdc.EST_COMBINED, pc_target=M)
    check_combined(g, *oracle_three(prob, N, 4, B, pc_target=M), N, B)
    assert g["counts"]["pc_combs"] > 0


def test_fp64_combined_with_weight_windows(mcdc):
    prob = td_box()
    lower = np.random.default_rng(5).uniform(0.05, 0.6, size=prob.n_bins)
    ww = {"lower": lower, "upper_ratio": 5.0, "survival_ratio": 2.5, "nmax": 16}
    N, B = 20_000, 10
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, tally_mode=mcdc.TALLY_GLOBAL,
                      estimator=mcdc.EST_COMBINED) as P:
        P.set_weight_windows(lower, 5.0, 2.5, 16)
        nb = P.n_bins
        s1, s2 = np.zeros(2 * nb), np.zeros(2 * nb)
        s12, mean, rel, parts, sp = (np.zeros(nb), np.zeros(nb), np.zeros(nb), np.zeros(5 * nb),
                                     np.zeros(5))
        stats, scal = P.run_ex(N, 6, batches=B, sum1=s1, sum2=s2, sum12=s12, mean=mean,
                               relerr=rel, parts=parts, scalar_parts=sp)
    shp = prob.tally_shape
    g = {"sum1": s1.reshape((2,) + shp), "sum2": s2.reshape((2,) + shp), "sum12": s12.reshape(shp),
         "mean": mean.reshape(shp), "relerr": rel.reshape(shp), "parts": parts.reshape((5,) + shp),
         "scalar": scal, "scalar_parts": sp, "counts": stats}
    check_combined(g, *oracle_three(prob, N, 6, B, ww=ww), N, B)
    assert stats["splits"] > 100


def test_fp32_combined_statistical(mcdc):
    prob = W.c2_two_region()
    N, B = 2_000_000, 40
    g = mcdc.run_numpy(prob, N, seed=2, batches=B, precision=mcdc.PREC_FP32,
                       estimator=mcdc.EST_COMBINED)
    o = O.run(prob, 400_000, seed=1, batches=B, estimator=O.EST_COMBINED)
    (mg, rg), (mo, ro) = g["scalar"], o["scalar"]
    z = (mg - mo) / np.hypot(mg * rg, mo * ro)
    assert abs(z) < 4.0, (mg, mo, z)
    sp = g["scalar_parts"]
    assert rg <= min(sp[1], sp[3]) * (1 + 1e-9)
    c = g["counts"]
    assert c["absorbed"] + c["leaked"] + c["censused"] == N


def test_combined_refusals(mcdc):
    import torch
    prob = td_box()
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, estimator=mcdc.EST_COMBINED) as P:
        with pytest.raises(mcdc.MCDCError):
            mcdc.run_batched([P], [1000], 1, batches=4)
        s1 = torch.zeros(2 * P.n_bins, dtype=torch.float64, device="cuda")
        s2 = torch.zeros(2 * P.n_bins, dtype=torch.float64, device="cuda")
        with pytest.raises(mcdc.MCDCError):
            P.run_noalloc(1000, 1, s1, s2, batches=4)
    with pytest.raises(mcdc.MCDCError):
        mcdc.Problem(prob, estimator=3)
