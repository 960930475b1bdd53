"""GPU parity of population control (the census-bank comb) against the FP64
CPU oracle, through the C-ABI.

FP64 mode: the same combs -- bank order by (history id, serial), teeth,
new streams -- so tallies agree to relative 1e-9 and event, end, comb and
particle counts exactly, weight sums to 1e-9; in 1-D and in 3-D together
with implicit capture and the collision estimator.  FP32 modes: the region
total and every bin against an independent oracle run.  Combinations the
comb does not support are refused.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W
from parity_util import (REL_TALLY, compare_counts, compare_tallies, fp32_bins_agree,
                         small_channel)

pytestmark = pytest.mark.gpu

PC_KEYS = ("pc_combs", "pc_in", "pc_out")
WEIGHT_KEYS = ("w_source", "w_absorbed", "w_leaked", "w_censused", "w_pc_in", "w_pc_out")


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def compare_pc(g, o):
    for k in PC_KEYS:
        assert g[k] == o[k], (k, g[k], o[k])
    for k in WEIGHT_KEYS:
        assert g[k] == pytest.approx(o[k], rel=REL_TALLY, abs=1e-12), (k, g[k], o[k])


def test_fp64_population_control_c2(mcdc):
    prob = W.c2_two_region()
    N, B, M = 40_003, 8, 3000
    g = mcdc.run_numpy(prob, N, seed=5, offset=17, batches=B, precision=mcdc.PREC_FP64,
                       pc_target=M)
    o = O.run(prob, N, seed=5, offset=17, batches=B, pc_target=M)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_pc(g["counts"], o["counts"])
    assert g["counts"]["pc_combs"] == B * 49
    assert g["scalar"][0] == pytest.approx(o["scalar"][0], rel=REL_TALLY)


def test_fp64_population_control_3d_with_implicit_capture_and_collision_estimator(mcdc):
    prob = small_channel()
    N, B, M = 12_000, 4, 2500
    kw = dict(estimator=mcdc.EST_COLLISION, implicit=(0.1, 0.3), pc_target=M)
    g = mcdc.run_numpy(prob, N, seed=8, batches=B, precision=mcdc.PREC_FP64, **kw)
    o = O.run(prob, N, seed=8, batches=B, estimator=O.EST_COLLISION, implicit=(0.1, 0.3),
              pc_target=M)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_pc(g["counts"], o["counts"])
    assert g["counts"]["pc_combs"] > 0


@pytest.mark.parametrize("prec", ["fp32", "fp32_local"])
def test_fp32_population_control_statistical(mcdc, prec):
    P32 = mcdc.PREC_FP32 if prec == "fp32" else mcdc.PREC_FP32_LOCAL
    prob = W.c2_two_region()
    N, B = 1_000_000, 40
    g = mcdc.run_numpy(prob, N, seed=2, batches=B, precision=P32, pc_target=N // B)
    o = O.run(prob, 200_000, seed=1, batches=B, pc_target=200_000 // B)
    c = g["counts"]
    assert c["histories"] + c["pc_out"] - c["pc_in"] == (
        c["absorbed"] + c["leaked"] + c["censused"] + c["roulette_killed"])
    assert c["w_pc_out"] == pytest.approx(c["w_pc_in"], rel=1e-5)
    (mg, rg), (mo, ro) = g["scalar"], o["scalar"]
    z = (mg - mo) / np.hypot(mg * rg, mo * ro)
    assert abs(z) < 4.0, (mg, mo, z)
    fp32_bins_agree(g, o, batches=B)


def test_population_control_refusals(mcdc):
    prob = W.c2_two_region()
    with pytest.raises(mcdc.MCDCError):       # the comb runs on the global tally
        mcdc.Problem(prob, tally_mode=mcdc.TALLY_SHARED, pc_target=100)
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64, pc_target=100) as P:
        with pytest.raises(mcdc.MCDCError):   # weight windows and a comb
            P.set_weight_windows(np.ones(P.n_bins), 5.0, 2.5, 16)
        with pytest.raises(mcdc.MCDCError):   # histories mix: no per-history records
            P.run_ex(1000, 1, batches=4, records=np.zeros(10, dtype=mcdc.RECORD_DTYPE))
        with pytest.raises(mcdc.MCDCError):   # batched runs are analog
            mcdc.run_batched([P], [1000], 1, batches=4, means=[np.zeros(P.n_bins)])
        # and the handle still runs
        st, _ = P.run_ex(2000, 1, batches=4)
        assert st["pc_combs"] > 0
