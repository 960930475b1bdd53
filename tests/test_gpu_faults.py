"""Failure paths on the GPU, without faulting it: a run whose split children
find the warp stacks full does not fail or trap -- the children that find no
room are not made, their parent keeps their weight, the count is reported,
and the flux stays unbiased -- and the same context runs a correct problem
right afterwards.  The kernels have no device-side waits, so there is no
timeout path to exercise in the tracker.  The tensor-core kernels of the
importance network do wait (on MMA completion, bounded): with the wait limit
at zero every wait gives up, the call reports MCDC_ERR_TIMEOUT, and the same
context computes correct results once the limit is restored."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def test_split_overflow_drops_children_unbiased_and_the_context_survives(mcdc):
    mat = np.zeros((2, 2, 2), np.uint8)
    prob = W.box("box", (2, 2, 2), (1.0, 1.0, 1.0), mat, [[1.0]], [[0.95]], np.ones((1, 1, 1)),
                 [1.0], (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), None, (0, 0, 0), (2, 2, 2),
                 bc=(W.BC_REFLECT,) * 6)
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32, tally_mode=mcdc.TALLY_SHARED,
                      block_size=128, overflow_per_cta=256) as P:
        # windows 1e6 times below the source weight: every event wants a
        # 16-fold split, far more children than 64 stack slots per warp hold
        P.set_weight_windows(np.full(P.n_bins, 1e-6), 5.0, 2.5, 16)
        mean, rel = np.zeros(P.n_bins), np.zeros(P.n_bins)
        stats, _ = P.run_ex(4000, 3, batches=16, mean=mean, relerr=rel)
        assert stats["splits_dropped"] > 0 and stats["children"] > 0
        # infinite medium: every cell's flux is 1 / (Sigma_a V_box)
        z = (mean - 1.0 / (0.05 * 8.0)) / (mean * rel)
        assert np.all(np.abs(z) < 4.5), z
        P.set_weight_windows(None)                    # back to analog
        stats, _ = P.run_ex(2000, 3, batches=4)
        assert stats["absorbed"] == 2000 and stats["splits_dropped"] == 0
    # and a fresh problem still matches the oracle exactly
    p2 = W.c1_slab()
    g = mcdc.run_numpy(p2, 5000, 2, batches=5, precision=mcdc.PREC_FP64)
    o = O.run(p2, 5000, seed=2, batches=5)
    nz = o["sum1"] != 0
    np.testing.assert_allclose(g["sum1"][nz], o["sum1"][nz], rtol=1e-9)


def test_tensor_core_wait_timeout_is_reported_and_the_context_survives(mcdc):
    rng = np.random.default_rng(5)
    n_in = 8
    p = rng.normal(0, 0.3, O.mlp_param_count(n_in))
    X = rng.uniform(-1, 1, (3000, n_in))
    y, w = rng.normal(size=3000), rng.uniform(0.5, 1.0, 3000)
    try:
        mcdc.set_wait_limit(0)
        with pytest.raises(mcdc.MCDCError) as e:
            mcdc.mlp_forward(p.astype(np.float32), X.astype(np.float32))
        assert e.value.code == mcdc.MCDC_ERR_TIMEOUT
        with pytest.raises(mcdc.MCDCError) as e:
            mcdc.mlp_loss_grad(p, X, y, w)
        assert e.value.code == mcdc.MCDC_ERR_TIMEOUT
    finally:
        mcdc.set_wait_limit(-1)
    got = mcdc.mlp_forward(p.astype(np.float32), X.astype(np.float32))
    ref = O.mlp_forward(p, X)
    assert np.abs(got - ref).max() < 2e-2 * np.abs(ref).max()


def test_children_budget_bounds_explosive_windows(mcdc):
    """Windows that fall tenfold every two cells split a right-moving particle
    at every crossing: with a budget of 200k children the run ends and drops
    the splits past the budget (the parent keeps the weight).  Past the
    budget a split makes nothing and the particle goes on as before: with a
    budget of 1 (no 256-child reservation ever succeeds) an FP64 run with
    these windows is the analog run event for event.  (The far-region flux
    of a 20k-history run here is too heavy-tailed for a z-test: analog FP32
    and FP64 runs of that size differ sixfold in it.)"""
    import numpy as np
    from paper_2409_04668_b300 import workloads as W
    nc = 40
    prob = W.slab("explosive_windows", 20.0, nc, np.zeros(nc), [[1.0]], [[0.9]], src=(0.0, 2.0))
    lower = 10.0 ** (-np.arange(nc) / 2.0)
    N = 20_000
    budget = 200_000
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32, tally_mode=mcdc.TALLY_GLOBAL,
                      max_children=budget, region=((30, 0, 0), (40, 1, 1))) as P:
        P.set_weight_windows(lower, 5.0, 2.5, 16)
        st, (m_w, r_w) = P.run_ex(N, 3, batches=20)
    assert st["splits_dropped"] > 0
    assert st["children"] <= budget
    assert np.isfinite(m_w) and m_w > 0
    sums = []
    for windows in (False, True):
        with mcdc.Problem(prob, precision=mcdc.PREC_FP64, tally_mode=mcdc.TALLY_GLOBAL,
                          max_children=1) as P:
            if windows:
                P.set_weight_windows(lower, 5.0, 2.5, 16)
            s1 = np.zeros(P.n_bins)
            st, _ = P.run_ex(N, 4, batches=20, sum1=s1)
            sums.append((s1, st))
    (s_a, st_a), (s_w, st_w) = sums
    assert st_w["children"] == 0 and st_w["splits_dropped"] > 0
    assert st_w["collisions"] == st_a["collisions"] and st_w["leaked"] == st_a["leaked"]
    np.testing.assert_allclose(s_w, s_a, rtol=1e-9, atol=0)
