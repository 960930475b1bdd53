"""The allocation-free run (mcdc_run_noalloc) against the regular run.

mcdc_run_noalloc serves callers that cannot call cudaMalloc while transport
runs (a pool allocator that owns all device memory, or a loop in which an
allocation would stall the device): its scratch lives in a fixed __device__
array inside the library.  These tests call it through the C-ABI twice in a
row on the same problem and compare each result with mcdc_run_ex's, bin by
bin, at the FP64 tally tolerance; they also check that requests beyond the
array's limits are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2409_04668_b300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 1e-9


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M, torch


def channel(n=12, T=8):
    full = W.c3_channel(3)
    f = 60 // n
    return W.box("channel_small", (n, n, n), (1.0 * f,) * 3, full.material[::f, ::f, ::f].copy(),
                 full.sigma_t, full.sigma_s / full.sigma_t, full.transfer, full.speed,
                 (0.0,) * 3, (10.0,) * 3, np.linspace(0.0, 1e-6, T + 1), (n // 2,) * 3, (n,) * 3)


def _close(a, b, rtol):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.all(np.isfinite(a))
    np.testing.assert_allclose(a, b, rtol=rtol, atol=1e-300)


@pytest.mark.parametrize("mode", ["shared", "global"])
def test_noalloc_matches_run_ex_twice(env, mode):
    M, torch = env
    if mode == "shared":
        prob, tm, n, B = W.c2_two_region(), M.TALLY_SHARED, 200_000, 16
    else:
        prob, tm, n, B = channel(), M.TALLY_GLOBAL, 20_000, 8     # 96768 bins
    dev = torch.device("cuda", 0)
    with M.Problem(prob, precision=M.PREC_FP64, tally_mode=tm) as P:
        ref = [torch.zeros(P.n_bins, dtype=torch.float64, device=dev) for _ in range(4)]
        P.run_ex(n, 17, offset=99, batches=B, sum1=ref[0], sum2=ref[1], mean=ref[2],
                 relerr=ref[3])
        torch.cuda.synchronize()
        assert float(ref[0].sum()) > 0
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            out = [torch.full((P.n_bins,), float("nan"), dtype=torch.float64, device=dev)
                   for _ in range(4)]
            P.run_noalloc(n, 17, out[0], out[1], offset=99, batches=B, mean=out[2],
                          relerr=out[3], stream=stream)
            torch.cuda.synchronize()
            _close(out[0], ref[0], REL)
            _close(out[1], ref[1], REL)
            _close(out[2], ref[2], REL)
            _close(out[3], ref[3], 1e-6)


def _inf_medium_ww():
    mat = np.zeros((2, 2, 4), np.uint8)
    return W.box("inf_ww", (4, 2, 2), (0.5, 1.0, 1.0), mat, [[1.0]], [[0.8]], np.ones((1, 1, 1)),
                 [1.0], (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), None, (0, 0, 0), (4, 2, 2),
                 bc=(W.BC_REFLECT,) * 6)


def test_noalloc_weight_windows_match_run_ex_twice(env):
    """Weight windows on the shared tally, whose warp stacks hold every child
    here: the allocation-free run splits and roulettes exactly as
    mcdc_run_ex does, with the same per-run children budget."""
    M, torch = env
    prob = _inf_medium_ww()
    lower = np.random.default_rng(7).uniform(0.05, 0.6, size=prob.n_bins)
    n, B = 20_000, 10
    dev = torch.device("cuda", 0)
    with M.Problem(prob, precision=M.PREC_FP64, tally_mode=M.TALLY_SHARED,
                   overflow_per_cta=8192) as P:
        P.set_weight_windows(lower, 5.0, 2.5, 16)
        ref = [torch.zeros(P.n_bins, dtype=torch.float64, device=dev) for _ in range(4)]
        st, _ = P.run_ex(n, 13, batches=B, sum1=ref[0], sum2=ref[1], mean=ref[2], relerr=ref[3])
        torch.cuda.synchronize()
        assert st["splits"] > 100 and st["roulette_killed"] > 100 and st["splits_dropped"] == 0
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            out = [torch.full((P.n_bins,), float("nan"), dtype=torch.float64, device=dev)
                   for _ in range(4)]
            P.run_noalloc(n, 13, out[0], out[1], batches=B, mean=out[2], relerr=out[3],
                          stream=stream)
            torch.cuda.synchronize()
            _close(out[0], ref[0], REL)
            _close(out[1], ref[1], REL)
            _close(out[2], ref[2], REL)
            _close(out[3], ref[3], 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32_local"])
def test_noalloc_network_windows_match_run_ex(env, prec):
    """Per-event network windows (global tally, the network kernels with their
    own launch shape and fragment block): the allocation-free run takes the
    same kernel and makes the same splits and roulettes as mcdc_run_ex while
    no warp stack overflows (whole stacks kept, so mcdc_run_ex spills nothing
    either) -- FP64 tallies to 1e-9; FP32 ones to FP32 summation-order noise."""
    M, torch = env
    prob = _inf_medium_ww()
    n_in, H = 3, 8
    npar = H * n_in + H + H * H + H + H + 1
    params = np.random.default_rng(5).normal(0.0, 0.5, npar).astype(np.float32)
    precision = M.PREC_FP64 if prec == "fp64" else M.PREC_FP32_LOCAL
    rtol = REL if prec == "fp64" else 1e-5
    n, B = 5_000, 10
    dev = torch.device("cuda", 0)
    with M.Problem(prob, precision=precision, tally_mode=M.TALLY_GLOBAL, overflow_tail=-1) as P:
        P.set_network_windows(params, H, 0.0, 1.5, 2.0, -4.0, 0.5, 4.0, 2.0, 4, n_in=n_in)
        ref = [torch.zeros(P.n_bins, dtype=torch.float64, device=dev) for _ in range(2)]
        st, _ = P.run_ex(n, 17, batches=B, sum1=ref[0], sum2=ref[1])
        torch.cuda.synchronize()
        assert st["splits"] > 1000 and st["roulette_killed"] > 20 and st["splits_dropped"] == 0
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            out = [torch.full((P.n_bins,), float("nan"), dtype=torch.float64, device=dev)
                   for _ in range(2)]
            P.run_noalloc(n, 17, out[0], out[1], batches=B, stream=stream)
            torch.cuda.synchronize()
            _close(out[0], ref[0], rtol)
            _close(out[1], ref[1], rtol)


def _explosive():
    nc = 40
    prob = W.slab("explosive_windows", 20.0, nc, np.zeros(nc), [[1.0]], [[0.9]], src=(0.0, 2.0))
    return prob, 10.0 ** (-np.arange(nc) / 2.0)


def test_noalloc_children_budget_bounds_explosive_windows(env):
    """Windows that fall tenfold every two cells ask for a split at every
    crossing of a right-moving particle, without end.  The allocation-free
    run draws its children from the problem's budget as mcdc_run_ex does;
    with a budget of 1 (a warp reserves 256 children at a time, so no
    reservation ever succeeds) no child is made, every weight stays 1 and
    no roulette fires, so the run ends and is the analog run event for
    event: FP64 sums to the tally tolerance, twice.  (Which particles get
    children under a budget that runs out partway depends on scheduling,
    so such runs are not compared bin by bin.)"""
    M, torch = env
    prob, lower = _explosive()
    n, B = 20_000, 20
    dev = torch.device("cuda", 0)
    kw = dict(precision=M.PREC_FP64, tally_mode=M.TALLY_GLOBAL)
    with M.Problem(prob, **kw) as P:
        ref = [torch.zeros(P.n_bins, dtype=torch.float64, device=dev) for _ in range(2)]
        P.run_ex(n, 4, batches=B, sum1=ref[0], sum2=ref[1])
    torch.cuda.synchronize()
    assert float(ref[0].sum()) > 0
    with M.Problem(prob, max_children=1, **kw) as P:
        P.set_weight_windows(lower, 5.0, 2.5, 16)
        for call in range(2):
            out = [torch.full((P.n_bins,), float("nan"), dtype=torch.float64, device=dev)
                   for _ in range(2)]
            P.run_noalloc(n, 4, out[0], out[1], batches=B,
                          stream=torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            _close(out[0], ref[0], REL)
            _close(out[1], ref[1], REL)


def test_noalloc_refuses_requests_beyond_its_limits(env):
    M, torch = env
    dev = torch.device("cuda", 0)
    big = channel(n=20, T=8)               # 20^3 x 7 x 8 = 448000 bins > 131072
    with M.Problem(big, precision=M.PREC_FP32, tally_mode=M.TALLY_GLOBAL) as P:
        s1 = torch.zeros(P.n_bins, dtype=torch.float64, device=dev)
        s2 = torch.zeros(P.n_bins, dtype=torch.float64, device=dev)
        with pytest.raises(M.MCDCError) as e:
            P.run_noalloc(1000, 1, s1, s2, batches=4)
        assert e.value.code == M.MCDC_ERR_INVALID
    with M.Problem(W.c1_slab(), precision=M.PREC_FP32) as P:
        s1 = torch.zeros(P.n_bins, dtype=torch.float64, device=dev)
        s2 = torch.zeros(P.n_bins, dtype=torch.float64, device=dev)
        with pytest.raises(M.MCDCError) as e:
            P.run_noalloc(100_000, 1, s1, s2, batches=5000)
        assert e.value.code == M.MCDC_ERR_INVALID
        h1 = np.zeros(P.n_bins)
        with pytest.raises(M.MCDCError) as e:                 # host outputs are refused
            P.run_noalloc(1000, 1, h1, h1, batches=4)
        assert e.value.code == M.MCDC_ERR_INVALID
