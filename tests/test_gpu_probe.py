"""The FP64-pipe probe behind the FP32-split roofline: it returns positive
rates within the B300's physical range (below the nominal 0.625 T FP64
lane-operations/s with some margin for clock boost, above 1 % of it), and the
tracker's FP64-pipe work per second stays below the measured ceiling."""
import pytest

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


def test_fp64_pipe_rates_are_physical(mcdc):
    add, cvt = mcdc.measure_fp64_pipe()
    for r in (add, cvt):
        assert 6e9 < r < 0.8e12, r


def test_tracker_stays_below_the_measured_fp64_ceiling(mcdc):
    add, cvt = mcdc.measure_fp64_pipe()
    mix = 2.0 / (1.0 / add + 1.0 / cvt)
    prob = W.c2_two_region()
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32) as P:
        P.run_ex(2_000_000, 1)
        st, _ = P.run_ex(10_000_000, 2)
    flights_per_s = st["segments"] / (st["kernel_ms"] * 1e-3)
    # 8 FP64-pipe operations per 1-D flight (conversions and adds of x and t)
    assert 8.0 * flights_per_s < 1.05 * mix, (8.0 * flights_per_s, mix)
