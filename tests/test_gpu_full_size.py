"""The full-size 3-D workloads, in the launch configuration the benchmark
times, checked where the oracle cannot run them whole: on sampled histories
and by properties that hold at any size.

* Channel box (60^3 mesh, 7 groups, 20 time bins) and deep-penetration box
  (100 x 40 x 40 mesh, 4 groups, 10 time bins), 1e8 histories each: the FP64
  run over all of them, with per-history records of the first 1e6, matches the
  oracle event for event on 1500 of those chosen at random; every history of
  the FP64 and the FP32-split runs ends exactly once (absorbed, leaked or
  censused); the FP32-split run's fractions of absorbed, leaked and censused
  histories agree with the FP64 run's (independent seeds: a two-sample
  binomial z below 5).  (Both region totals are zero: 1e8 analog histories
  never reach these regions, which is what the weight windows are for.)
* 256 batched problems (3.3e8 histories): the batched FP32 run accounts for
  every history of every problem.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W
from parity_util import compare_records

pytestmark = pytest.mark.gpu

N = 100_000_000
N_REC = 1_000_000


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def _balanced(st, n):
    assert st["histories"] == n
    assert st["absorbed"] + st["leaked"] + st["censused"] == n, st


@pytest.mark.parametrize("name", ["c3_channel", "c4_deep"])
def test_full_size_sampled_histories_and_balance(mcdc, name):
    prob = getattr(W, name)()
    with mcdc.Problem(prob, precision=mcdc.PREC_FP64) as P:
        rec = np.zeros(N_REC, dtype=mcdc.RECORD_DTYPE)
        st64, (m64, r64) = P.run_ex(N, 1, records=rec, n_records=N_REC)
    _balanced(st64, N)
    pick = np.sort(np.random.default_rng(3).choice(N_REC, 1500, replace=False))
    compare_records(rec[pick], O.trace(prob, 1, pick), dim=3)
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32) as P:
        st32, (m32, r32) = P.run_ex(N, 2)
    _balanced(st32, N)
    print(name, "segments per history FP64", st64["segments"] / N, "FP32", st32["segments"] / N,
          "region", m64, r64, m32, r32)
    for k in ("absorbed", "leaked", "censused"):
        p64, p32 = st64[k] / N, st32[k] / N
        pp = 0.5 * (p64 + p32)
        se = np.sqrt(2.0 * pp * (1.0 - pp) / N)
        z = (p32 - p64) / se if se > 0 else 0.0
        print(k, p64, p32, "z", z)
        assert abs(z) < 5.0, (k, p64, p32, z)


def test_full_size_batched_problems_account_for_every_history(mcdc):
    probs, hist = W.c5_batch()
    handles = [mcdc.Problem(p, precision=mcdc.PREC_FP32, block_size=256) for p in probs]
    try:
        st, scal = mcdc.run_batched(handles, hist, 5, batches=16)
    finally:
        for h in handles:
            h.close()
    total = int(np.sum(hist))
    _balanced(st, total)
    assert len(scal) == len(probs)
