"""The comb's first-tooth rule (population control, csrc/comb.cu), checked on the
host: the tooth positions are T_k = ((double)k + xi) * (W / M) in FP64 (two
roundings, no fused multiply-add), and the first tooth at or after s is the
first k with T_k >= s.  The kernel estimates it as ceil(fma(s, M / W, -xi)) and
accepts the estimate when the ceiling lies more than 1e-5 teeth from it,
because the roundings involved move the boundary by less than ~8 u M (u =
2^-53), below 2e-6 teeth for M < 2^31.  Here the accepted estimates are compared
with a brute-force search over k on random and adversarial inputs (s placed on
and next to tooth positions, large M).  Python floats are IEEE doubles; the
single-rounding fused multiply-add is formed exactly with fractions."""
import math
from fractions import Fraction

import numpy as np


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def tooth(k, xi, wn):
    return (float(k) + xi) * wn


def first_exact(s, xi, wn, M):
    lo, hi = 0, M                     # first k in [0, M] with T_k >= s (M if none)
    while lo < hi:
        mid = (lo + hi) // 2
        if tooth(mid, xi, wn) >= s:
            hi = mid
        else:
            lo = mid + 1
    return lo


def first_fast(s, xi, wn, inv, M):
    """The kernel's accepted estimate, or None when it falls back."""
    e = fma(s, inv, -xi)
    ce = math.ceil(e)
    if ce <= 0:
        return 0 if e < -1e-5 else None
    if ce >= M:
        return M if e > M - 1.0 + 1e-5 else None
    return ce if 1e-5 < ce - e < 1.0 - 1e-5 else None


def test_accepted_estimates_are_exact():
    rng = np.random.default_rng(2409)
    checked = fallback = 0
    random_cases = random_accepted = 0
    for trial in range(4000):
        M = int(rng.choice([1, 2, 7, 1000, 312_500, 2**20 + 3, 2**30 + 7]))
        W = float(rng.uniform(0.1, 1e6)) * float(10.0 ** rng.integers(-6, 6))
        xi = float(rng.uniform(0.0, 1.0)) if trial % 7 else 1.0
        wn, inv = W / M, M / W
        for _ in range(8):
            k = int(rng.integers(0, M))
            t = tooth(k, xi, wn)
            kind = rng.integers(0, 4)
            if kind == 0:
                s = t                                  # exactly on a tooth
            elif kind == 1:
                s = math.nextafter(t, math.inf)        # one ulp past it
            elif kind == 2:
                s = math.nextafter(t, -math.inf)       # one ulp before it
            else:
                s = float(rng.uniform(0.0, W))
            got = first_fast(s, xi, wn, inv, M)
            if kind == 3:
                random_cases += 1
                random_accepted += got is not None
            if got is None:
                fallback += 1
                continue
            assert got == first_exact(s, xi, wn, M), (M, W, xi, s, got)
            checked += 1
    # the fast path takes nearly every random position; positions on or one
    # ulp from a tooth fall back to the exact evaluation
    assert checked > 5000 and fallback > 1000
    assert random_accepted > 0.999 * random_cases
