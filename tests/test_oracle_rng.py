"""Pins of the oracle's random-number layer against published and exact values.

* Philox4x32-10 against the known-answer vectors of Salmon et al. (SC'11).
* The 53-bit mapping to (0, 1] at its end points and one interior step.
* The isotropic direction law by deterministic quadrature over (xi_mu,
  xi_phi): the first and second moments of a uniform direction on the
  sphere are E[u] = 0 and E[u_i u_j] = delta_ij / 3, and |u| = 1.
* Uniformity of a Philox stream (chi-square over 64 cells).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(v, 16) for v in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert [int(v) for v in O.philox(ctr, key)] == expect


def test_uniform_end_points():
    assert O.uniform(0, 0) == 2.0 ** -53
    assert O.uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0
    assert O.uniform(0, 0x800) == 2.0 * 2.0 ** -53
    # the low 11 bits are dropped
    assert O.uniform(0, 0x7FF) == 2.0 ** -53
    # half way
    assert O.uniform(0x80000000, 0) == 0.5 + 2.0 ** -53


def test_isotropic_moments_by_quadrature():
    n = 200
    xs = (np.arange(n) + 0.5) / n
    acc1 = np.zeros(3)
    acc2 = np.zeros((3, 3))
    for a in xs:
        for b in xs:
            u = O.isotropic(a, b)
            assert abs(np.dot(u, u) - 1.0) < 1e-14
            acc1 += u
            acc2 += np.outer(u, u)
    acc1 /= n * n
    acc2 /= n * n
    assert np.allclose(acc1, 0.0, atol=1e-12)
    assert np.allclose(acc2, np.eye(3) / 3.0, atol=1e-4)


def test_isotropic_axis_convention():
    # mu is the x cosine; phi = 0 points the transverse part along +y
    u = O.isotropic(0.75, 1e-12)
    assert u[0] == 0.5
    assert u[1] == pytest.approx(np.sqrt(0.75))
    assert abs(u[2]) < 1e-10
    u = O.isotropic(0.5, 0.25)       # mu = 0, phi = pi/2 -> +z
    assert np.allclose(u, [0.0, 0.0, 1.0], atol=1e-15)


def test_philox_stream_uniformity():
    counts = np.zeros(64)
    n = 20000
    for i in range(n):
        out = O.philox([i, 7, 123, 0], [1, 0])
        for w in out:
            counts[w >> 26] += 1
    exp = 4 * n / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # 63 degrees of freedom: P(chi2 > 110) < 1e-4
    assert chi2 < 110
