"""Collision-order-resolved pins of the oracle's whole transport loop, by
RNG-injection quadrature (the test hook orc_inject_grid replaces the Philox
draws of a history by the nodes of a product quadrature rule).

A beam enters a one-cell slab [0, L] at x = 0 along +x (one group, sigma_t,
scattering ratio c, vacuum on both sides).  Its expected track length after
exactly k collisions is, per source particle:

  k = 0:  T0 = (1 - e^{-st L}) / st
  k = 1:  T1 = int_0^L c st e^{-st x} T(x) dx
  k = 2:  T2 = int_0^L c st phi1(x) T(x) dx,
          phi1(x) = int_0^L c st e^{-st x'} E1(st |x - x'|) / 2 dx'

with T(x) = [1 - (E2(st x) + E2(st (L - x))) / 2] / st the expected track of
an isotropic flight from x (E_n the exponential integrals): the textbook
collided-flux kernels of the slab, evaluated here by scipy quadrature,
independent of the oracle.  The oracle's loop draws the first flight's
distance, the absorption test, the new cosine, the next flight's distance
and so on; integrating those draws over product rules (graded where -ln xi
and the grazing cosine are singular, split where the first flight leaves the
slab) gives the three numbers as deterministic quadratures.  Orders 0 and 1
converge as h^2 (Richardson from two rules reaches ~1e-6); order 2, whose
integrand jumps where the second flight leaves the slab, converges more
slowly and is held to 1 %.  The absorption test is integrated exactly (c is
a multiple of the absorption rule's cell width).
"""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W

# draw slots of a beam history in a one-cell slab: source blocks 0-3 (slots
# 0-7), flight 1 (8), collision 1 (absorption 10, group 11, cosine 12,
# azimuth 13), flight 2 (14), collision 2 (16, 17, 18, 19), flight 3 (20)
N_SLOTS = 22
S_D1, S_ABS1, S_MU1, S_D2, S_ABS2, S_MU2, S_D3 = 8, 10, 12, 14, 16, 18, 20


def references(L, st, c):
    E1 = special.exp1

    def E2(a):
        return special.expn(2, a)

    def T(x):
        return (1.0 - (E2(st * x) + E2(st * (L - x))) / 2.0) / st

    T0 = (1.0 - np.exp(-st * L)) / st
    T1 = integrate.quad(lambda x: c * st * np.exp(-st * x) * T(x), 0.0, L, epsabs=1e-13)[0]

    def phi1(x2):
        f = lambda x1: c * st * np.exp(-st * x1) * E1(st * abs(x2 - x1)) / 2.0
        return (integrate.quad(f, 0.0, x2, limit=200, epsabs=1e-13)[0] +
                integrate.quad(f, x2, L, limit=200, epsabs=1e-13)[0])

    T2 = integrate.quad(lambda x: c * st * phi1(x) * T(x), 0.0, L, limit=200, epsabs=1e-12)[0]
    return T0, T1, T2


def rule_first_flight(m, L, st):
    """xi below e^{-st L}: the flight leaves the slab (one node); above it a
    midpoint rule in the distance d = -ln(xi) / st on [0, L] with the exact
    xi-measure of each cell as its weight."""
    a = np.exp(-st * L)
    d = L * np.arange(m + 1) / m
    xi = np.exp(-st * d)
    dm = L * (np.arange(m) + 0.5) / m
    return np.concatenate([[a / 2], np.exp(-st * dm)]), np.concatenate([[a], xi[:-1] - xi[1:]])


def rule_distance(m):
    """xi = u^2 (nodes crowd xi -> 0, where -ln xi grows without bound)."""
    u = np.arange(m + 1) / m
    return ((np.arange(m) + 0.5) / m) ** 2, np.diff(u ** 2)


def rule_cosine(m):
    """Uniform in xi (mu = 2 xi - 1)."""
    return (np.arange(m) + 0.5) / m, np.full(m, 1.0 / m)


def rule_absorption(c, cells):
    """Midpoints of `cells` equal cells: exact for the step xi < c."""
    x = (np.arange(cells) + 0.5) / cells
    assert abs(c * cells - round(c * cells)) < 1e-12
    return x, np.full(cells, 1.0 / cells)


CASES = [(2.0, 1.0, 0.5, 2), (3.0, 0.7, 0.75, 4)]


@pytest.mark.parametrize("L,st,c,cells", CASES)
def test_uncollided_and_once_collided_track_lengths(L, st, c, cells):
    prob = W.slab("order_slab", L, 1, np.zeros(1), [[st]], [[c]], src=(0.0, 0.0),
                  kind=W.SRC_BEAM)
    T0, T1, _ = references(L, st, c)
    est = []
    for m in (100, 200):
        dims = [(S_D1, *rule_first_flight(m, L, st)), (S_ABS1, *rule_absorption(c, cells)),
                (S_MU1, *rule_cosine(m)), (S_D2, *rule_distance(m))]
        est.append(O.inject_grid(prob, N_SLOTS, dims, max_order=1))
    rich = (4.0 * est[1] - est[0]) / 3.0               # h^2 convergence
    assert abs(est[1][0] - T0) < 2e-5 * T0 and abs(est[1][1] - T1) < 1e-4 * T1
    assert rich[0] == pytest.approx(T0, rel=2e-6)
    assert rich[1] == pytest.approx(T1, rel=1e-5)


@pytest.mark.parametrize("L,st,c,cells", CASES)
def test_twice_collided_track_length(L, st, c, cells):
    prob = W.slab("order_slab", L, 1, np.zeros(1), [[st]], [[c]], src=(0.0, 0.0),
                  kind=W.SRC_BEAM)
    T0, T1, T2 = references(L, st, c)
    err = []
    for m in (12, 24):
        dims = [(S_D1, *rule_first_flight(m, L, st)), (S_ABS1, *rule_absorption(c, cells)),
                (S_MU1, *rule_cosine(m)), (S_D2, *rule_distance(m)),
                (S_ABS2, *rule_absorption(c, cells)), (S_MU2, *rule_cosine(m)),
                (S_D3, *rule_distance(m))]
        o = O.inject_grid(prob, N_SLOTS, dims, max_order=2)
        err.append(abs(o[2] - T2) / T2)
    assert err[1] < 1e-2 and err[1] < err[0], err
