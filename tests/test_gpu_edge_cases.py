"""FP64 event-for-event parity with the oracle on the limits and degenerate
cases of the method: the largest group count (16) with up- and down-scatter,
the largest mesh axis (65535 cells), a single-cell mesh, a point source, a
beam through mesh corners (three-axis ties and zero-length flights), void
cells, mixed reflecting and vacuum faces, one time bin and many (1000) time
bins.  Each case compares every primary's end, group, counter, flight,
collision and crossing counts, position, time and weight, the event counts
and every tally bin (relative 1e-9)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_04668_b300 import workloads as W
from parity_util import compare_counts, compare_records, compare_tallies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def check(mcdc, prob, N, seed, dim, B=4, **kw):
    g = mcdc.run_numpy(prob, N, seed=seed, batches=B, records=N, precision=mcdc.PREC_FP64, **kw)
    o = O.run(prob, N, seed=seed, batches=B)
    compare_tallies(g, o)
    compare_counts(g["counts"], o["counts"])
    compare_records(g["records"], O.trace(prob, seed, np.arange(N)), dim=dim)
    return g, o


def test_sixteen_groups_with_up_and_down_scatter(mcdc):
    G, nc = 16, 20
    rng = np.random.default_rng(11)
    st = rng.uniform(0.5, 2.0, (2, G))
    c = rng.uniform(0.2, 0.9, (2, G))
    P = rng.uniform(0.0, 1.0, (2, G, G))
    P /= P.sum(axis=2, keepdims=True)
    speed = np.logspace(0, 2, G)[::-1]
    mats = (np.arange(nc) >= nc // 2).astype(np.uint8)
    pdf = np.full(G, 1.0 / G)
    prob = W.slab("sixteen_groups", 10.0, nc, mats, st, c, speed=speed, src=(0.0, 10.0),
                  edges=np.linspace(0.0, 0.5, 6), transfer=P, src_pdf=pdf)
    g, o = check(mcdc, prob, 5000, 3, dim=1)
    assert len(np.unique(g["records"]["g"])) == G


@pytest.mark.parametrize("tally", ["auto", "global"])
def test_largest_mesh_axis(mcdc, tally):
    n = 65535
    prob = W.slab("slab_65535", 65.535, n, np.zeros(n), [[1.0]], [[0.5]], src=(0.0, 65.535))
    tm = mcdc.TALLY_GLOBAL if tally == "global" else mcdc.TALLY_AUTO
    check(mcdc, prob, 2000, 5, dim=1, tally_mode=tm)


def test_single_cell_mixed_faces_one_time_bin(mcdc):
    mat = np.zeros((1, 1, 1), np.uint8)
    bc = (W.BC_REFLECT, W.BC_VACUUM, W.BC_REFLECT, W.BC_REFLECT, W.BC_VACUUM, W.BC_REFLECT)
    prob = W.box("one_cell", (1, 1, 1), (2.0, 1.5, 1.0), mat, [[1.0]], [[0.7]], np.ones((1, 1, 1)),
                 [1.0], (0.0, 0.0, 0.0), (2.0, 1.5, 1.0), np.array([0.0, 3.0]), (0, 0, 0),
                 (1, 1, 1), bc=bc)
    check(mcdc, prob, 20_000, 7, dim=3)


def test_point_source_and_void_cells(mcdc):
    n = 6
    mat = np.zeros((n, n, n), np.uint8)
    mat[2:4, :, :] = 1                           # a void slab across the box
    prob = W.box("void_box", (n, n, n), (1.0, 1.0, 1.0), mat, [[1.0], [0.0]], [[0.6], [0.0]],
                 np.ones((2, 1, 1)), [1.0], (2.5, 2.5, 0.5), (2.5, 2.5, 0.5),
                 np.linspace(0.0, 8.0, 9), (0, 0, 4), (n, n, n))
    g, _ = check(mcdc, prob, 20_000, 9, dim=3)
    assert g["counts"]["leaked"] > 0


def test_beam_through_mesh_corners(mcdc):
    # the beam runs along the cube diagonal, exactly through the cell corners:
    # three faces tie at every corner (lowest axis first, then zero-length flights)
    n = 5
    u = 1.0 / math.sqrt(3.0)
    mat = np.zeros((n, n, n), np.uint8)
    prob = W.box("corner_beam", (n, n, n), (1.0, 1.0, 1.0), mat, [[0.3]], [[0.5]],
                 np.ones((1, 1, 1)), [1.0], (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), None, (0, 0, 0),
                 (n, n, n), kind=W.SRC_BEAM, direction=(u, u, u))
    g, o = check(mcdc, prob, 5000, 13, dim=3)
    assert o["counts"]["crossings"] > 3 * 5000 * 0.5


def test_thousand_time_bins(mcdc):
    prob = W.slab("many_bins", 10.0, 40, np.zeros(40), [[1.0]], [[0.9]], speed=(2.0,),
                  src=(0.0, 10.0), edges=np.linspace(0.0, 25.0, 1001), src_t=(0.0, 5.0))
    g, o = check(mcdc, prob, 3000, 17, dim=1, tally_mode=mcdc.TALLY_GLOBAL)
    assert o["counts"]["census"] > 3000 * 50
