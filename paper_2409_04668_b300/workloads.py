"""Seeded synthetic problems shaped like the paper's time-dependent workloads.

This module only builds input data (mesh, materials, source, time grid); it
holds none of the transport arithmetic.  Both the CUDA library's tests and the
CPU oracle's tests take their inputs from here.

The paper's own benchmark is a time-dependent one-group Kobayashi dog-leg
void-duct problem ("Performance" section); its geometry and data are not
reproduced.  ``c3_channel`` is a synthetic stand-in of the same kind: a
near-void dog-leg channel through a scatterer, wrapped by an absorber, with
the source at the channel mouth and the flux tallied in time.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

BC_VACUUM, BC_REFLECT = 0, 1
SRC_ISOTROPIC, SRC_BEAM = 0, 1
INF = math.inf


@dataclasses.dataclass
class Problem:
    name: str
    n: tuple                      # cells (nx, ny, nz)
    origin: tuple                 # low corner (cm)
    width: tuple                  # cell widths; inf on an unbounded axis with n == 1
    material: np.ndarray          # uint8 [nz, ny, nx]
    bc: tuple                     # (-x, +x, -y, +y, -z, +z)
    sigma_t: np.ndarray           # [M, G] 1/cm
    sigma_s: np.ndarray           # [M, G] 1/cm, <= sigma_t
    transfer: np.ndarray          # [M, G, G] rows sum to 1
    speed: np.ndarray             # [G] cm per time unit
    src_lo: tuple
    src_hi: tuple
    src_kind: int
    src_dir: tuple
    src_pdf: np.ndarray           # [G]
    src_t0: float
    src_t1: float
    edges: Optional[np.ndarray]   # [T+1] census times, None = steady state
    region_lo: tuple              # cell box [lo, hi) of the scalar tally
    region_hi: tuple

    @property
    def n_groups(self) -> int:
        return int(self.sigma_t.shape[1])

    @property
    def n_tbins(self) -> int:
        return 1 if self.edges is None else len(self.edges) - 1

    @property
    def tally_shape(self) -> tuple:
        nx, ny, nz = self.n
        return (nz, ny, nx, self.n_groups, self.n_tbins)

    @property
    def n_bins(self) -> int:
        return int(np.prod(self.tally_shape))


def _materials(sig_t: Sequence[Sequence[float]], scat: Sequence[Sequence[float]],
               transfer: np.ndarray):
    st = np.asarray(sig_t, dtype=np.float64)
    c = np.asarray(scat, dtype=np.float64)
    return st, st * c, np.asarray(transfer, dtype=np.float64)


def downscatter_transfer(n_mat: int, n_grp: int, rng: np.random.Generator) -> np.ndarray:
    """Lower-triangular group transfer: P(g -> g') ~ U(0,1) for g' >= g,
    normalised per row; the last group scatters into itself only."""
    P = np.zeros((n_mat, n_grp, n_grp))
    for m in range(n_mat):
        for g in range(n_grp):
            row = np.zeros(n_grp)
            row[g:] = rng.uniform(0.0, 1.0, n_grp - g)
            P[m, g] = row / row.sum()
    return P


def slab(name, length, n_cells, mats_of_cell, sig_t, scat, speed=(1.0,), src=(0.0, None),
         edges=None, bc=(BC_VACUUM, BC_VACUUM), kind=SRC_ISOTROPIC, direction=(1.0, 0.0, 0.0),
         transfer=None, src_pdf=None, src_t=(0.0, 0.0)):
    """A 1-D slab: y and z are unbounded (one cell of infinite width)."""
    st = np.asarray(sig_t, dtype=np.float64)
    G = st.shape[1]
    if transfer is None:
        transfer = np.tile(np.eye(G), (st.shape[0], 1, 1))
    st, ss, tr = _materials(sig_t, scat, transfer)
    lo, hi = src
    hi = length if hi is None else hi
    return Problem(
        name=name, n=(n_cells, 1, 1), origin=(0.0, 0.0, 0.0),
        width=(length / n_cells, INF, INF),
        material=np.asarray(mats_of_cell, dtype=np.uint8).reshape(1, 1, n_cells),
        bc=(bc[0], bc[1], BC_VACUUM, BC_VACUUM, BC_VACUUM, BC_VACUUM),
        sigma_t=st, sigma_s=ss, transfer=tr, speed=np.asarray(speed, dtype=np.float64),
        src_lo=(lo, 0.0, 0.0), src_hi=(hi, 0.0, 0.0), src_kind=kind, src_dir=tuple(direction),
        src_pdf=np.asarray(src_pdf if src_pdf is not None else np.eye(G)[0], dtype=np.float64),
        src_t0=float(src_t[0]), src_t1=float(src_t[1]),
        edges=None if edges is None else np.asarray(edges, dtype=np.float64),
        region_lo=(0, 0, 0), region_hi=(n_cells, 1, 1))


def c1_slab() -> Problem:
    """10 cm slab (10 mfp), one group, sigma_t 1, sigma_s 0.5, vacuum both
    sides, uniform isotropic source over the slab, steady state, 100 bins."""
    return slab("c1_slab_10cm_1g_steady", 10.0, 100, np.zeros(100), [[1.0]], [[0.5]])


def c2_two_region() -> Problem:
    """20 cm slab, region 1 = [0,10] (sigma_t 1.0, sigma_s 0.9), region 2 =
    [10,20] (sigma_t 2.0, sigma_s 0.2); one group, v = 1; pulse at t = 0
    uniform over region 1; 50 time bins on [0, 20]; 200 spatial bins."""
    mats = np.where(np.arange(200) < 100, 0, 1)
    return slab("c2_slab_20cm_2region_td", 20.0, 200, mats, [[1.0], [2.0]], [[0.9], [0.1]],
                speed=(1.0,), src=(0.0, 10.0), edges=np.linspace(0.0, 20.0, 51))


def box(name, n, width, material, sig_t, scat, transfer, speed, src_lo, src_hi, edges,
        region_lo, region_hi, bc=None, kind=SRC_ISOTROPIC, direction=(1.0, 0.0, 0.0),
        src_pdf=None, src_t=(0.0, 0.0), origin=(0.0, 0.0, 0.0)):
    st, ss, tr = _materials(sig_t, scat, transfer)
    G = st.shape[1]
    return Problem(
        name=name, n=tuple(int(v) for v in n), origin=tuple(float(v) for v in origin),
        width=tuple(float(v) for v in width), material=np.ascontiguousarray(material, np.uint8),
        bc=tuple(bc) if bc is not None else (BC_VACUUM,) * 6,
        sigma_t=st, sigma_s=ss, transfer=tr, speed=np.asarray(speed, dtype=np.float64),
        src_lo=tuple(float(v) for v in src_lo), src_hi=tuple(float(v) for v in src_hi),
        src_kind=kind, src_dir=tuple(direction),
        src_pdf=np.asarray(src_pdf if src_pdf is not None else np.eye(G)[0], dtype=np.float64),
        src_t0=float(src_t[0]), src_t1=float(src_t[1]),
        edges=None if edges is None else np.asarray(edges, dtype=np.float64),
        region_lo=tuple(region_lo), region_hi=tuple(region_hi))


def c3_channel(seed: int = 3) -> Problem:
    """60^3 cm box on a 60^3 1-cm mesh.  Material 0: near-void channel
    (sigma_t 1e-4, c 0.5), 1: scatterer (sigma_t 0.5, c 0.9), 2: absorber
    (sigma_t 1.0, c 0.1).  The channel is a 10x10 cm dog-leg from the corner:
    along y, then x, then z; the absorber is a 10 cm shell on the three far
    faces.  7 groups, downscatter transfer U(0,1) normalised, speeds 1e9 to
    1e3 cm/s log-spaced, 20 time bins on [0, 1e-6 s], pulse at t = 0 in the
    10 cm cube at the channel mouth."""
    N = 60
    m = np.ones((N, N, N), dtype=np.uint8)            # [z, y, x]
    z, y, x = np.meshgrid(np.arange(N) + 0.5, np.arange(N) + 0.5, np.arange(N) + 0.5,
                          indexing="ij")
    far = (x > 50) | (y > 50) | (z > 50)
    m[far] = 2
    leg1 = (x < 10) & (z < 10) & (y < 40)
    leg2 = (y > 30) & (y < 40) & (z < 10) & (x < 40)
    leg3 = (x > 30) & (x < 40) & (y > 30) & (y < 40) & (z < 40)
    m[leg1 | leg2 | leg3] = 0
    G = 7
    rng = np.random.default_rng(seed)
    tr = downscatter_transfer(3, G, rng)
    sig_t = [[1e-4] * G, [0.5] * G, [1.0] * G]
    scat = [[0.5] * G, [0.9] * G, [0.1] * G]
    speed = np.logspace(9, 3, G)
    return box("c3_channel_60cube_7g_td", (N, N, N), (1.0, 1.0, 1.0), m, sig_t, scat, tr,
               speed, (0.0, 0.0, 0.0), (10.0, 10.0, 10.0), np.linspace(0.0, 1e-6, 21),
               (30, 30, 30), (40, 40, 40))


def c4_deep(seed: int = 4) -> Problem:
    """100x40x40 cm box, 1 cm mesh; absorber slab x in [35, 65] (sigma_t 1.0,
    c 0.3, 30 mfp) in a filler (sigma_t 0.1, c 0.9); 4 groups with speeds
    1e9, 1e7, 1e5, 1e3 cm/s; 10 time bins on [0, 1e-5 s]; pulse at t = 0 in
    the 10 cm corner cube; scalar tally region x in [90, 100]."""
    nx, ny, nz = 100, 40, 40
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[:, :, 35:65] = 1
    G = 4
    rng = np.random.default_rng(seed)
    tr = downscatter_transfer(2, G, rng)
    sig_t = [[0.1] * G, [1.0] * G]
    scat = [[0.9] * G, [0.3] * G]
    return box("c4_deep_100x40x40_4g_td", (nx, ny, nz), (1.0, 1.0, 1.0), m, sig_t, scat, tr,
               [1e9, 1e7, 1e5, 1e3], (0.0, 0.0, 0.0), (10.0, 10.0, 10.0),
               np.linspace(0.0, 1e-5, 11), (90, 0, 0), (100, ny, nz))


def c4_shallow(seed: int = 4) -> Problem:
    """The deep-penetration box with a 10 cm absorber (x in [35, 45], 10 mfp)
    and the scalar region right behind it (x in [45, 55]): analog histories
    do score there, rarely, so learned and analog figures of merit compare
    directly."""
    p = c4_deep(seed)
    m = np.zeros_like(p.material)
    m[:, :, 35:45] = 1
    return dataclasses.replace(p, name="c4_shallow_100x40x40_4g_td", material=m,
                               region_lo=(45, 0, 0), region_hi=(55, 40, 40))


def c5_batch(n_problems: int = 256, seed: int = 5, hist_lo: float = 1e4, hist_hi: float = 1e7):
    """Independent 3-D problems of uneven size: mesh n^3 with n ~ U{16..64},
    G ~ U{1..7}, four materials with sigma_t ~ U[0.1, 2] and c ~ U[0.1, 0.95]
    scattered cell by cell, uniform isotropic source over the box, steady
    state; histories log-uniform in [hist_lo, hist_hi].  Returns
    (problems, histories)."""
    rng = np.random.default_rng(seed)
    probs, hists = [], []
    for p in range(n_problems):
        n = int(rng.integers(16, 65))
        G = int(rng.integers(1, 8))
        M = 4
        mat = rng.integers(0, M, size=(n, n, n)).astype(np.uint8)
        st = rng.uniform(0.1, 2.0, size=(M, G))
        c = rng.uniform(0.1, 0.95, size=(M, G))
        tr = downscatter_transfer(M, G, rng)
        speed = np.logspace(9, 3, G) if G > 1 else np.array([1e9])
        probs.append(box(f"c5_{p:03d}_n{n}_g{G}", (n, n, n), (1.0, 1.0, 1.0), mat, st, c, tr,
                         speed, (0.0, 0.0, 0.0), (float(n),) * 3, None, (0, 0, 0), (n, n, n)))
        hists.append(int(round(math.exp(rng.uniform(math.log(hist_lo), math.log(hist_hi))))))
    return probs, hists


CONFIGS = {"c1": c1_slab, "c2": c2_two_region, "c3": c3_channel, "c4": c4_deep}
