"""The importance network on the GPU against the FP64 oracle, and the
learned weight windows against the analog tracker.

* forward pass and every gradient group agree with the oracle within the
  BF16 tolerance (relative 2e-2 of each group's norm);
* training through mcdc_train_importance lowers the loss;
* on a deep-penetration problem (an absorber slab between the source and
  the tally region) the learned weight windows keep the region estimate
  unbiased against an analog run and raise the figure of merit
  1 / (relerr^2 T).
"""
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


def _case(n_in=8, n=3000, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.25, O.mlp_param_count(n_in)).astype(np.float32)
    X = rng.uniform(-1, 1, (n, n_in)).astype(np.float32)
    X[:, 4:] = 0
    X[np.arange(n), 4 + rng.integers(0, n_in - 4, n)] = 1.0
    y = rng.normal(0, 1, n).astype(np.float32)
    w = rng.uniform(0.2, 1.0, n).astype(np.float32)
    w[rng.random(n) < 0.2] = 0.0          # masked samples contribute nothing
    return p, X, y, w


def test_param_count_matches_oracle(mcdc):
    for n_in in (1, 5, 8, 16):
        assert mcdc.mcdc_mlp_param_count(n_in) == O.mlp_param_count(n_in)
    assert mcdc.mcdc_mlp_param_count(17) == -1


def test_forward_matches_oracle(mcdc):
    p, X, y, w = _case()
    got = mcdc.mlp_forward(p, X)
    ref = O.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) < 2e-2 * scale, np.max(np.abs(got - ref)) / scale


@pytest.mark.parametrize("n", [64, 3000, 7777])
def test_gradient_matches_oracle(mcdc, n):
    p, X, y, w = _case(n=n, seed=n)
    loss_g, g = mcdc.mlp_loss_grad(p, X, y, w)
    loss_o, go = O.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), y, w)
    assert abs(loss_g - loss_o) < 2e-2 * abs(loss_o)
    n_in = X.shape[1]
    bounds = np.cumsum([0, 64 * n_in, 64, 64 * 64, 64, 64, 1])
    for a, b in zip(bounds[:-1], bounds[1:]):
        ref = go[a:b]
        err = np.linalg.norm(g[a:b] - ref) / max(np.linalg.norm(ref), 1e-12)
        assert err < 2e-2, (a, b, err)


def deep_slab(absorber=12):
    """A reduced deep-penetration box: 40x8x8 cm, absorber slab of the given
    thickness (sigma_t 1, c 0.3) in a filler (sigma_t 0.1, c 0.9), 2 groups,
    steady state, source in the corner, scalar region at the far end."""
    nx, ny, nz = 40, 8, 8
    m = np.zeros((nz, ny, nx), np.uint8)
    a0 = 12
    m[:, :, a0:a0 + absorber] = 1
    tr = W.downscatter_transfer(2, 2, np.random.default_rng(11))
    return W.box("deep_slab", (nx, ny, nz), (1.0, 1.0, 1.0), m, [[0.1, 0.1], [1.0, 1.0]],
                 [[0.9, 0.9], [0.3, 0.3]], tr, [1e9, 1e7], (0, 0, 0), (4.0, 8.0, 8.0), None,
                 (34, 0, 0), (40, ny, nz))


def test_learned_weight_windows_raise_the_figure_of_merit(mcdc):
    prob = deep_slab(absorber=6)      # thin enough for the analog run to score behind it
    pilot_n, N = 1_000_000, 2_000_000
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32_LOCAL, overflow_per_cta=8192 * 4) as P:
        mean = np.zeros(P.n_bins)
        rel = np.zeros(P.n_bins)
        P.run_ex(pilot_n, 1, mean=mean, relerr=rel)
        st_a, (m_a, r_a) = P.run_ex(N, 2, batches=40)
        rep = P.train_importance(mean, rel, epochs=60, batch=256)
        st_w, (m_w, r_w) = P.run_ex(N, 2, batches=40)
    print("report", rep)
    print("analog", m_a, r_a, st_a["kernel_ms"], "learned", m_w, r_w, st_w["kernel_ms"],
          "splits", st_w["splits"], "roulette", st_w["roulette_killed"])
    assert rep["loss_last"] < 0.5 * rep["loss_first"]
    assert st_w["splits"] > 0 and st_w["roulette_killed"] > 0
    # unbiased: the two estimates of the region flux agree
    z = (m_w - m_a) / np.hypot(m_a * r_a, m_w * r_w)
    assert abs(z) < 4.0, z
    fom_a = 1.0 / (r_a ** 2 * st_a["kernel_ms"])
    fom_w = 1.0 / (r_w ** 2 * st_w["kernel_ms"])
    print("FOM analog", fom_a, "learned", fom_w, "ratio", fom_w / fom_a)
    assert fom_w > 2.0 * fom_a


def test_learned_weight_windows_reach_where_analog_does_not(mcdc):
    prob = deep_slab(absorber=12)
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32_LOCAL, overflow_per_cta=8192 * 4) as P:
        mean = np.zeros(P.n_bins)
        rel = np.zeros(P.n_bins)
        P.run_ex(1_000_000, 1, mean=mean, relerr=rel)
        _, (m_a, r_a) = P.run_ex(1_000_000, 2, batches=20)
        P.train_importance(mean, rel, epochs=60, batch=256)
        st, (m_w, r_w) = P.run_ex(1_000_000, 2, batches=20)
    print("12 cm: analog", m_a, r_a, "learned", m_w, r_w, st["kernel_ms"])
    assert m_a == 0.0                      # no analog history gets through
    assert m_w > 0.0 and r_w < 0.05


def test_importance_windows_from_a_region_source_pilot_are_unbiased(mcdc):
    """Importance (adjoint) windows: the pilot is a run whose source is the
    tally region (the adjoint by reciprocity here: cross sections do not
    depend on the group); the windows fall towards the region and rise away
    from it, and the region estimate agrees with analog."""
    import dataclasses
    prob = deep_slab(absorber=6)
    lo = tuple(prob.origin[a] + prob.region_lo[a] * prob.width[a] for a in range(3))
    hi = tuple(prob.origin[a] + prob.region_hi[a] * prob.width[a] for a in range(3))
    adj = dataclasses.replace(prob, src_lo=lo, src_hi=hi, src_pdf=np.full(2, 0.5))
    with mcdc.Problem(adj, precision=mcdc.PREC_FP32_LOCAL) as A:
        am, ar = np.zeros(A.n_bins), np.zeros(A.n_bins)
        A.run_ex(1_000_000, 3, mean=am, relerr=ar)
    N = 2_000_000
    with mcdc.Problem(prob, precision=mcdc.PREC_FP32_LOCAL) as P:
        _, (m_a, r_a) = P.run_ex(N, 2, batches=40)
        P.train_importance(am, ar, epochs=60, batch=256, adjoint=1)
        st, (m_w, r_w) = P.run_ex(N, 5, batches=40)
    print("importance windows: analog", m_a, r_a, "learned", m_w, r_w, st["kernel_ms"],
          "splits", st["splits"], "roulette", st["roulette_killed"])
    assert st["splits"] > 0 and st["roulette_killed"] > 0
    z = (m_w - m_a) / np.hypot(m_a * r_a, m_w * r_w)
    assert abs(z) < 4.0, z
    assert r_w < r_a
