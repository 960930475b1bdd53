"""The importance network on the GPU against the oracle, and the learned
weight windows against the analog tracker.

Element by element (every forward output, every gradient element, every
trained parameter), against two oracle evaluations of the same definition:

* the oracle with the matrix products' operands rounded to BF16 (the
  precision fixed for the network; accumulation in FP64): the GPU differs
  from it only by FP32 accumulation and by rare BF16 rounding flips of an
  operand whose FP32 value lies next to a rounding boundary, so a gradient
  element may differ by at most 16 x 2^-8 x its largest per-sample term plus
  2^-16 x the sum of its absolute terms, and an output by 1 % of its
  worst-case BF16 bound -- tolerances that a sign flip or a swapped element
  exceeds for more than 99 % of the elements (checked in each test);
* the exact FP64 oracle: the GPU stays inside the first-order bound of the
  BF16 rounding (orc_mlp_error_bounds, pinned on the CPU against an
  independent emulation).

Training (mcdc_mlp_train, the kernel of mcdc_train_importance): one Adam step
moves every parameter whose gradient sign is certain by exactly lr against
it; several epochs of minibatches track the oracle's Adam within 1 % of the
total step; the fit is reproducible bit for bit.

The learned weight windows keep a deep-penetration estimate unbiased
against an analog run and raise the figure of merit 1 / (relerr^2 T).
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


U = 2.0 ** -8


def _tol(gm, gs):
    """GPU against the BF16-operand oracle, per gradient element."""
    return 16 * U * gm + 2.0 ** -16 * gs


@pytest.mark.parametrize("n_in,n", [(8, 3000), (5, 1000), (16, 777)])
def test_forward_matches_oracle(mcdc, n_in, n):
    p, X, y, w = _case(n_in=n_in, n=n, seed=n)
    pd, Xd = p.astype(np.float64), X.astype(np.float64)
    got = mcdc.mlp_forward(p, X)
    fb, _, _, _, _ = O.mlp_error_bounds(pd, Xd, y, w)
    ref16 = O.mlp_forward(pd, Xd, bf16=True)
    ref = O.mlp_forward(pd, Xd)
    # FP32 sums of 64 terms and rare BF16 rounding flips: measured up to 0.002
    # of the worst-case BF16 bound fb on a B300
    assert np.all(np.abs(got - ref16) <= 0.01 * fb), np.max(np.abs(got - ref16) / fb)
    assert np.all(np.abs(got - ref) <= fb), np.max(np.abs(got - ref) / fb)
    # a wrong output (the neighbouring sample's) would not pass
    assert np.mean(np.abs(ref16 - np.roll(ref16, 1)) > 0.01 * fb) > 0.99


@pytest.mark.parametrize("n_in,n", [(8, 64), (8, 3000), (8, 7777), (16, 3000), (5, 1000)])
def test_gradient_matches_oracle(mcdc, n_in, n):
    p, X, y, w = _case(n_in=n_in, n=n, seed=n)
    pd, Xd = p.astype(np.float64), X.astype(np.float64)
    loss_g, g = mcdc.mlp_loss_grad(p, X, y, w)
    loss16, g16 = O.mlp_loss_grad(pd, Xd, y, w, bf16=True)
    loss_o, go = O.mlp_loss_grad(pd, Xd, y, w)
    _, gb, lb, gs, gm = O.mlp_error_bounds(pd, Xd, y, w)
    tol = _tol(gm, gs)
    bad = np.nonzero(np.abs(g - g16) > tol)[0]
    assert bad.size == 0, (bad[:10], (np.abs(g - g16) / tol)[bad[:10]])
    assert np.all(np.abs(g - go) <= gb), np.max(np.abs(g - go) / gb)
    assert abs(loss_g - loss16) <= 1e-5 * loss16 and abs(loss_g - loss_o) <= lb
    # the tolerance separates a sign flip and a swap of neighbours
    assert np.mean(2 * np.abs(g16) > tol) > 0.99
    assert np.mean(np.abs(g16 - np.roll(g16, 1)) > tol) > 0.99


def test_training_one_adam_step_matches_oracle(mcdc):
    """A single minibatch, one epoch: the first Adam step moves each parameter
    by lr * g / (|g| + 1e-8) against its gradient g."""
    n_in, n, lr = 8, 4096, 1e-3
    p, X, y, w = _case(n_in=n_in, n=n, seed=41)
    w = np.maximum(w, 0.05).astype(np.float32)
    pd, Xd = p.astype(np.float64), X.astype(np.float64)
    got, lf, ll = mcdc.mlp_train(p, X, y, w, epochs=1, batch=n, lr=lr)
    ref, lfo, _ = O.mlp_train(pd, Xd, y, w, 1, n, lr, bf16=True)
    _, g16 = O.mlp_loss_grad(pd, Xd, y, w, bf16=True)
    _, _, _, gs, gm = O.mlp_error_bounds(pd, Xd, y, w)
    sure = np.abs(g16) > _tol(gm, gs)            # the GPU's gradient has this sign
    assert sure.mean() > 0.99
    ulp = np.spacing(np.abs(pd).astype(np.float32) + np.float32(lr)).astype(np.float64)
    assert np.all(np.abs(got - ref)[sure] <= 4 * ulp[sure] + 1e-5 * lr)
    assert np.all(np.abs(got - pd)[~sure] <= lr * (1 + 1e-6))
    assert lf == pytest.approx(lfo, rel=1e-5) and ll == lf


@pytest.mark.parametrize("n_in,n,batch,epochs", [(8, 5000, 1024, 3), (12, 20000, 4096, 4)])
def test_training_epochs_match_oracle(mcdc, n_in, n, batch, epochs):
    """Several epochs over minibatches (the last one shorter): every
    parameter within 1 % of the total step K lr of the oracle's Adam on the
    BF16-operand gradients, the epoch losses within 1e-4, and two fits equal
    bit for bit."""
    lr = 2e-3
    p, X, y, w = _case(n_in=n_in, n=n, seed=100 + n)
    w = np.maximum(w, 0.05).astype(np.float32)
    got, lf, ll = mcdc.mlp_train(p, X, y, w, epochs, batch, lr)
    ref, lfo, llo = O.mlp_train(p.astype(np.float64), X.astype(np.float64), y, w, epochs, batch,
                                lr, bf16=True)
    K = epochs * ((n + batch - 1) // batch)
    assert np.all(np.abs(got - ref) <= 0.01 * K * lr), np.max(np.abs(got - ref)) / (K * lr)
    assert lf == pytest.approx(lfo, rel=1e-4) and ll == pytest.approx(llo, rel=1e-4)
    assert ll < lf
    again, _, _ = mcdc.mlp_train(p, X, y, w, epochs, batch, lr)
    assert np.array_equal(got, again)


def test_training_refuses_bad_arguments(mcdc):
    p, X, y, w = _case(n=300)
    with pytest.raises(mcdc.MCDCError) as e:
        mcdc.mlp_train(p, X, y, np.zeros_like(w), 1, 128, 1e-3)   # zero-weight minibatches
    assert e.value.code == mcdc.MCDC_ERR_INVALID
    with pytest.raises(mcdc.MCDCError):
        mcdc.mlp_train(p, X, y, w, 1, 32, 1e-3)                    # batch < 64


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
