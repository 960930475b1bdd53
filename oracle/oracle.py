"""ctypes wrapper around the C oracle (``liborc.so``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the product path.  It imports
nothing from the CUDA package; problems are passed as any object carrying the
attributes of a problem description (mesh, materials, source, time grid).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcProblem(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 3), ("origin", C.c_double * 3), ("width", C.c_double * 3),
        ("material", C.c_void_p), ("bc", C.c_int32 * 6),
        ("n_mat", C.c_int32), ("n_grp", C.c_int32),
        ("sigma_t", C.c_void_p), ("sigma_s", C.c_void_p), ("transfer", C.c_void_p),
        ("speed", C.c_void_p),
        ("src_lo", C.c_double * 3), ("src_hi", C.c_double * 3), ("src_kind", C.c_int32),
        ("src_dir", C.c_double * 3), ("src_pdf", C.c_void_p),
        ("src_t0", C.c_double), ("src_t1", C.c_double),
        ("n_tbin", C.c_int32), ("edges", C.c_void_p),
        ("ww_lower", C.c_void_p), ("ww_upper_ratio", C.c_double),
        ("ww_survival_ratio", C.c_double), ("ww_nmax", C.c_int32),
        ("ww_net", C.c_void_p), ("ww_net_in", C.c_int32), ("ww_net_h", C.c_int32),
        ("ww_net_shift", C.c_double), ("ww_net_scale", C.c_double),
        ("ww_net_top", C.c_double), ("ww_net_floor", C.c_double), ("ww_net_wl0", C.c_double),
        ("region_lo", C.c_int32 * 3), ("region_hi", C.c_int32 * 3),
        ("estimator", C.c_int32), ("implicit_capture", C.c_int32),
        ("weight_cutoff", C.c_double), ("cutoff_survival", C.c_double),
        ("pc_target", C.c_int32),
    ]


class OrcCounts(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in (
        "histories", "segments", "collisions", "crossings", "census", "absorbed", "leaked",
        "censused", "splits", "children", "roulette_killed", "roulette_survived")] + [
        (k, C.c_double) for k in ("w_source", "w_absorbed", "w_leaked", "w_censused")] + [
        (k, C.c_uint64) for k in ("pc_combs", "pc_in", "pc_out")] + [
        (k, C.c_double) for k in ("w_pc_in", "w_pc_out")]


RECORD_DTYPE = np.dtype([
    ("hid", np.uint64), ("end", np.int32), ("g", np.int32), ("ctr", np.uint32),
    ("n_seg", np.uint32), ("n_col", np.uint32), ("n_cross", np.uint32),
    ("x", np.float64), ("y", np.float64), ("z", np.float64), ("t", np.float64),
    ("w", np.float64)], align=True)

END_ABSORBED, END_LEAKED, END_CENSUSED, END_ROULETTE = 1, 2, 3, 4
EST_TRACK, EST_COLLISION, EST_COMBINED = 0, 1, 2


def lib():
    global _lib
    if _lib is None:
        # an alternative build of the oracle (e.g. one with a planted mistake)
        path = os.environ.get("MCDC_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        L.orc_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_uniform.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_uniform.restype = C.c_double
        L.orc_isotropic.argtypes = [C.c_double, C.c_double, C.c_void_p]
        L.orc_run.argtypes = [C.POINTER(OrcProblem), C.c_uint64, C.c_uint64, C.c_uint64,
                              C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(OrcCounts)]
        L.orc_run.restype = C.c_int
        L.orc_trace.argtypes = [C.POINTER(OrcProblem), C.c_uint64, C.c_void_p, C.c_int64,
                                C.c_void_p]
        L.orc_trace.restype = C.c_int
        L.orc_comb.argtypes = [C.c_int64, C.c_void_p, C.c_int64, C.c_double, C.c_void_p]
        L.orc_net_features.argtypes = [C.POINTER(OrcProblem), C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_int32, C.c_int32, C.c_void_p]
        L.orc_combine.argtypes = [C.c_int64] + [C.c_void_p] * 5 + [C.c_uint64, C.c_int32,
                                                                    C.c_double] + [C.c_void_p] * 3
        if hasattr(L, "orc_mlp_forward"):
            _bind_mlp(L)
        _lib = L
    return _lib


def _bind_mlp(L):
    L.orc_mlp_train.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.orc_mlp_train.restype = None
    L.orc_mlp_error_bounds.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
    L.orc_mlp_error_bounds.restype = None
    L.orc_mlp_window_bound.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.c_double, C.c_double, C.c_double, C.c_void_p]
    L.orc_mlp_window_bound.restype = None
    L.orc_mlp_param_count.argtypes = [C.c_int32, C.c_int32]
    L.orc_mlp_param_count.restype = C.c_int64
    L.orc_mlp_forward.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                  C.c_void_p, C.c_void_p]
    L.orc_mlp_loss_grad.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_adam_step.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Holds the arrays a C struct points into for the length of a call."""

    def __init__(self):
        self.arrays = []

    def ptr(self, a):
        self.arrays.append(a)
        return a.ctypes.data


def _struct(prob, ww=None, keep=None, estimator=EST_TRACK, implicit=None, pc_target=0):
    """implicit: None (analog collisions) or (weight cutoff, survival weight);
    pc_target: particles per batch after each census comb (0: no comb)."""
    s = OrcProblem()
    s.n[:] = list(prob.n)
    s.origin[:] = [float(v) for v in prob.origin]
    s.width[:] = [float(v) for v in prob.width]
    mat = np.ascontiguousarray(prob.material, dtype=np.uint8)
    s.material = keep.ptr(mat)
    s.bc[:] = list(prob.bc)
    st = _f64(prob.sigma_t)
    s.n_mat, s.n_grp = st.shape
    s.sigma_t = keep.ptr(st)
    s.sigma_s = keep.ptr(_f64(prob.sigma_s))
    s.transfer = keep.ptr(_f64(prob.transfer))
    s.speed = keep.ptr(_f64(prob.speed))
    s.src_lo[:] = [float(v) for v in prob.src_lo]
    s.src_hi[:] = [float(v) for v in prob.src_hi]
    s.src_kind = int(prob.src_kind)
    s.src_dir[:] = [float(v) for v in prob.src_dir]
    s.src_pdf = keep.ptr(_f64(prob.src_pdf))
    s.src_t0, s.src_t1 = float(prob.src_t0), float(prob.src_t1)
    if prob.edges is None:
        s.n_tbin, s.edges = 0, None
    else:
        e = _f64(prob.edges)
        s.n_tbin, s.edges = len(e) - 1, keep.ptr(e)
    if ww is not None:
        # a table of lower bounds ("lower"), or per-event windows from the
        # network ("net": parameters, "hidden", "shift", "scale", "top",
        # "floor", "wl0", optional "n_in": 3 for a network over the position
        # alone, else 4 + G; R15)
        if "net" in ww:
            s.ww_net = keep.ptr(_f64(ww["net"]))
            s.ww_net_in = int(ww.get("n_in", 4 + int(np.asarray(prob.sigma_t).shape[1])))
            s.ww_net_h = int(ww.get("hidden", 64))
            s.ww_net_shift, s.ww_net_scale = float(ww["shift"]), float(ww["scale"])
            s.ww_net_top, s.ww_net_floor = float(ww["top"]), float(ww["floor"])
            s.ww_net_wl0 = float(ww["wl0"])
        else:
            s.ww_lower = keep.ptr(_f64(ww["lower"]))
        s.ww_upper_ratio = float(ww.get("upper_ratio", 5.0))
        s.ww_survival_ratio = float(ww.get("survival_ratio", 2.5))
        s.ww_nmax = int(ww.get("nmax", 16))
    s.region_lo[:] = list(prob.region_lo)
    s.region_hi[:] = list(prob.region_hi)
    s.estimator = int(estimator)
    s.pc_target = int(pc_target)
    if implicit is not None:
        s.implicit_capture = 1
        s.weight_cutoff, s.cutoff_survival = float(implicit[0]), float(implicit[1])
    return s


def n_bins(prob):
    T = 1 if prob.edges is None else len(prob.edges) - 1
    return int(np.prod(prob.n)) * int(np.asarray(prob.sigma_t).shape[1]) * T


def tally_shape(prob):
    nx, ny, nz = prob.n
    T = 1 if prob.edges is None else len(prob.edges) - 1
    return (nz, ny, nx, int(np.asarray(prob.sigma_t).shape[1]), T)


def run(prob, n, seed, offset=0, batches=32, threads=None, ww=None, estimator=EST_TRACK,
        implicit=None, pc_target=0):
    """Runs histories [offset, offset+n); returns mean/relerr/sums shaped
    [nz, ny, nx, G, T], the region scalar and the event counts.  estimator:
    EST_TRACK (track length), EST_COLLISION, or EST_COMBINED (both from the
    same histories; mean/relerr/scalar are their minimum-variance combination,
    sum1/sum2 gain a leading axis [track, collision], sum12 holds the summed
    products of the two batch sums, alpha the track-length coefficient per bin
    and scalar_alpha the region scalar's);
    implicit: None or (weight cutoff, survival weight) for implicit capture;
    pc_target: population control, particles per batch after each comb at an
    interior census edge."""
    L = lib()
    keep = _Keep()
    s = _struct(prob, ww, keep, estimator, implicit, pc_target)
    nb = n_bins(prob)
    ne = 2 if estimator == EST_COMBINED else 1
    mean, rel, s12 = np.zeros(nb), np.zeros(nb), np.zeros(nb)
    s1, s2 = np.zeros(ne * nb), np.zeros(ne * nb)
    scalar = np.zeros(3)
    cnt = OrcCounts()
    if threads is None:
        threads = os.cpu_count() or 1
    rc = L.orc_run(C.byref(s), int(n), int(seed), int(offset), int(batches), int(threads),
                   mean.ctypes.data, rel.ctypes.data, s1.ctypes.data, s2.ctypes.data,
                   s12.ctypes.data, scalar.ctypes.data, C.byref(cnt))
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    shp = tally_shape(prob)
    counts = {k: getattr(cnt, k) for k, _ in OrcCounts._fields_}
    out = {"mean": mean.reshape(shp), "relerr": rel.reshape(shp), "scalar": (scalar[0], scalar[1]),
           "counts": counts, "threads": int(threads)}
    if ne == 2:
        out["sum1"] = s1.reshape((2,) + shp)
        out["sum2"] = s2.reshape((2,) + shp)
        out["sum12"] = s12.reshape(shp)
        alpha = np.zeros(nb)
        vol = float(np.prod([w if np.isfinite(w) and w > 0 else 1.0 for w in prob.width]))
        combine(s1[:nb], s2[:nb], s1[nb:], s2[nb:], s12, n, batches, vol, alpha=alpha)
        out["alpha"] = alpha.reshape(shp)
        out["scalar_alpha"] = scalar[2]
    else:
        out["sum1"] = s1.reshape(shp)
        out["sum2"] = s2.reshape(shp)
    return out


def net_features(prob, x, y, z, t, tbin, g, n_in=None):
    """The network's inputs for a particle (R15); n_in 3: the position only."""
    L = lib()
    keep = _Keep()
    n_in = n_in or 4 + int(np.asarray(prob.sigma_t).shape[1])
    s = _struct(prob, {"net": np.zeros(1), "shift": 0.0, "scale": 1.0, "top": 0.0,
                       "floor": 0.0, "wl0": 1.0, "n_in": n_in}, keep)
    f = np.zeros(n_in)
    L.orc_net_features(C.byref(s), float(x), float(y), float(z), float(t), int(tbin), int(g),
                       f.ctypes.data)
    return f


def combine(s1x, s2x, s1y, s2y, s12, n_hist, batches, volume, alpha=None):
    """Minimum-variance combination of two correlated batch series (the
    oracle's R14) from their batch sums: returns (mean, relerr), and fills
    alpha (the coefficient of the first series) if given."""
    L = lib()
    a = [np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (s1x, s2x, s1y, s2y, s12)]
    k = len(a[0])
    mean, rel = np.zeros(k), np.zeros(k)
    ap = alpha.ctypes.data if alpha is not None else None
    L.orc_combine(k, *[v.ctypes.data for v in a], int(n_hist), int(batches), float(volume),
                  mean.ctypes.data, rel.ctypes.data, ap)
    return mean, rel


def trace(prob, seed, hids, ww=None, implicit=None, pc_target=0):
    """Per-history summary of the primary particle of each listed history
    (refused under population control, where histories mix)."""
    L = lib()
    keep = _Keep()
    s = _struct(prob, ww, keep, EST_TRACK, implicit, pc_target)
    h = np.ascontiguousarray(hids, dtype=np.uint64)
    out = np.zeros(len(h), dtype=RECORD_DTYPE)
    rc = L.orc_trace(C.byref(s), int(seed), h.ctypes.data, len(h), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the problem")
    return out


def comb(weights, M, xi):
    """Indices of the particles the M teeth of a comb with offset xi pick."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    sel = np.zeros(int(M), dtype=np.int64)
    lib().orc_comb(w.size, w.ctypes.data, int(M), float(xi), sel.ctypes.data)
    return sel


def philox(ctr, key):
    L = lib()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    L.orc_philox4x32_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def uniform(hi, lo):
    return lib().orc_uniform(int(hi), int(lo))


def isotropic(xi_mu, xi_phi):
    u = np.zeros(3)
    lib().orc_isotropic(float(xi_mu), float(xi_phi), u.ctypes.data)
    return u


# ---- importance network (FP64) ------------------------------------------

def mlp_param_count(n_in, hidden=64):
    return int(lib().orc_mlp_param_count(int(n_in), int(hidden)))


def mlp_forward(params, X, hidden=64, bf16=False):
    """Network output per sample (FP64; bf16: the matrix products' operands
    rounded to BF16 first, the precision the network runs in)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(X.shape[0])
    lib().orc_mlp_forward(X.shape[1], hidden, int(bf16), p.ctypes.data, X.shape[0],
                          X.ctypes.data, out.ctypes.data)
    return out


def mlp_loss_grad(params, X, y, w, hidden=64, bf16=False):
    """Weighted mean-square loss and its gradient (backpropagation, FP64;
    bf16 as in mlp_forward, the backward products included)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.zeros(p.size)
    loss = lib().orc_mlp_loss_grad(X.shape[1], hidden, int(bf16), p.ctypes.data, X.shape[0],
                                   X.ctypes.data, y.ctypes.data, w.ctypes.data, g.ctypes.data)
    return loss, g


def mlp_error_bounds(params, X, y, w, hidden=64):
    """Tolerance of the tensor-core evaluation: first-order bounds of the
    rounding error of every forward output and every gradient element when
    every matrix-product operand is rounded to BF16 and sums run in FP32
    (see orc_mlp_error_bounds).  Returns (f_bound[n], g_bound[np], loss_bound,
    g_abssum[np], g_absmax[np]): the last two are, per gradient element, the sum
    and the largest of the absolute values of its per-sample terms."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    fb = np.zeros(X.shape[0])
    gb, gs, gm = np.zeros(p.size), np.zeros(p.size), np.zeros(p.size)
    lb = C.c_double()
    lib().orc_mlp_error_bounds(X.shape[1], hidden, p.ctypes.data, X.shape[0], X.ctypes.data,
                               y.ctypes.data, w.ctypes.data, fb.ctypes.data, gb.ctypes.data,
                               C.byref(lb), gs.ctypes.data, gm.ctypes.data)
    return fb, gb, lb.value, gs, gm


def mlp_window_bound(params, X, hidden=64, u=2.0 ** -11, eps_t=2.0 ** -9, x_abs=2.0 ** -22):
    """First-order bound of the warp-batched window evaluation's output error
    per sample (see orc_mlp_window_bound): operands of unit roundoff u (2^-11:
    binary16), FP32 sums, activations h + h tanh(h) with tanh within eps_t,
    inputs computed in FP32 with absolute error x_abs."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(X.shape[0])
    lib().orc_mlp_window_bound(X.shape[1], hidden, p.ctypes.data, X.shape[0], X.ctypes.data,
                               float(u), float(eps_t), float(x_abs), out.ctypes.data)
    return out


def adam_step(p, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam_step(p.size, p.ctypes.data, m.ctypes.data, v.ctypes.data, g.ctypes.data,
                        lr, b1, b2, eps, int(t))


def mlp_train(params, X, y, w, epochs, batch, lr, hidden=64, bf16=False):
    """Adam over minibatches of consecutive samples (see orc_mlp_train);
    returns (parameters, first-epoch loss, last-epoch loss)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    p = np.array(params, dtype=np.float64, order="C")
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    lf, ll = C.c_double(), C.c_double()
    lib().orc_mlp_train(X.shape[1], hidden, int(bf16), p.ctypes.data, X.shape[0], X.ctypes.data,
                        y.ctypes.data, w.ctypes.data, int(epochs), int(batch), float(lr),
                        C.byref(lf), C.byref(ll))
    return p, lf.value, ll.value


def inject_grid(prob, n_slots, dims, max_order, fixed=None, threads=None):
    """RNG-injection quadrature (test hook, see orc_inject_grid): the
    weighted mean, over a product rule on the uniform numbers a history
    draws, of the track length made after exactly k collisions, k =
    0..max_order.  dims: list of (slot, nodes, weights), the weights of each
    rule summing to 1; other slots hold `fixed` (default 0.5)."""
    L = lib()
    if not hasattr(L, "_inj_bound"):
        L.orc_inject_grid.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                      C.c_void_p]
        L.orc_inject_grid.restype = C.c_int
        L._inj_bound = True
    keep = _Keep()
    st = _struct(prob, None, keep)
    fx = np.full(n_slots, 0.5) if fixed is None else _f64(fixed)
    ds = np.ascontiguousarray([d[0] for d in dims], dtype=np.int32)
    dm = np.ascontiguousarray([len(d[1]) for d in dims], dtype=np.int32)
    nodes = np.ascontiguousarray(np.concatenate([np.asarray(d[1], float) for d in dims]))
    wts = np.ascontiguousarray(np.concatenate([np.asarray(d[2], float) for d in dims]))
    out = np.zeros(max_order + 1)
    rc = L.orc_inject_grid(C.byref(st), n_slots, fx.ctypes.data, len(dims), ds.ctypes.data,
                           dm.ctypes.data, nodes.ctypes.data, wts.ctypes.data, int(max_order),
                           int(threads or os.cpu_count() or 1), out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the injection grid")
    return out
