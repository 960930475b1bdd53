"""Thin Python binding of the C-ABI in ``include/mcdc.h`` (argument marshalling
only: every step of a run executes in the CUDA library).

The low-level functions keep the C names (``mcdc_problem_create``,
``mcdc_run``, ``mcdc_run_ex``, ``mcdc_set_weight_windows``,
``mcdc_problem_destroy``, ...).  ``Problem`` wraps a handle built from a
``workloads.Problem`` description.  Device outputs are torch tensors (their
``data_ptr``); the run's stream is torch's current stream unless given.

Importing this module loads ``libmcdc_b300.so`` and raises if it is missing:
there is no fallback path.  With the environment variable ``MCDC_CHECKS=1``
it loads the checked build ``libmcdc_b300_checks.so`` instead (the same entry
points; every kernel index bounds-checked, a failure returned as
``MCDC_ERR_CHECK``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_NAME = "libmcdc_b300_checks.so" if os.environ.get("MCDC_CHECKS") == "1" else "libmcdc_b300.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)

MCDC_OK = 0
MCDC_ERR_INVALID, MCDC_ERR_OOM, MCDC_ERR_CUDA = -1, -2, -3
MCDC_ERR_BANK_OVERFLOW, MCDC_ERR_TIMEOUT, MCDC_ERR_NO_DEVICE = -4, -5, -6
MCDC_ERR_CHECK = -7
PREC_FP64, PREC_FP32, PREC_FP32_LOCAL = 0, 1, 2
TALLY_AUTO, TALLY_SHARED, TALLY_GLOBAL = 0, 1, 2
EST_TRACK, EST_COLLISION, EST_COMBINED = 0, 1, 2


class mcdc_mesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("material", C.c_void_p), ("bc", C.c_int32 * 6)]


class mcdc_materials(C.Structure):
    _fields_ = [("n_materials", C.c_int32), ("n_groups", C.c_int32),
                ("sigma_t", C.c_void_p), ("sigma_s", C.c_void_p), ("transfer", C.c_void_p),
                ("speed", C.c_void_p)]


class mcdc_source(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("kind", C.c_int32),
                ("dir", C.c_double * 3), ("group_pdf", C.c_void_p),
                ("t0", C.c_double), ("t1", C.c_double)]


class mcdc_time_grid(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("edges", C.c_void_p)]


class mcdc_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tally_mode", C.c_int32), ("n_batches", C.c_int32),
                ("block_size", C.c_int32), ("bank_per_cta", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("warp_aggregate", C.c_int32),
                ("autotune", C.c_int32), ("overflow_per_cta", C.c_int32),
                ("region_lo", C.c_int32 * 3), ("region_hi", C.c_int32 * 3),
                ("estimator", C.c_int32), ("implicit_capture", C.c_int32),
                ("weight_cutoff", C.c_double), ("cutoff_survival", C.c_double),
                ("pc_target", C.c_int32), ("flight_sampling", C.c_int32),
                ("max_children", C.c_int64), ("slice_bytes_max", C.c_int64),
                ("overflow_tail", C.c_int32), ("spill_particles", C.c_int64)]


class mcdc_stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in (
        "histories", "segments", "collisions", "crossings", "census", "absorbed", "leaked",
        "censused", "splits", "children", "roulette_killed", "roulette_survived")] + [
        (k, C.c_double) for k in ("w_source", "w_absorbed", "w_leaked", "w_censused",
                                  "kernel_ms", "total_ms")] + [
        (k, C.c_int32) for k in ("block_size", "bank_per_cta", "ctas_per_sm", "tally_mode",
                                 "n_batches", "warp_aggregate")] + [("splits_dropped", C.c_uint64)] + [
        (k, C.c_uint64) for k in ("pc_combs", "pc_in", "pc_out")] + [
        (k, C.c_double) for k in ("w_pc_in", "w_pc_out")]


class mcdc_record(C.Structure):
    _fields_ = [("hid", C.c_uint64), ("end", C.c_int32), ("g", C.c_int32),
                ("ctr", C.c_uint32), ("n_seg", C.c_uint32), ("n_col", C.c_uint32),
                ("n_cross", C.c_uint32), ("x", C.c_double), ("y", C.c_double),
                ("z", C.c_double), ("t", C.c_double), ("w", C.c_double)]


RECORD_DTYPE = np.dtype([
    ("hid", np.uint64), ("end", np.int32), ("g", np.int32), ("ctr", np.uint32),
    ("n_seg", np.uint32), ("n_col", np.uint32), ("n_cross", np.uint32),
    ("x", np.float64), ("y", np.float64), ("z", np.float64), ("t", np.float64),
    ("w", np.float64)], align=True)
assert RECORD_DTYPE.itemsize == C.sizeof(mcdc_record)


class mcdc_run_args(C.Structure):
    _fields_ = [("n_histories", C.c_uint64), ("n_batches", C.c_int32), ("seed", C.c_uint64),
                ("hist_offset", C.c_uint64), ("mean_out", C.c_void_p),
                ("relerr_out", C.c_void_p), ("sum1_out", C.c_void_p),
                ("sum2_out", C.c_void_p), ("scalar_out", C.c_void_p),
                ("records", C.c_void_p), ("n_records", C.c_uint64), ("stream", C.c_void_p),
                ("sum12_out", C.c_void_p), ("parts_out", C.c_void_p),
                ("scalar_parts_out", C.c_void_p)]


class mcdc_mlp_options(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double),
                ("seed", C.c_uint64), ("source_wl", C.c_double), ("upper_ratio", C.c_double),
                ("survival_ratio", C.c_double), ("nmax", C.c_int32), ("min_ratio", C.c_double),
                ("time_resolved", C.c_int32), ("group_resolved", C.c_int32),
                ("adjoint", C.c_int32), ("per_event", C.c_int32),
                ("distill_steps", C.c_int32), ("distill_hidden", C.c_int32)]


class mcdc_mlp_report(C.Structure):
    _fields_ = [("samples", C.c_int64), ("loss_first", C.c_double), ("loss_last", C.c_double),
                ("train_ms", C.c_double), ("bake_ms", C.c_double), ("steps", C.c_int32),
                ("target_mean", C.c_double), ("distill_steps", C.c_int32),
                ("distill_loss", C.c_double)]


# name -> (restype, argtypes); kept in the order of include/mcdc.h
SIGNATURES = {
    "mcdc_default_options": (None, [C.POINTER(mcdc_options)]),
    "mcdc_problem_create": (C.c_int, [C.POINTER(mcdc_mesh), C.POINTER(mcdc_materials),
                                      C.POINTER(mcdc_source), C.POINTER(mcdc_time_grid),
                                      C.POINTER(mcdc_options), C.POINTER(C.c_void_p)]),
    "mcdc_run": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p]),
    "mcdc_run_ex": (C.c_int, [C.c_void_p, C.POINTER(mcdc_run_args), C.POINTER(mcdc_stats)]),
    "mcdc_set_weight_windows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                          C.c_int32]),
    "mcdc_tally_size": (C.c_int64, [C.c_void_p]),
    "mcdc_problem_destroy": (None, [C.c_void_p]),
    "mcdc_run_batched": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_uint64, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(mcdc_stats)]),
    "mcdc_default_mlp_options": (None, [C.POINTER(mcdc_mlp_options)]),
    "mcdc_train_importance": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.POINTER(mcdc_mlp_options), C.POINTER(mcdc_mlp_report)]),
    "mcdc_mlp_param_count": (C.c_int64, [C.c_int32]),
    "mcdc_mlp_forward": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p]),
    "mcdc_set_wait_limit": (C.c_int, [C.c_int32]),
    "mcdc_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int64, C.c_void_p, C.POINTER(C.c_double)]),
    "mcdc_mlp_train": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int64, C.c_int32, C.c_int32, C.c_double,
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mcdc_run_noalloc": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcdc_measure_fp64_pipe": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mcdc_set_network_windows": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                           C.c_double, C.c_double, C.c_double, C.c_double,
                                           C.c_double, C.c_double, C.c_double, C.c_int32]),
    "mcdc_get_weight_windows": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mcdc_network_window_lower": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_int64, C.c_void_p]),
    "mcdc_philox": (C.c_int, [C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p]),
    "mcdc_build_checked": (C.c_int, []),
    "mcdc_check_selftest": (C.c_int, [C.c_void_p]),
    "mcdc_last_error": (C.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2409_04668_b300.build` (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
mcdc_default_options = _lib.mcdc_default_options
mcdc_problem_create = _lib.mcdc_problem_create
mcdc_run = _lib.mcdc_run
mcdc_run_ex = _lib.mcdc_run_ex
mcdc_set_weight_windows = _lib.mcdc_set_weight_windows
mcdc_tally_size = _lib.mcdc_tally_size
mcdc_problem_destroy = _lib.mcdc_problem_destroy
mcdc_run_noalloc = _lib.mcdc_run_noalloc
mcdc_default_mlp_options = _lib.mcdc_default_mlp_options
mcdc_run_batched = _lib.mcdc_run_batched
mcdc_train_importance = _lib.mcdc_train_importance
mcdc_mlp_param_count = _lib.mcdc_mlp_param_count
mcdc_mlp_forward = _lib.mcdc_mlp_forward
mcdc_mlp_loss_grad = _lib.mcdc_mlp_loss_grad
mcdc_mlp_train = _lib.mcdc_mlp_train
mcdc_set_wait_limit = _lib.mcdc_set_wait_limit
mcdc_measure_fp64_pipe = _lib.mcdc_measure_fp64_pipe
mcdc_set_network_windows = _lib.mcdc_set_network_windows
mcdc_get_weight_windows = _lib.mcdc_get_weight_windows
mcdc_network_window_lower = _lib.mcdc_network_window_lower
mcdc_philox = _lib.mcdc_philox
mcdc_build_checked = _lib.mcdc_build_checked
mcdc_check_selftest = _lib.mcdc_check_selftest
mcdc_last_error = _lib.mcdc_last_error


class MCDCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mcdc error {code}: {msg}")
        self.code = code


def check(rc):
    if rc != MCDC_OK:
        raise MCDCError(rc, mcdc_last_error().decode())
    return rc


def _ptr(x):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    return x.data_ptr()


class Problem:
    """A problem handle on the current CUDA device (see mcdc_problem_create)."""

    def __init__(self, prob, precision=PREC_FP32, tally_mode=TALLY_AUTO, n_batches=0,
                 block_size=0, bank_per_cta=0, ctas_per_sm=0, warp_aggregate=0,
                 overflow_per_cta=0, region=None, estimator=0, implicit=None, pc_target=0,
                 flight_sampling=0, max_children=0, slice_bytes_max=0, overflow_tail=None,
                 spill_particles=0):
        """estimator: EST_TRACK, EST_COLLISION or EST_COMBINED; implicit: None (analog
        collisions) or (weight cutoff, survival weight) for implicit capture;
        pc_target: population control, particles per batch after each comb
        at an interior census edge (0: off); flight_sampling: FP32 modes, 0
        carries the optical depth across surface and census events, 1 samples
        the distance to collision every flight (the FP64 twin's random
        numbers); max_children: weight windows, split children one run may
        make (0: 4096 per history, at least 2^27; negative: no limit);
        slice_bytes_max: global tally, largest memory for one tally slice per
        batch (one launch for all batches; 0: 8 GiB; negative: one launch per
        batch); overflow_tail: global tally with weight windows, stack slots a
        warp keeps for new children once its own particles are used up (None:
        the library default; -1: the whole stack); spill_particles: global tally
        with weight windows, capacity of each spill bank (0: 2^26)."""
        self.desc = prob
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        m = mcdc_mesh()
        m.nx, m.ny, m.nz = (int(v) for v in prob.n)
        m.x0, m.y0, m.z0 = (float(v) for v in prob.origin)
        m.dx, m.dy, m.dz = (float(v) for v in prob.width)
        m.material = arr(prob.material, np.uint8)
        m.bc[:] = [int(v) for v in prob.bc]
        mt = mcdc_materials()
        st = np.asarray(prob.sigma_t, dtype=np.float64)
        mt.n_materials, mt.n_groups = st.shape
        mt.sigma_t = arr(st, np.float64)
        mt.sigma_s = arr(prob.sigma_s, np.float64)
        mt.transfer = arr(prob.transfer, np.float64)
        mt.speed = arr(prob.speed, np.float64)
        s = mcdc_source()
        s.lo[:] = [float(v) for v in prob.src_lo]
        s.hi[:] = [float(v) for v in prob.src_hi]
        s.kind = int(prob.src_kind)
        s.dir[:] = [float(v) for v in prob.src_dir]
        s.group_pdf = arr(prob.src_pdf, np.float64)
        s.t0, s.t1 = float(prob.src_t0), float(prob.src_t1)
        tg = mcdc_time_grid()
        if prob.edges is not None:
            tg.n_bins = len(prob.edges) - 1
            tg.edges = arr(prob.edges, np.float64)
        o = mcdc_options()
        mcdc_default_options(C.byref(o))
        o.precision = precision
        o.tally_mode = tally_mode
        o.n_batches = n_batches
        o.block_size = block_size
        o.bank_per_cta = bank_per_cta
        o.ctas_per_sm = ctas_per_sm
        o.warp_aggregate = warp_aggregate
        o.overflow_per_cta = overflow_per_cta
        lo, hi = region if region is not None else (prob.region_lo, prob.region_hi)
        o.region_lo[:] = [int(v) for v in lo]
        o.region_hi[:] = [int(v) for v in hi]
        o.estimator = int(estimator)
        o.pc_target = int(pc_target)
        o.flight_sampling = int(flight_sampling)
        o.max_children = int(max_children)
        o.slice_bytes_max = int(slice_bytes_max)
        if overflow_tail is not None:
            o.overflow_tail = int(overflow_tail)
        o.spill_particles = int(spill_particles)
        if implicit is not None:
            o.implicit_capture = 1
            o.weight_cutoff, o.cutoff_survival = float(implicit[0]), float(implicit[1])
        h = C.c_void_p()
        check(mcdc_problem_create(C.byref(m), C.byref(mt), C.byref(s), C.byref(tg), C.byref(o),
                                  C.byref(h)))
        self.handle = h
        self.n_bins = int(mcdc_tally_size(h))
        self.shape = tuple(prob.tally_shape)

    def set_weight_windows(self, lower, upper_ratio=5.0, survival_ratio=2.5, nmax=16):
        if lower is None:
            check(mcdc_set_weight_windows(self.handle, None, 0.0, 0.0, 0))
            return
        if isinstance(lower, np.ndarray):
            lower = np.ascontiguousarray(lower, dtype=np.float64)
        check(mcdc_set_weight_windows(self.handle, _ptr(lower), float(upper_ratio),
                                      float(survival_ratio), int(nmax)))

    def run_ex(self, n, seed, offset=0, batches=0, mean=None, relerr=None, sum1=None, sum2=None,
               records=None, n_records=None, stream=None, want_scalar=True, want_stats=True,
               sum12=None, parts=None, scalar_parts=None):
        """One run; outputs are filled in place (numpy arrays or torch tensors).
        Combined estimator: sum1/sum2 hold [2, n_bins], sum12 [n_bins], parts
        [5, n_bins] and scalar_parts [5] (numpy; track mean, relerr, collision
        mean, relerr, coefficient).  Returns (stats dict or None, (scalar mean,
        scalar relerr) or None)."""
        a = mcdc_run_args()
        a.n_histories = int(n)
        a.n_batches = int(batches)
        a.seed = int(seed)
        a.hist_offset = int(offset)
        a.mean_out = _ptr(mean)
        a.relerr_out = _ptr(relerr)
        a.sum1_out = _ptr(sum1)
        a.sum2_out = _ptr(sum2)
        scal = np.zeros(2) if want_scalar else None
        a.scalar_out = _ptr(scal)
        a.records = _ptr(records)
        a.n_records = int(n_records if n_records is not None else
                          (len(records) if records is not None else 0))
        a.stream = stream
        a.sum12_out = _ptr(sum12)
        a.parts_out = _ptr(parts)
        a.scalar_parts_out = _ptr(scalar_parts)
        st = mcdc_stats() if want_stats else None
        check(mcdc_run_ex(self.handle, C.byref(a), C.byref(st) if st is not None else None))
        stats = {k: getattr(st, k) for k, _ in mcdc_stats._fields_} if st is not None else None
        return stats, (tuple(scal) if scal is not None else None)

    def run_noalloc(self, n, seed, sum1, sum2, offset=0, batches=32, mean=None, relerr=None,
                    stream=None):
        """Allocation-free run (see mcdc_run_noalloc): device tensors only;
        returns once the work is queued on `stream`."""
        check(mcdc_run_noalloc(self.handle, int(n), int(seed), int(offset), int(batches),
                               _ptr(sum1), _ptr(sum2), _ptr(mean), _ptr(relerr), stream))

    def set_network_windows(self, params, hidden, shift, scale, top, floor, wl0,
                            upper_ratio=5.0, survival_ratio=2.5, nmax=16, n_in=None):
        """Per-event windows from the network (see mcdc_set_network_windows);
        params None turns windows off; n_in: 3 (position) or 4 + G (default)."""
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        G = int(np.asarray(self.desc.sigma_t).shape[1])
        check(mcdc_set_network_windows(self.handle, _ptr(p), int(n_in or 4 + G), int(hidden),
                                       float(shift), float(scale), float(top), float(floor),
                                       float(wl0), float(upper_ratio), float(survival_ratio),
                                       int(nmax)))

    def get_weight_windows(self):
        """The last window table set or baked, [n_bins] (see mcdc_get_weight_windows)."""
        out = np.zeros(self.n_bins)
        check(mcdc_get_weight_windows(self.handle, _ptr(out)))
        return out

    def network_window_lower(self, x, t, g):
        """Lower bounds the network's window checks apply at the states
        (positions x[n, 3], times t[n], groups g[n]); see
        mcdc_network_window_lower."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
        g = np.ascontiguousarray(g, dtype=np.int32).reshape(-1)
        assert t.size == x.shape[0] and g.size == x.shape[0]
        out = np.zeros(x.shape[0])
        check(mcdc_network_window_lower(self.handle, _ptr(x), _ptr(t), _ptr(g), x.shape[0],
                                        _ptr(out)))
        return out

    def train_importance(self, pilot_mean, pilot_relerr=None, **opts):
        """Fits the importance network to a pilot tally and switches this
        problem to the weight windows it predicts; returns the report."""
        o = mcdc_mlp_options()
        mcdc_default_mlp_options(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        mean = np.ascontiguousarray(pilot_mean, dtype=np.float64) if isinstance(
            pilot_mean, np.ndarray) else pilot_mean
        rel = np.ascontiguousarray(pilot_relerr, dtype=np.float64) if isinstance(
            pilot_relerr, np.ndarray) else pilot_relerr
        r = mcdc_mlp_report()
        check(mcdc_train_importance(self.handle, _ptr(mean), _ptr(rel), C.byref(o), C.byref(r)))
        return {k: getattr(r, k) for k, _ in mcdc_mlp_report._fields_}

    def run(self, n, seed, tally_out=None):
        check(mcdc_run(self.handle, int(n), int(seed), _ptr(tally_out)))

    def close(self):
        if getattr(self, "handle", None):
            mcdc_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_numpy(prob, n, seed, offset=0, batches=0, records=0, **opts):
    """Convenience: one run with host outputs; returns a dict like the
    oracle wrapper's (mean, relerr, sum1, sum2 shaped [nz,ny,nx,G,T],
    scalar, counts, records; with the combined estimator sum1/sum2 gain a
    leading [track, collision] axis and sum12, parts, scalar_parts appear)."""
    comb = opts.get("estimator", EST_TRACK) == EST_COMBINED
    ne = 2 if comb else 1
    with Problem(prob, **opts) as P:
        nb = P.n_bins
        mean, rel = np.zeros(nb), np.zeros(nb)
        s1, s2 = np.zeros(ne * nb), np.zeros(ne * nb)
        s12 = np.zeros(nb) if comb else None
        parts = np.zeros(5 * nb) if comb else None
        sparts = np.zeros(5) if comb else None
        rec = np.zeros(records, dtype=RECORD_DTYPE) if records else None
        stats, scal = P.run_ex(n, seed, offset=offset, batches=batches, mean=mean, relerr=rel,
                               sum1=s1, sum2=s2, records=rec, sum12=s12, parts=parts,
                               scalar_parts=sparts)
        shp = P.shape
    out = {"mean": mean.reshape(shp), "relerr": rel.reshape(shp), "scalar": scal,
           "counts": stats, "records": rec}
    if comb:
        out.update(sum1=s1.reshape((2,) + shp), sum2=s2.reshape((2,) + shp),
                   sum12=s12.reshape(shp), parts=parts.reshape((5,) + shp), scalar_parts=sparts)
    else:
        out.update(sum1=s1.reshape(shp), sum2=s2.reshape(shp))
    return out


def mlp_forward(params, X):
    """Network prediction on the GPU (FP32 host arrays in and out)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    out = np.zeros(X.shape[0], dtype=np.float32)
    check(mcdc_mlp_forward(_ptr(p), X.shape[1], _ptr(X), X.shape[0], _ptr(out)))
    return out


def philox(seed, ctr):
    """Philox4x32-10 blocks of the counters ctr ([n, 4] uint32) under seed, on
    the GPU with the tracker's routine; returns [n, 4] uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    check(mcdc_philox(int(seed), _ptr(c), c.shape[0], _ptr(out)))
    return out


def measure_fp64_pipe():
    """Measured FP64 add and FP32<->FP64 conversion rates of the current GPU
    (lane-operations per second), see mcdc_measure_fp64_pipe."""
    a, c = C.c_double(), C.c_double()
    check(mcdc_measure_fp64_pipe(C.byref(a), C.byref(c)))
    return a.value, c.value


def build_checked():
    """True when the loaded library is the checked build (mcdc_build_checked)."""
    return bool(mcdc_build_checked())


def check_selftest():
    """The checks' self-test kernel (mcdc_check_selftest): the error words
    (flags, site, index low, index high) and the accesses made."""
    w = np.zeros(5, dtype=np.int32)
    check(mcdc_check_selftest(w.ctypes.data))
    idx = (int(np.uint32(w[3])) << 32) | int(np.uint32(w[2]))
    return {"flags": int(w[0]), "site": int(w[1]), "index": idx, "made": int(w[4])}


def set_wait_limit(tries):
    """Tries of the tensor-core kernels' bounded waits (negative: default)."""
    check(mcdc_set_wait_limit(int(tries)))


def mlp_loss_grad(params, X, y, w):
    """Weighted least-squares loss and gradient computed by the GPU kernels."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    g = np.zeros(p.size, dtype=np.float32)
    loss = C.c_double()
    check(mcdc_mlp_loss_grad(_ptr(p), X.shape[1], _ptr(X), _ptr(y), _ptr(w), X.shape[0], _ptr(g),
                             C.byref(loss)))
    return loss.value, g


def mlp_train(params, X, y, w, epochs, batch, lr):
    """Trains the network (see mcdc_mlp_train); returns (parameters,
    first-epoch loss, last-epoch loss)."""
    p = np.array(params, dtype=np.float32, order="C")
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    lf, ll = C.c_double(), C.c_double()
    check(mcdc_mlp_train(_ptr(p), X.shape[1], _ptr(X), _ptr(y), _ptr(w), X.shape[0], int(epochs),
                         int(batch), float(lr), C.byref(lf), C.byref(ll)))
    return p, lf.value, ll.value


def run_batched(problems, n_histories, seed, batches=0, means=None, relerrs=None):
    """One batched run over Problem handles (see mcdc_run_batched); means /
    relerrs are lists of output arrays (numpy or torch) or None.  Returns
    (stats dict, [(region mean, region relerr)] per problem)."""
    n = len(problems)
    handles = (C.c_void_p * n)(*[p.handle.value for p in problems])
    hist = np.ascontiguousarray(n_histories, dtype=np.uint64)
    mp = (C.c_void_p * n)(*[_ptr(x) for x in means]) if means is not None else None
    rp = (C.c_void_p * n)(*[_ptr(x) for x in relerrs]) if relerrs is not None else None
    scal = np.zeros(2 * n)
    st = mcdc_stats()
    check(mcdc_run_batched(handles, n, _ptr(hist), int(seed), int(batches), mp, rp, _ptr(scal),
                           C.byref(st)))
    stats = {k: getattr(st, k) for k, _ in mcdc_stats._fields_}
    return stats, [(scal[2 * i], scal[2 * i + 1]) for i in range(n)]
