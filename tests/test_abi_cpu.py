"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function include/mcdc.h declares, and rejects invalid problems on the
host with MCDC_ERR_INVALID before touching a device (or reports
MCDC_ERR_NO_DEVICE when none is present)."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_2409_04668_b300 import build as B
from paper_2409_04668_b300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "mcdc.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mcdc_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2409_04668_b300 import mcdc
    return mcdc


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mcdc_problem_create", "mcdc_run", "mcdc_problem_destroy", "mcdc_run_ex",
                     "mcdc_set_weight_windows", "mcdc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = C.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name), name
        assert name in lib.SIGNATURES, name


def test_checked_build_loads_and_exports_every_declared_symbol(lib):
    """The bounds-checked twin (-DMCDC_CHECKS) builds, exports the same
    boundary and says it is checked; the normal build says it is not (no
    device is needed for either answer)."""
    path = B.build(checked=True)
    raw = C.CDLL(path)
    for name in declared_functions():
        assert hasattr(raw, name), name
    raw.mcdc_build_checked.restype = C.c_int
    assert raw.mcdc_build_checked() == 1
    assert lib.build_checked() is (os.environ.get("MCDC_CHECKS") == "1")
    words = np.zeros(5, dtype=np.int32)
    raw.mcdc_check_selftest.restype = C.c_int
    raw.mcdc_check_selftest.argtypes = [C.c_void_p]
    if not _has_gpu():
        assert raw.mcdc_check_selftest(None) == lib.MCDC_ERR_INVALID
        assert raw.mcdc_check_selftest(words.ctypes.data) == lib.MCDC_ERR_NO_DEVICE


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def _create(lib, prob, **kw):
    try:
        P = lib.Problem(prob, **kw)
    except lib.MCDCError as e:
        return e.code, str(e)
    P.close()
    return 0, ""


def _bad(prob, **changes):
    import dataclasses
    return dataclasses.replace(prob, **changes)


@pytest.mark.parametrize("case", [
    "sigma_s_gt_sigma_t", "negative_sigma", "nan_sigma", "bad_transfer_row", "bad_material_id",
    "source_outside", "source_before_first_edge", "edges_not_increasing", "bad_speed",
    "bad_pdf", "beam_not_unit", "bad_bc"])
def test_invalid_problems_rejected_on_host(lib, case):
    p = W.c2_two_region()
    if case == "sigma_s_gt_sigma_t":
        q = _bad(p, sigma_s=p.sigma_t * 1.5)
    elif case == "negative_sigma":
        q = _bad(p, sigma_t=-p.sigma_t)
    elif case == "nan_sigma":
        st = p.sigma_t.copy()
        st[0, 0] = math.nan
        q = _bad(p, sigma_t=st)
    elif case == "bad_transfer_row":
        q = _bad(p, transfer=p.transfer * 0.5)
    elif case == "bad_material_id":
        m = p.material.copy()
        m[0, 0, 3] = 7
        q = _bad(p, material=m)
    elif case == "source_outside":
        q = _bad(p, src_hi=(25.0, 0.0, 0.0))
    elif case == "source_before_first_edge":
        q = _bad(p, src_t0=-1.0, src_t1=-1.0)
    elif case == "edges_not_increasing":
        e = p.edges.copy()
        e[5] = e[4]
        q = _bad(p, edges=e)
    elif case == "bad_speed":
        q = _bad(p, speed=np.array([0.0]))
    elif case == "bad_pdf":
        q = _bad(p, src_pdf=np.array([0.5]))
    elif case == "beam_not_unit":
        q = _bad(p, src_kind=W.SRC_BEAM, src_dir=(1.0, 1.0, 0.0))
    elif case == "bad_bc":
        q = _bad(p, bc=(0, 0, 0, 0, 0, 9))
    code, msg = _create(lib, q)
    assert code == lib.MCDC_ERR_INVALID, (code, msg)


@pytest.mark.parametrize("case", ["unknown_estimator", "cutoff_above_survival", "zero_cutoff",
                                  "closed_steady_pure_scatterer", "closed_steady_void",
                                  "comb_negative_target", "comb_with_shared_tally",
                                  "comb_in_steady_state", "comb_source_after_first_bin",
                                  "bad_flight_sampling"])
def test_invalid_options_rejected_on_host(lib, case):
    p, kw = W.c2_two_region(), {}
    if case == "unknown_estimator":
        kw["estimator"] = 3
    elif case == "cutoff_above_survival":
        kw["implicit"] = (0.5, 0.25)
    elif case == "zero_cutoff":
        kw["implicit"] = (0.0, 0.5)
    elif case == "comb_negative_target":
        kw["pc_target"] = -5
    elif case == "comb_with_shared_tally":
        kw.update(pc_target=100, tally_mode=lib.TALLY_SHARED)
    elif case == "comb_in_steady_state":
        p, kw["pc_target"] = W.c1_slab(), 100
    elif case == "comb_source_after_first_bin":
        p, kw["pc_target"] = _bad(p, src_t1=1.0), 100
    elif case == "bad_flight_sampling":
        kw["flight_sampling"] = 2
    else:
        # steady state, every face reflecting: only absorption can end a history
        mat = np.zeros((2, 2, 2), np.uint8)
        c = 1.0 if case == "closed_steady_pure_scatterer" else 0.0
        st = 1.0 if case == "closed_steady_pure_scatterer" else 0.0
        p = W.box("closed", (2, 2, 2), (1.0, 1.0, 1.0), mat, [[st]], [[c]], np.ones((1, 1, 1)),
                  [1.0], (0.0,) * 3, (2.0,) * 3, None, (0, 0, 0), (2, 2, 2),
                  bc=(W.BC_REFLECT,) * 6)
    code, msg = _create(lib, p, **kw)
    assert code == lib.MCDC_ERR_INVALID, (code, msg)
    if case.startswith("closed"):
        assert "reflecting" in msg, msg


def test_valid_problem_without_gpu_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    code, msg = _create(lib, W.c1_slab())
    assert code == lib.MCDC_ERR_NO_DEVICE, msg


def test_philox_arguments_checked_on_host(lib):
    assert lib.mcdc_philox(1, None, -1, None) == lib.MCDC_ERR_INVALID
    assert lib.mcdc_philox(1, None, 4, None) == lib.MCDC_ERR_INVALID
    assert lib.mcdc_philox(1, None, 0, None) == lib.MCDC_OK
    import torch
    if not torch.cuda.is_available():
        c = np.zeros((2, 4), np.uint32)
        o = np.zeros_like(c)
        assert lib.mcdc_philox(1, c.ctypes.data, 2, o.ctypes.data) == lib.MCDC_ERR_NO_DEVICE
