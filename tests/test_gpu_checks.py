"""The bounds-checked build (libmcdc_b300_checks.so, compiled with
-DMCDC_CHECKS) on the GPU: its self-test records the first failing site and
index and skips the access; the parity suites, run through the checked
library in a child process, pass with no check failing -- every index the
tracker and the comb compute (cells, groups, materials, time bins, tally
entries, window bins, pool slots, stacks of split children, input banks, comb
slots) stays inside what it indexes on those workloads, and the results still
equal the oracle's."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

SUITES = [
    "tests/test_gpu_parity.py",
    "tests/test_gpu_edge_cases.py",
    "tests/test_gpu_estimators.py",
    "tests/test_gpu_combined.py",
    "tests/test_gpu_population_control.py",
    "tests/test_gpu_net_windows.py",
    "tests/test_gpu_faults.py",
]


def _checked_env():
    from paper_2409_04668_b300 import build as B
    B.build(checked=True)
    env = dict(os.environ)
    env["MCDC_CHECKS"] = "1"
    return env


def test_normal_build_has_no_checks():
    from paper_2409_04668_b300 import mcdc as M
    if M.build_checked():
        pytest.skip("this process loaded the checked build")
    r = M.check_selftest()
    assert r == {"flags": 0, "site": 0, "index": 0, "made": 16}


def test_checked_selftest_records_first_failure_and_skips_access():
    code = ("from paper_2409_04668_b300 import mcdc as M\n"
            "assert M.build_checked()\n"
            "r = M.check_selftest()\n"
            "print(r['flags'], r['site'], r['index'], r['made'])\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=_checked_env(),
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    flags, site, index, made = map(int, out.stdout.split()[-4:])
    assert flags == 4                # ERRBIT_CHECK alone
    assert site == 12                # the self-test's site
    assert 16 <= index <= 31         # one of the lanes past the array's end
    assert made == 16                # every in-range access made, none beyond


def test_parity_suites_pass_through_the_checked_build():
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + SUITES
    out = subprocess.run(cmd, cwd=ROOT, env=_checked_env(), capture_output=True, text=True,
                         timeout=1800)
    tail = (out.stdout + out.stderr)[-4000:]
    assert out.returncode == 0, tail
    assert " passed" in tail and "failed" not in tail, tail
