"""The device generator (the tracker's own Philox4x32-10 routine with its
precomputed round keys, through mcdc_philox) against three things outside
it: the published known-answer vectors (Salmon et al., SC'11), cuRAND's
device Philox4x32-10 on a million random counters and keys (an independent
implementation; compiled here from tests/curand_philox_ref.cu), and the
oracle's generator.  Key = (seed low, seed high), counter words as given."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def mcdc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2409_04668_b300 import build
    build.build()
    from paper_2409_04668_b300 import mcdc as M
    return M


def _kat():
    rows = []
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            w = [int(v, 16) for v in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answers(mcdc):
    for ctr, key, expect in _kat():
        got = mcdc.philox(key[0] | (key[1] << 32), np.array([ctr], np.uint32))
        assert [int(v) for v in got[0]] == expect


@pytest.fixture(scope="module")
def curand_ref(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox_ref.so")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "curand_philox_ref.cu")], check=True)
    lib = C.CDLL(out)
    lib.curand_philox_ref.restype = C.c_int
    lib.curand_philox_ref.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    return lib


def test_matches_curand(mcdc, curand_ref):
    rng = np.random.default_rng(2409)
    n = 1 << 17
    for s in range(8):
        seed = int(rng.integers(0, 2**64, dtype=np.uint64))
        if s == 0:
            seed = 0xFFFFFFFFFFFFFFFF
        ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
        ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0xFFFFFFFF, 0, 0, 1]]
        key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32), (n, 1))
        ref = np.zeros_like(ctr)
        assert curand_ref.curand_philox_ref(ctr.ctypes.data, key.ctypes.data, n,
                                            ref.ctypes.data) == 0
        got = mcdc.philox(seed, ctr)
        bad = np.nonzero((got != ref).any(axis=1))[0]
        assert bad.size == 0, (hex(seed), bad[:5], got[bad[:2]], ref[bad[:2]])


def test_matches_oracle(mcdc):
    rng = np.random.default_rng(7)
    seed = 0x0123456789ABCDEF
    ctr = rng.integers(0, 2**32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    got = mcdc.philox(seed, ctr)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for q in range(ctr.shape[0]):
        assert [int(v) for v in got[q]] == [int(v) for v in O.philox(ctr[q], key)]


def test_device_buffers_and_refusals(mcdc):
    import torch
    ctr = torch.arange(64, dtype=torch.int32, device="cuda").reshape(16, 4)
    out = torch.zeros_like(ctr)
    mcdc.check(mcdc.mcdc_philox(5, ctr.data_ptr(), 16, out.data_ptr()))
    host = mcdc.philox(5, ctr.cpu().numpy().astype(np.uint32))
    assert np.array_equal(out.cpu().numpy().astype(np.uint32), host)
    with pytest.raises(mcdc.MCDCError):
        mcdc.check(mcdc.mcdc_philox(5, None, 4, None))
    assert mcdc.mcdc_philox(5, None, 0, None) == mcdc.MCDC_OK


def test_uniformity_of_1e8_draws(mcdc):
    """Chi-square of 1.3e8 words (2^25 blocks with the transport's counter
    layout: event counter 0..7, serial 0, history ids 0..2^22 - 1) over 1024
    equal cells of the top 10 bits, and of consecutive word pairs over 32 x 32
    cells: both must look uniform (p > 1e-4 against the chi-square law)."""
    from scipy import stats
    seed = 20240904
    n_hist = 1 << 22
    cells = np.zeros(1024, np.int64)
    pairs = np.zeros(1024, np.int64)
    words = 0
    for c in range(8):
        ctr = np.zeros((n_hist, 4), np.uint32)
        ctr[:, 0] = c
        ctr[:, 2] = np.arange(n_hist, dtype=np.uint32)
        out = mcdc.philox(seed, ctr)
        w = out.reshape(-1)
        cells += np.bincount(w >> 22, minlength=1024)
        pairs += np.bincount(((w[0::2] >> 27) << 5) | (w[1::2] >> 27), minlength=1024)
        words += w.size
    for name, h in (("cells", cells), ("pairs", pairs)):
        e = h.sum() / h.size
        chi2 = float(((h - e) ** 2 / e).sum())
        p = float(stats.chi2.sf(chi2, h.size - 1))
        print(name, words, "chi2", chi2, "p", p)
        assert 1e-4 < p, (name, chi2, p)
