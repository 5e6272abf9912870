"""The oracle's Philox4x32-10 (the injection's random numbers, Section 5)
against an independent implementation: CUDA's curand device API, called from
a small probe kernel compiled here (tests/probes/curand_philox.cu).

The paper fixes no generator; the library and the oracle both implement
Philox4x32-10 (Salmon et al. 2011) from its published definition, with the
counter (k, call, 0, 0) and the 64-bit seed as the key (low word first).  The
statistical pins of the oracle cannot tell a wrong round constant or
multiplier from the right one; a word-for-word match with curand can.
curand's curand_Philox4x32_10(ctr, key) takes the same 4-word counter and
2-word key, in the same word order, so no mapping is needed.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as orc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("probe") / "libcurand_philox.so")
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "probes", "curand_philox.cu"), "-o", so], check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    lib.curand_philox_words.restype = ctypes.c_int
    lib.curand_philox_words.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    return lib


def _cases():
    rng = np.random.default_rng(20261203)
    ctr, key = [], []
    # edge words
    for c in ([0, 0, 0, 0], [0xffffffff] * 4, [1, 0, 0, 0], [0, 0, 0, 1]):
        for k in ([0, 0], [0xffffffff, 0xffffffff], [1, 0]):
            ctr.append(c)
            key.append(k)
    # the injection's counters (particle k, call number, 0, 0) under 64-bit seeds
    for seed in (0, 11, 0x0123456789abcdef, (1 << 64) - 1):
        for call in (0, 1, 7, 1000):
            for k in (0, 1, 2, 31, 1 << 20):
                ctr.append([k, call, 0, 0])
                key.append([seed & 0xffffffff, seed >> 32])
    # random words
    ctr += rng.integers(0, 1 << 32, (256, 4), dtype=np.uint64).tolist()
    key += rng.integers(0, 1 << 32, (256, 2), dtype=np.uint64).tolist()
    return np.array(ctr, dtype=np.uint32), np.array(key, dtype=np.uint32)


def test_oracle_philox_equals_curand_word_for_word(probe):
    ctr, key = _cases()
    n = ctr.shape[0]
    # the probe's grid covers ceil(n/128) blocks of 128 threads and guards i < n
    d_ctr = torch.from_numpy(ctr.view(np.int32).copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int32).copy()).cuda()
    d_out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    assert d_ctr.shape == (n, 4) and d_key.shape == (n, 2)
    stream = torch.cuda.current_stream()
    rc = probe.curand_philox_words(d_ctr.data_ptr(), d_key.data_ptr(), d_out.data_ptr(), n,
                                   ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint32)
    want = np.stack([orc.philox(ctr[i], key[i]) for i in range(n)])
    bad = np.flatnonzero((got != want).any(axis=1))
    assert bad.size == 0, (bad[:5], ctr[bad[:5]], key[bad[:5]], got[bad[:5]], want[bad[:5]])
