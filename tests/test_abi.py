"""The C-ABI library loads and exports every symbol include/mhdpic.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mhdpic_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_1087_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mhdpic_init", "mhdpic_sort", "mhdpic_interp_push", "mhdpic_deposit",
                     "mhdpic_apply_feedback", "mhdpic_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib):
    from paper_1412_1087_gb300 import mhdpic
    assert set(_declared()) <= set(mhdpic.SIGNATURES)


def test_strerror_and_argument_errors_without_gpu(lib):
    from paper_1412_1087_gb300 import mhdpic as m
    m.load()
    assert m.load().mhdpic_strerror(0) == b"success"
    # invalid arguments are rejected on the host before any CUDA call
    ctx = ctypes.c_void_p()
    rc = m.load().mhdpic_init(ctypes.byref(ctx), 0, None, None, None, None, None, None)
    assert rc == -1 and ctx.value is None
    assert b"nbox" in m.load().mhdpic_last_error()
    g = (m.Grid * 1)()
    p = (m.Params * 1)()
    g[0].ndim = 4
    opt = m.Options()
    parts = m.Particles()
    import numpy as np
    bs = np.zeros(2, dtype=np.int64)
    parts.box_start = bs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    gas = m.Gas(1, 1, 1, 1)
    rc = m.load().mhdpic_init(ctypes.byref(ctx), 1, g, p, ctypes.byref(opt), ctypes.byref(parts),
                              ctypes.byref(gas), None)
    assert rc == -1
    assert b"ndim" in m.load().mhdpic_last_error()
    assert m.load().mhdpic_destroy(None) == 0
    assert m.load().mhdpic_num_keys(None) == -1


def test_no_oracle_on_the_product_path():
    """The library and its binding never load the oracle."""
    pkg = os.path.join(ROOT, "paper_1412_1087_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "liboracle" not in src and "mhdpic_oracle" not in src, fn
