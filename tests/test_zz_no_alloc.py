"""The allocation-free charge/current deposit (mhdpic_deposit_moments_noalloc).

It is meant for callers that must not allocate device memory once running (a
fixed device-memory budget, allocation-free time-step loops, or call sites
that cannot accept the device synchronisation of cudaMalloc/cudaFree).  Its
result must equal that of the context-based deposit (mhdpic_deposit, read
back with mhdpic_get_deposits) within the tolerance the parity tests use, on
two calls in a row through the shared scratch array.
"""
import ctypes

import numpy as np
import pytest

from paper_1412_1087_gb300 import workloads as wl
from tests._parity import rel_l2, tilt_B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402


def _structs(box):
    g = m.Grid()
    g.ndim = box.ndim
    for d in range(3):
        g.n[d], g.dx[d], g.x0[d], g.bc[d] = box.n[d], box.dx[d], box.x0[d], box.bc[d]
    p = m.Params()
    p.qm_cr, p.qm_gas, p.C, p.m_cr, p.hall, p.shape = box.qm_cr, box.qm_gas, box.C, box.m_cr, box.hall, m.MHDPIC_SHAPE_TSC
    return g, p


def _call(eng, box, prec, out):
    g, p = _structs(box)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if prec == m.MHDPIC_PREC_MIXED:
        m.mhdpic_deposit_moments_noalloc(g, p, prec, box.np, cell=eng.cell.data_ptr(), off=eng.off.data_ptr(),
                                         p=eng.p.data_ptr(), out=out.data_ptr(), stream=stream)
    else:
        m.mhdpic_deposit_moments_noalloc(g, p, prec, box.np, x=eng.x.data_ptr(), p64=eng.p64.data_ptr(),
                                         out=out.data_ptr(), stream=stream)
    torch.cuda.synchronize()


@pytest.mark.parametrize("case", ["mixed2d", "fp64_3d", "mixed3d_reflect"])
def test_noalloc_deposit_equals_context_deposit_on_two_calls(case):
    if case == "mixed2d":
        box, prec = tilt_B(wl.periodic_thermal_2d(nx=29, ny=21, ppc=9, dv_amp=0.4, seed=31), 31), m.MHDPIC_PREC_MIXED
    elif case == "fp64_3d":
        box, prec = wl.alfvenic_beam_3d(n=14, ppc=6, nmodes=8, seed=32), m.MHDPIC_PREC_FP64
    else:
        box, prec = tilt_B(wl.shock_2d(nx=96, ny=10, ppc=8.0, seed=33), 33, amp=0.1), m.MHDPIC_PREC_MIXED
    eng = m.Engine([box], precision=prec)
    ref = eng.deposits(1).cpu().numpy()          # moments of the current positions
    outs = []
    for _ in range(2):
        out = torch.full((4, box.ncell), float("nan"), dtype=torch.float64, device="cuda")
        _call(eng, box, prec, out)
        outs.append(out.cpu().numpy())
    # the context deposits mixed-precision moments as the push does (f32
    # weights), the allocation-free call in double: the parity tolerance of
    # each precision
    tol = 1e-5 if prec == m.MHDPIC_PREC_MIXED else 1e-12
    for o in outs:
        for q in range(4):
            assert rel_l2(o[q], ref[q]) < tol, (case, q, rel_l2(o[q], ref[q]))
    # the second call starts from a cleared scratch: identical to the first
    assert np.array_equal(outs[0], outs[1])
    eng.close()


def test_noalloc_rejects_grids_beyond_its_limit():
    box = wl.periodic_thermal_2d(nx=16, ny=16, ppc=1, seed=34)
    g, p = _structs(box)
    g.n[0] = 1024
    g.n[1] = 1024                                  # 2^20 cells > the 2^18 limit
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MhdpicError, match="allocation-free limit"):
        m.mhdpic_deposit_moments_noalloc(g, p, m.MHDPIC_PREC_MIXED, 0, out=out.data_ptr())
