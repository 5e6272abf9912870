"""The allocation-free charge/current deposit (mhdpic_deposit_moments_noalloc).

It is meant for callers that must not allocate device memory once running (a
fixed device-memory budget, allocation-free time-step loops, or call sites
that cannot accept the device synchronisation of cudaMalloc/cudaFree).  Its
result must equal both the oracle's deposit of the same particles and the
context-based deposit (mhdpic_deposit, read back with mhdpic_get_deposits)
within the tolerance the parity tests use, on two calls in a row through the
shared scratch array.
"""
import ctypes

import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl
from tests._parity import momenta_of, positions_of, rel_l2, tilt_B

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
        m.mhdpic_deposit_moments_noalloc(g, p, prec, box.np, pos=eng.pos.data_ptr(), vel=eng.vel.data_ptr(),
                                         out=out.data_ptr(), stream=stream)
    else:
        m.mhdpic_deposit_moments_noalloc(g, p, prec, box.np, x=eng.x.data_ptr(), p64=eng.p64.data_ptr(),
                                         out=out.data_ptr(), stream=stream)
    torch.cuda.synchronize()


CASES = ["mixed2d", "fp64_3d", "mixed2d_reflect", "mixed2d_open", "fp64_2d_open"]


def _case(case):
    M, F = m.MHDPIC_PREC_MIXED, m.MHDPIC_PREC_FP64
    if case == "mixed2d":
        return tilt_B(wl.periodic_thermal_2d(nx=29, ny=21, ppc=9, dv_amp=0.4, seed=31), 31), M
    if case == "fp64_3d":
        return wl.alfvenic_beam_3d(n=14, ppc=6, nmodes=8, seed=32), F
    if case == "mixed2d_reflect":
        return tilt_B(wl.shock_2d(nx=96, ny=10, ppc=8.0, seed=33), 33, amp=0.1), M
    # the open inflow face of the shock box: free slots (cell -1 / x NaN) deposit nothing
    box = wl.shock_front_2d(nx=96, ny=10, ppc=8.0, front=0.25, seed=35)
    return tilt_B(box, 35, amp=0.1), (M if case == "mixed2d_open" else F)


@pytest.mark.parametrize("case", CASES)
def test_noalloc_deposit_equals_oracle_and_context_deposit_on_two_calls(case):
    box, prec = _case(case)
    eng = m.Engine([box], precision=prec)
    ref = eng.deposits(1).cpu().numpy()          # moments of the current positions
    # the oracle's deposit of the same particles (free slots have x NaN there)
    x, v = positions_of(eng), momenta_of(eng)
    if prec == m.MHDPIC_PREC_MIXED:
        x[:, eng.cell.cpu().numpy() < 0] = np.nan
    want = orc.deposit_moments(orc.grid_of(box), orc.params_of(box), x, v, box.ncell)
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
            assert rel_l2(o[q], want[q]) < tol, (case, q, rel_l2(o[q], want[q]))
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
    # sides whose product would wrap around in 64 bits are rejected side by side
    g.n[0], g.n[1] = 1 << 21, 1 << 21
    with pytest.raises(m.MhdpicError, match="allocation-free limit"):
        m.mhdpic_deposit_moments_noalloc(g, p, m.MHDPIC_PREC_MIXED, 0, out=out.data_ptr())
    g3, p3 = _structs(wl.alfvenic_beam_3d(n=6, ppc=1, nmodes=2, seed=36))
    g3.n[0], g3.n[1], g3.n[2] = 1 << 21, 1 << 21, 1 << 22
    with pytest.raises(m.MhdpicError, match="allocation-free limit"):
        m.mhdpic_deposit_moments_noalloc(g3, p3, m.MHDPIC_PREC_MIXED, 0, out=out.data_ptr())
