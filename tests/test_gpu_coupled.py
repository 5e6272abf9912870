"""The coupled MHD-PIC step on the GPU (App. A.3, eq:scheme) against the FP64
oracle, and the Bell linear test (App. B.2) run through the C ABI.

Tolerances: the gas kernels compute in FP64 in both precisions; the FP64 path
matches the oracle to 1e-12 relative, the mixed path to 1e-5 relative L2 (its
particle deposits are FP32 with fixed-point sums).  The Bell growth rate and
drift are held to the paper's 2% against the dispersion relation.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl
from tests._parity import rel_l2, sorted_oracle_state, tilt_B
from tests.test_oracle_coupled import bell_omega

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402

MIXED, FP64 = m.MHDPIC_PREC_MIXED, m.MHDPIC_PREC_FP64
SOURCES, LINEAR_X = m.MHDPIC_GAS_SOURCES, m.MHDPIC_GAS_LINEAR_X
TOL = {FP64: 1e-12, MIXED: 1e-5}


def _boxes():
    def thermal():
        b = tilt_B(wl.periodic_thermal_2d(nx=29, ny=21, ppc=9, dv_amp=0.4, seed=21), 21)
        b.hall = 1
        b.m_cr = 0.03
        return b

    def bell_hall():
        b = wl.bell_linear(eps=0.2, Lambda=2.0, amp=0.05, nx=32, ny=8, ppc=3)
        return b

    return {"thermal_hall": thermal, "bell_linear_hall": bell_hall}


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("model", [SOURCES, LINEAR_X])
@pytest.mark.parametrize("name", list(_boxes()))
def test_coupled_step_matches_oracle(prec, model, name):
    box = _boxes()[name]()
    eng = m.Engine([box], precision=prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    tol = TOL[prec]
    dt = box.dt
    mom0, eg0, B0 = st.mom.copy(), st.egas.copy(), st.B.copy()
    # predictor: staged half-step fields
    half, E = st.predict(dt, model)
    eng.gas_predict(dt, model)
    f = eng.fields().cpu().numpy()
    scale = np.linalg.norm(box.B)
    for q in range(3):
        assert rel_l2(f[q], E[q], floor=1e-3 * scale) < (1e-12 if prec == FP64 else 1e-6), ("E", q)
        assert rel_l2(f[3 + q], half[3][q], floor=1e-3 * scale) < (1e-12 if prec == FP64 else 1e-6), ("B", q)
    # push in the half-step fields
    st.mom_dep[:] = 0.0
    orc.push(st.g, st.p, dt, st.x, st.v, E, half[3], st.corr, st.mom_dep)
    eng.interp_push(dt, 1)
    gc = eng.deposits(0).cpu().numpy()
    for q in range(4):
        assert rel_l2(gc[q], st.corr[q]) < tol, ("corrector", q)
    # corrector: the gas changes
    st.correct(dt, model, half)
    eng.gas_correct(dt, model)
    gm = eng.mom.cpu().numpy()
    ge = eng.egas.cpu().numpy()
    gB = eng.B.cpu().numpy()
    for q in range(3):
        assert rel_l2(gm[q] - mom0[q], st.mom[q] - mom0[q], floor=1e-9 * np.linalg.norm(mom0) + 1e-300) < tol, q
        assert rel_l2(gB[q] - B0[q], st.B[q] - B0[q], floor=1e-9 * scale) < tol, ("B", q)
    assert rel_l2(ge - eg0, st.egas - eg0, floor=1e-300) < tol
    # the accumulators are cleared
    assert np.abs(eng.deposits(0).cpu().numpy()).max() == 0.0
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("eps,Lam", [(0.5, 0.0), (0.05, 4.0)])
def test_bell_linear_growth_on_the_gpu(prec, eps, Lam):
    """App. B.2 through the C ABI: the most unstable mode grows and drifts as
    eq:belldisp1 says, within the paper's 2%."""
    box = wl.bell_linear(eps=eps, Lambda=Lam)
    eng = m.Engine([box], precision=prec)
    w = bell_omega(eps, Lam)
    nsteps = int(3.0 / (w.imag * box.dt))
    nx, ny = box.n[0], box.n[1]
    xc = (np.arange(nx) + 0.5) / nx
    e = np.exp(-2j * math.pi * xc)
    amps = []
    t0 = None
    for s in range(nsteps + 1):
        if s % 4 == 0 or s == nsteps:
            B = eng.B.cpu().numpy()
            psi = (B[1] + 1j * B[2]).reshape(ny, nx).mean(axis=0)
            amps.append((s * box.dt, (psi * e).mean()))
        if s < nsteps:
            tot = eng.coupled_step(box.dt, LINEAR_X, totals=(s == 0 or s == nsteps - 1))
            if s == 0:
                t0 = tot[0]
    t1 = tot[0]
    t = np.array([a[0] for a in amps])
    a = np.array([a[1] for a in amps])
    h = len(t) // 3
    growth = np.polyfit(t[h:], np.log(np.abs(a[h:])), 1)[0]
    omega_r = -np.polyfit(t[h:], np.unwrap(np.angle(a))[h:], 1)[0]
    assert abs(growth / w.imag - 1.0) < 0.02, growth
    assert abs(omega_r / w.real - 1.0) < 0.02, omega_r
    # gas + CR momentum conserved (FP64 totals of the fixed-point deposits)
    drift = np.abs((t1[:3] + t1[4:7]) - (t0[:3] + t0[4:7])).max() / abs(t0[4])
    assert drift < (1e-12 if prec == FP64 else 1e-6), drift
    assert eng.status() == 0
    eng.close()


def test_coupled_calls_are_checked():
    box = wl.bell_linear(eps=0.5)
    eng = m.Engine([box], precision=MIXED)
    with pytest.raises(m.MhdpicError):
        eng.gas_correct(box.dt, SOURCES)         # no predictor yet
    with pytest.raises(m.MhdpicError):
        eng.gas_predict(box.dt, 7)               # unknown model
    with pytest.raises(m.MhdpicError):
        eng.gas_predict(-1.0, SOURCES)
    eng.gas_predict(box.dt, LINEAR_X)
    eng.interp_push(box.dt, 1)
    with pytest.raises(m.MhdpicError):
        eng.gas_correct(2.0 * box.dt, LINEAR_X)  # not the predictor's dt
    eng.gas_correct(box.dt, LINEAR_X)
    eng.close()
    shock = wl.shock_2d(nx=64, ny=8, ppc=4.0, seed=1)   # reflecting x walls
    eng = m.Engine([shock], precision=MIXED)
    with pytest.raises(m.MhdpicError):
        eng.gas_predict(shock.dt, LINEAR_X)
    eng.gas_predict(shock.dt, SOURCES)
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_plain_push_after_the_corrector_stages_the_corrected_gas(prec):
    """A coupled step, then a plain step (push + feedback) without a new
    predictor: the push stages the fields of the corrected gas itself (as the
    feedback call would) and sizes its corrector scale for them, so no
    overflow is flagged and the step matches the oracle's push in the fields
    of the corrected gas."""
    box = _boxes()["thermal_hall"]()
    eng = m.Engine([box], precision=prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    dt = box.dt
    st.coupled_step(dt, SOURCES)
    eng.coupled_step(dt, SOURCES)
    # the plain step: fields of the corrected gas and the moments of x^(n+1)
    corr, md = st.push_only(dt)
    corr_ref = corr.copy()
    orc.apply_feedback(st.g, st.mom, st.egas, corr)   # zeroes corr
    eng.interp_push(dt, 1)
    gc = eng.deposits(0).cpu().numpy()
    eng.apply_feedback()
    tol = TOL[prec]
    for q in range(4):
        assert rel_l2(gc[q], corr_ref[q]) < tol, ("corrector", q)
    gm = eng.mom.cpu().numpy()
    for q in range(3):
        assert rel_l2(gm[q] - box.mom[q], st.mom[q] - box.mom[q], floor=1e-300) < tol * 10, q
    assert eng.status() == 0, m.status_names(eng.status())
    eng.close()
