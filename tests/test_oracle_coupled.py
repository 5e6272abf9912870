"""Pins of the oracle's coupled step: the predictor-corrector of App. A.3
(eq:scheme) with the two gas models.

Each test compares the oracle with something it does not compute itself: the
paper's dispersion relation of the Bell instability (eq:belldisp1, and its
printed special cases eq:disp_mu and the CR-Hall limit of App. B.2), the
exact solution of a linear ODE under the midpoint rule, the eigenvalue of a
centred difference on a Fourier mode, the closed-form rotation of a cold CR
beam against the gas in a uniform field, and exact conservation.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl

LINEAR_X = 1
SOURCES = 0


def _state(box, v=None):
    x = np.ascontiguousarray(wl.absolute_positions(box).astype(np.float64))
    vv = np.ascontiguousarray((box.p if v is None else v).astype(np.float64))
    return orc.State(box, x, vv)


def bell_omega(eps, Lam, k=2.0 * math.pi):
    """omega of the unstable mode from the paper's eq:belldisp1 (App. C), for
    the box of wl.bell_linear: wavenumber k, J = 2 f1 k, U_s = v_A/eps,
    R = Lambda eps (0 without the CR-Hall term), v_A = B0 = 1."""
    f1 = 1.0 + 0.25 * Lam * Lam
    J = 2.0 * f1 * k
    U = 1.0 / eps
    R = Lam * eps
    f = 1.0 - R + 0.25 * Lam * Lam
    g = (1.0 - R) * (1.0 - 0.5 * R)
    Ut = U * (1.0 - 0.5 * R)
    # omega~^2 - f k^2 = -g k J (1 - omega~/(k Ut)), omega~ = omega - (Lambda/2) k
    a = g * J / Ut
    c = g * k * J - f * k * k
    wt = 0.5 * a + np.sqrt(complex(0.25 * a * a - c))
    return wt + 0.5 * Lam * k


def test_dispersion_helper_reduces_to_the_papers_special_cases():
    # eq:disp_mu: omega = k0 v_A (eps + i sqrt(1 - eps^2)) without the Hall term
    for eps in (0.1, 0.5, 0.9):
        w = bell_omega(eps, 0.0)
        k0 = 2.0 * math.pi
        assert abs(w - k0 * complex(eps, math.sqrt(1.0 - eps * eps))) < 1e-12 * k0
    # CR-Hall limit (R, eps -> 0): omega = k_m v_A (Lambda/2 + i sqrt(f)), f = 1 + (Lambda/2)^2
    for Lam in (0.2, 1.0, 4.0):
        w = bell_omega(1e-7, Lam)
        km = 2.0 * math.pi
        f = 1.0 + 0.25 * Lam * Lam
        assert abs(w - km * complex(0.5 * Lam, math.sqrt(f))) < 1e-5 * km


def _bell_run(eps, Lam, efolds=3.0):
    box = wl.bell_linear(eps=eps, Lambda=Lam)
    st = _state(box)
    w = bell_omega(eps, Lam)
    nsteps = int(efolds / (w.imag * box.dt))
    nx, ny = box.n[0], box.n[1]
    xc = (np.arange(nx) + 0.5) / nx
    e = np.exp(-2j * math.pi * xc)
    amps = []
    t0 = st.totals()
    for s in range(nsteps + 1):
        psi = (st.B[1] + 1j * st.B[2]).reshape(ny, nx).mean(axis=0)
        amps.append((psi * e).mean())
        if s < nsteps:
            st.coupled_step(box.dt, LINEAR_X)
    amps = np.array(amps)
    t = np.arange(nsteps + 1) * box.dt
    h = len(t) // 3
    growth = np.polyfit(t[h:], np.log(np.abs(amps[h:])), 1)[0]
    omega_r = -np.polyfit(t[h:], np.unwrap(np.angle(amps))[h:], 1)[0]
    return w, growth, omega_r, t0, st.totals()


@pytest.mark.parametrize("eps,Lam", [(0.5, 0.0), (0.1, 0.0), (0.9, 0.0), (0.05, 1.0), (0.05, 4.0)])
def test_bell_linear_growth_matches_the_dispersion_relation(eps, Lam):
    """App. B.2: the eigenvector of the most unstable mode grows and drifts as
    the linear theory says; the paper's code is within 2% at ~32 cells per
    wavelength, and so is this scheme."""
    w, growth, omega_r, t0, t1 = _bell_run(eps, Lam)
    assert abs(growth / w.imag - 1.0) < 0.02
    assert abs(omega_r / w.real - 1.0) < 0.02
    # total (gas + CR) momentum exactly conserved: the centred fluxes telescope
    scale = abs(t0[4])
    assert np.abs((t1[:3] + t1[4:7]) - (t0[:3] + t0[4:7])).max() < 1e-13 * scale


def test_alfven_wave_is_the_midpoint_rule_solution():
    """Without CRs the coupled step of model 1 is the midpoint rule on the
    centred-difference wave system: a Fourier mode with eigenvalues
    +-i B_x sin(k dx)/dx multiplies by G = 1 + z + z^2/2, z = +-i w dt, per step."""
    box = wl.bell_linear(eps=0.5, amp=0.0, nx=32, ny=2)
    box.m_cr = 0.0
    nx, ny, nc = box.n[0], box.n[1], box.ncell
    dx = box.dx[0]
    k = 2.0 * math.pi * 3   # third harmonic of the box
    xc = (np.arange(nx) + 0.5) * dx
    a, b = 1e-3, 4e-4
    by0 = np.tile(a * np.cos(k * xc), ny)
    vy0 = np.tile(b * np.sin(k * xc), ny)
    box.B[1] = by0
    box.mom[1] = vy0
    st = _state(box)
    dt = 0.3 * dx
    nsteps = 50
    for _ in range(nsteps):
        st.coupled_step(dt, LINEAR_X)
    wd = math.sin(k * dx) / dx
    # characteristic variables s_pm = v_y +- b_y (B_x = rho = 1) obey ds/dt = +-D s
    Gp = (1.0 + 1j * wd * dt - 0.5 * (wd * dt) ** 2) ** nsteps   # D e^{ikx} = i wd e^{ikx}
    Gm = (1.0 - 1j * wd * dt - 0.5 * (wd * dt) ** 2) ** nsteps
    # s_pm(0) = b sin(kx) +- a cos(kx) = Re[c_pm e^{ikx}]
    cp = a - 1j * b
    cm = -a - 1j * b
    ph = np.exp(1j * k * xc)
    sp = np.real(cp * Gp * ph)
    sm = np.real(cm * Gm * ph)
    vy = np.tile(0.5 * (sp + sm), ny)
    by = np.tile(0.5 * (sp - sm), ny)
    assert np.abs(st.mom[1] - vy).max() < 1e-15 + 1e-12 * a
    assert np.abs(st.B[1] - by).max() < 1e-15 + 1e-12 * a
    # the z components and B_x never move
    assert np.abs(st.B[2]).max() == 0.0 and np.abs(st.mom[2]).max() == 0.0
    assert np.all(st.B[0] == 1.0)


def test_hall_induction_is_the_curl_of_F_over_ng():
    """dB/dt gains curl(F/n_g) (from -curl E with E = E0 - F/n_g, eq:emfcr2):
    in 1-D, dB_y/dt = -dH_z/dx and dB_z/dt = dH_y/dx; on a Fourier mode the
    centred difference is i sin(k dx)/dx."""
    nx, ny = 16, 3
    g = orc.make_grid(2, (nx, ny, 1), dx=(0.25, 0.25, 1.0))
    nc = nx * ny
    rho = np.ones(nc)
    mom = np.zeros((3, nc))
    B = np.zeros((3, nc))
    B[0] = 1.0
    dx = 0.25
    k = 2.0 * math.pi * 2 / (nx * dx)
    xc = (np.arange(nx) + 0.5) * dx
    H = np.zeros((3, nc))
    H[1] = np.tile(np.cos(k * xc), ny)
    H[2] = np.tile(np.sin(k * xc), ny)
    dmom, dB = orc.gas_rhs(g, LINEAR_X, rho, mom, B, H)
    kd = math.sin(k * dx) / dx
    # d/dx cos = -kd sin, d/dx sin = kd cos (centred difference of the modes)
    np.testing.assert_allclose(dB[1], -np.tile(kd * np.cos(k * xc), ny), atol=1e-12)
    np.testing.assert_allclose(dB[2], np.tile(-kd * np.sin(k * xc), ny), atol=1e-12)
    assert np.abs(dmom).max() == 0.0 and np.abs(dB[0]).max() == 0.0
    # model 0 evolves nothing but the CR sources
    dmom0, dB0 = orc.gas_rhs(g, SOURCES, rho, mom, B, H)
    assert np.abs(dmom0).max() == 0.0 and np.abs(dB0).max() == 0.0


def _two_fluid(hall, Om_dt, nsteps, ratio=0.3):
    """A cold CR beam moving at v_y = 1 through gas at rest in B = x_hat
    (uniform: one particle per cell at the centre); returns the rotation angle
    of W = U_CR - v_g, |W|, the centre-of-mass velocity and the expected
    rotation rate."""
    box = wl.bell_linear(eps=0.5, amp=0.0, nx=8, ny=8)
    box.C = 1e4
    box.qm_cr = 1.0
    box.qm_gas = 1.0
    box.hall = hall
    dV = box.dx[0] * box.dx[1]
    box.m_cr = ratio * dV     # rho_CR = ratio * rho_gas
    v = np.zeros((3, box.np))
    v[1] = 1.0
    st = _state(box, v)
    n = st.mom_dep[0].mean()
    R = n / (box.qm_gas + n) if hall else 0.0
    # dW/dt = (1-R)(q/mc)(1 + rho_CR/rho_g) W x B for NR cold fluids, with or
    # without the CR-Hall term (R = 0 without it)
    Om = (1.0 - R) * box.qm_cr * (1.0 + ratio)
    dt = Om_dt / Om
    for _ in range(nsteps):
        st.coupled_step(dt, SOURCES)
    gam = np.sqrt(1.0 + (st.v ** 2).sum(axis=0) / box.C ** 2)
    U = (st.v / gam).mean(axis=1)
    vg = st.mom.mean(axis=1) / st.rho.mean()
    W = U - vg
    ang = math.atan2(W[2], W[1])
    expect = math.remainder(-nsteps * Om_dt, 2.0 * math.pi)
    vcm = (vg + ratio * U) / (1.0 + ratio)
    return ang, expect, np.linalg.norm(W), vcm, st


@pytest.mark.parametrize("hall", [0, 1])
def test_cold_beam_rotates_against_the_gas_at_the_two_fluid_rate(hall):
    """Model 0 (uniform gas, CR sources only): the relative velocity of a cold
    beam and the gas rotates about B at (1-R)(q/mc)(1 + rho_CR/rho_g)|B|, to
    second order in dt; the centre-of-mass velocity is unchanged."""
    a1, e1, wn1, vcm1, st = _two_fluid(hall, 0.02, 400)
    a2, e2, wn2, _, _ = _two_fluid(hall, 0.01, 800)
    err1 = abs(math.remainder(a1 - e1, 2 * math.pi))
    err2 = abs(math.remainder(a2 - e2, 2 * math.pi))
    assert err1 < 2e-4
    assert 3.0 < err1 / err2 < 5.0                       # second order
    np.testing.assert_allclose(vcm1, [0.0, 0.3 / 1.3, 0.0], atol=1e-8)
    if not hall:
        assert abs(wn1 - 1.0) < 1e-5
    else:
        # the push's CR-Hall field uses F_CR of the moments at x^n (the
        # predictor's feedback, App. A.3): the relative speed decays at first
        # order in dt, by about half as much at half the step
        assert 0.4 < (1.0 - wn2) / (1.0 - wn1) < 0.6


def test_coupled_step_conserves_gas_plus_cr_energy_and_momentum():
    box = wl.bell_linear(eps=0.3, Lambda=2.0, amp=0.05)
    st = _state(box)
    t0 = st.totals()
    for _ in range(20):
        st.coupled_step(box.dt, LINEAR_X)
    t1 = st.totals()
    scale = abs(t0[4]) + abs(t0[7]) + abs(t0[3])
    assert np.abs((t1[:3] + t1[4:7]) - (t0[:3] + t0[4:7])).max() < 1e-13 * scale
    assert abs((t1[3] + t1[7]) - (t0[3] + t0[7])) < 1e-13 * scale


@pytest.mark.parametrize("hall", [0, 1])
def test_predictor_sources_obey_newtons_third_law_and_eq_eng(hall):
    """The predictor's gas sources are minus the force and power the CRs take
    from the field they see: with E the cell field of the staging routine
    (E0 - F/n_g with the CR-Hall term, eq:emfcr2), the momentum source is
    -(n E + J x B) (eq:lorentz2 rewritten) and the energy source -J.E
    (eq:eng).  Model 0, so only the sources act."""
    box = wl.periodic_thermal_2d(nx=12, ny=10, ppc=6, dv_amp=0.4, seed=11)
    rng = np.random.default_rng(5)
    box.B = np.ascontiguousarray(box.B + 0.3 * rng.standard_normal(box.B.shape))
    box.hall = hall
    box.qm_gas = 0.7
    box.m_cr = 0.05
    st = _state(box)
    dt = 0.01
    half, _ = st.predict(dt, SOURCES)
    E = orc.field_prep(st.g, st.p, st.rho, st.mom, st.B, st.mom_dep)
    n = st.mom_dep[0]
    J = st.mom_dep[1:4]
    F = n * E + np.cross(J.T, st.B.T).T
    np.testing.assert_allclose((st.mom - half[1]) / (0.5 * dt), F, rtol=1e-9, atol=1e-9 * np.abs(F).max())
    P = (J * E).sum(axis=0)
    np.testing.assert_allclose((st.egas - half[2]) / (0.5 * dt), P, rtol=1e-9, atol=1e-9 * np.abs(P).max())
    assert np.array_equal(half[3], st.B) and np.array_equal(half[0], st.rho)
