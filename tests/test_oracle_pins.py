"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes an oracle formula: each compares the oracle with a
closed form, an invariant, a hand-expanded value, a value the paper prints, or
an independent library routine (numpy's stable argsort).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _uniform_fields(n, ndim, E=(0.0, 0.0, 0.0), B=(1.0, 0.0, 0.0)):
    nc = int(np.prod(n))
    Ep = np.zeros((3, nc))
    Bp = np.zeros((3, nc))
    for d in range(3):
        Ep[d] = E[d]
        Bp[d] = B[d]
    return Ep, Bp


# ---------------------------------------------------------------------------
# TSC shape (Section 3)
# ---------------------------------------------------------------------------

def test_tsc_weights_hand_expanded():
    for case in _golden("tsc_weights.json")["cases"]:
        i, w = orc.tsc_weights(case["s"])
        assert i == case["cell"]
        np.testing.assert_array_equal(w, np.array(case["weights"]))


def test_tsc_weight_moments():
    """sum w = 1, sum w k = delta, sum w k^2 = delta^2 + 1/4 (quadratic spline)."""
    rng = np.random.default_rng(3)
    k = np.array([-1.0, 0.0, 1.0])
    for s in rng.uniform(-50, 50, 200):
        i, w = orc.tsc_weights(s)
        delta = s - i - 0.5
        assert -0.5 <= delta < 0.5
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs((w * k).sum() - delta) < 1e-15
        assert abs((w * k * k).sum() - (delta * delta + 0.25)) < 1e-15
        assert np.all(w >= 0)


def test_tsc_is_continuous_across_cell_faces():
    """At a cell face the stencils of both neighbouring cells give the same weights."""
    for face in [3.0, 10.0, 0.0]:
        i1, w1 = orc.tsc_weights(face)              # lower corner of cell `face`
        i0, w0 = orc.tsc_weights(np.nextafter(face, -np.inf))
        a = dict(zip([i1 - 1, i1, i1 + 1], w1))
        b = dict(zip([i0 - 1, i0, i0 + 1], w0))
        for key in set(a) | set(b):
            assert abs(a.get(key, 0.0) - b.get(key, 0.0)) < 1e-14


def test_gather_reproduces_linear_field_exactly():
    """A field linear in x, y, z at cell centres is interpolated exactly (first moment)."""
    n = (16, 16, 16)
    g = orc.make_grid(3, n, dx=(0.5, 2.0, 1.0), x0=(1.0, -3.0, 0.25))
    xs = [g.x0[d] + (np.arange(n[d]) + 0.5) * g.dx[d] for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    f = (2.0 + 0.3 * X - 1.7 * Y + 0.9 * Z).reshape(1, -1)
    rng = np.random.default_rng(4)
    for _ in range(50):
        # stay two cells from the periodic seam so no wrapped cell enters
        p = [g.x0[d] + g.dx[d] * rng.uniform(2.0, n[d] - 2.0) for d in range(3)]
        val = orc.gather(g, p, f)[0]
        assert abs(val - (2.0 + 0.3 * p[0] - 1.7 * p[1] + 0.9 * p[2])) < 1e-12


def test_flat_deposit_from_uniform_load():
    """One particle per cell at the same offset gives an exactly uniform density."""
    n = (8, 6, 1)
    g = orc.make_grid(2, n)
    planes = np.zeros((1, 48))
    for j in range(6):
        for i in range(8):
            orc.deposit(g, [i + 0.3, j + 0.8], [1.0], planes)
    np.testing.assert_allclose(planes, 1.0, rtol=0, atol=1e-15)


def test_brute_force_deposit_two_particles_hand_expanded():
    """Two particles on a 5 x 5 periodic grid, weights written out by hand."""
    g = orc.make_grid(2, (5, 5, 1))
    planes = np.zeros((1, 25))
    # particle A at s = (2.75, 2.25): x-weights (1/32, 11/16, 9/32) on cells 1,2,3;
    # y-weights (9/32, 11/16, 1/32) on rows 1,2,3
    orc.deposit(g, [2.75, 2.25], [2.0], planes)
    # particle B at s = (0.5, 4.5): both centred, weights (1/8, 3/4, 1/8); x wraps 4,0,1 and y 3,4,0
    orc.deposit(g, [0.5, 4.5], [1.0], planes)
    exp = np.zeros((5, 5))
    wx = {1: 1 / 32, 2: 11 / 16, 3: 9 / 32}
    wy = {1: 9 / 32, 2: 11 / 16, 3: 1 / 32}
    for jy, a in wy.items():
        for ix, b in wx.items():
            exp[jy, ix] += 2.0 * a * b
    w8 = {-1: 1 / 8, 0: 3 / 4, 1: 1 / 8}
    for dj, a in w8.items():
        for di, b in w8.items():
            exp[(4 + dj) % 5, (0 + di) % 5] += a * b
    np.testing.assert_allclose(planes.reshape(5, 5), exp, rtol=0, atol=1e-15)


def test_reflecting_wall_folds_weight_and_mirrors_particle():
    g = orc.make_grid(2, (6, 4, 1), bc=(1, 0, 0))
    planes = np.zeros((1, 24))
    orc.deposit(g, [0.2, 1.5], [1.0], planes)           # stencil reaches cell -1
    assert abs(planes.sum() - 1.0) < 1e-15
    row = planes.reshape(4, 6)[1]
    # y = 1.5 is a cell centre: row 1 carries 3/4 of the charge.  Along x,
    # cell -1 folds onto cell 0: w(-1) + w(0) = (1/2)(0.8)^2 + 3/4 - 0.09
    assert abs(row[0] - 0.75 * (0.32 + 0.66)) < 1e-15
    assert abs(row[1] - 0.75 * 0.02) < 1e-15
    # the upper wall mirrors it: s = 5.8 puts (0.02, 0.66, 0.32) on cells 4,
    # 5 and 6, and cell 6 folds onto cell 5
    planes[:] = 0.0
    orc.deposit(g, [5.8, 1.5], [1.0], planes)
    row = planes.reshape(4, 6)[1]
    assert abs(row[5] - 0.75 * (0.66 + 0.32)) < 1e-15
    assert abs(row[4] - 0.75 * 0.02) < 1e-15
    assert abs(planes.sum() - 1.0) < 1e-15
    x, v = orc.boundary(g, [-0.25, 1.0], [3.0, 1.0, 2.0])
    assert x[0] == 0.25 and v[0] == -3.0 and v[1] == 1.0
    x, v = orc.boundary(g, [6.5, 1.0], [3.0, 1.0, 2.0])
    assert x[0] == 5.5 and v[0] == -3.0
    x, v = orc.boundary(g, [6.0, 1.0], [3.0, 1.0, 2.0])
    assert x[0] < 6.0 and v[0] == -3.0
    x, v = orc.boundary(g, [1.0, -0.5], [3.0, 1.0, 2.0])  # y periodic
    assert x[1] == 3.5 and v[1] == 1.0


# ---------------------------------------------------------------------------
# Boris push (Appendix A.2) in uniform fields: closed forms
# ---------------------------------------------------------------------------

def _centre_yz(x, v, C, B0=1.0, qm=1.0, wE=0.0):
    """Guiding centre in the y-z plane for B along +x: c = z - i (w - w_E)/Omega."""
    gam = math.sqrt(1.0 + (v @ v) / (C * C))
    om = qm * B0 / gam
    w = complex(v[1], v[2]) / gam
    return complex(x[1], x[2]) - 1j * (w - wE) / om, om


@pytest.mark.parametrize("rel", [False, True])
def test_gyration_pure_B_exact_orbit(rel):
    """Appendix B.1 with v0 = 0: circle of radius R_L about a fixed centre, |v|
    conserved exactly, phase advancing by 2 atan(Omega dt / 2) per step, for a
    random variable dt as in the paper."""
    gp = _golden("gyration_appB1.json")["relativistic" if rel else "nonrelativistic"]
    b = wl.gyration(relativistic=rel)
    g, p = orc.grid_of(b), orc.params_of(b)
    x = wl.absolute_positions(b)
    v = b.p.astype(np.float64)
    E, B = _uniform_fields(b.n, 3)
    C = b.C
    c0, om = _centre_yz(x[:, 0], v[:, 0], C)
    gam1 = math.sqrt(C * C + gp["v_perp"] ** 2) / C
    assert abs(om - gp["qm"] * gp["B0"] / gam1) < 1e-15
    if rel:
        assert abs(gam1 - gp["gamma_1_approx"]) < 0.06
        assert abs(om - gp["Omega_L_approx"]) < 0.001
    else:
        # the paper rounds: gamma_1 = sqrt(101)/10 at v_perp = 0.1 C
        assert abs(om - gp["Omega_L"]) < 0.006
    RL = gp["v_perp"] / (gp["qm"] * gp["B0"])
    assert RL == gp["R_L"]
    assert abs(abs(complex(x[1, 0], x[2, 0]) - c0) - RL) < 1e-12 * RL
    rng = np.random.default_rng(7)
    phase = 0.0
    w0 = complex(v[1, 0], v[2, 0])
    vmag0 = np.linalg.norm(v[:, 0])
    L = b.n[1] * b.dx[1]
    for _ in range(300):
        dt = gp["dt_mean"] + gp["dt_amp"] * math.cos(rng.uniform(0, 2 * math.pi))
        orc.push(g, p, dt, x, v, E, B, None, None)
        phase -= 2.0 * math.atan(om * dt / 2.0)
        # unwrap the periodic box around the centre
        z = complex(x[1, 0], x[2, 0])
        dz = z - c0
        dz = complex((dz.real + L / 2) % L - L / 2, (dz.imag + L / 2) % L - L / 2)
        assert abs(abs(dz) - RL) < 1e-11 * RL
        assert abs(np.linalg.norm(v[:, 0]) - vmag0) < 1e-13 * vmag0
        assert x[0, 0] == b.dx[0] * (b.n[0] // 2)
    w = complex(v[1, 0], v[2, 0])
    dphi = math.remainder(math.atan2(w.imag, w.real) - math.atan2(w0.imag, w0.real) - phase, 2 * math.pi)
    assert abs(dphi) < 1e-11


def test_boris_second_order_phase_error():
    """Phase error after a fixed time T scales as dt^2 (Appendix A.2: second order)."""
    errs = []
    for nsteps in (40, 80, 160):
        b = wl.gyration()
        g, p = orc.grid_of(b), orc.params_of(b)
        x, v = wl.absolute_positions(b), b.p.astype(np.float64)
        E, B = _uniform_fields(b.n, 3)
        T = 20.0
        dt = T / nsteps
        for _ in range(nsteps):
            orc.push(g, p, dt, x, v, E, B, None, None)
        gam = math.sqrt(1.0 + (v[:, 0] @ v[:, 0]) / b.C ** 2)
        om = 1.0 / gam
        w = complex(v[1, 0], v[2, 0])
        exact = -om * T + math.pi / 2.0     # initial four-velocity points along +z
        errs.append(abs(math.remainder(math.atan2(w.imag, w.real) - exact, 2 * math.pi)))
    assert 3.8 < errs[0] / errs[1] < 4.2
    assert 3.8 < errs[1] / errs[2] < 4.2


def test_exb_drift_nonrelativistic_exact():
    """Gas moving at v0 y_hat through B = x_hat gives E0 = -v x B; in the
    non-relativistic limit the guiding centre moves at exactly v0 y_hat."""
    v0 = 0.3
    b = wl.gyration(v0=v0, C=1e9)
    g, p = orc.grid_of(b), orc.params_of(b)
    x, v = wl.absolute_positions(b), b.p.astype(np.float64)
    md = np.zeros((4, b.ncell))
    E = orc.field_prep(g, p, b.rho, b.mom, b.B, md)
    np.testing.assert_allclose(E[2], v0, rtol=1e-15)   # E0 = (0, 0, v0 B0)
    assert np.all(E[0] == 0) and np.all(E[1] == 0)
    c0, _ = _centre_yz(x[:, 0], v[:, 0], b.C, wE=v0)
    t = 0.0
    rng = np.random.default_rng(11)
    L = b.n[1] * b.dx[1]
    for _ in range(200):
        dt = 0.5 + 0.1 * math.cos(rng.uniform(0, 2 * math.pi))
        orc.push(g, p, dt, x, v, E, b.B, None, None)
        t += dt
        c, _ = _centre_yz(x[:, 0], v[:, 0], b.C, wE=v0)
        d = c - (c0 + v0 * t)
        d = complex((d.real + L / 2) % L - L / 2, d.imag)
        assert abs(d) < 1e-10


def test_gyration_with_drift_energy_oscillation_level():
    """Appendix B.1: with v0 = 1 the co-moving energy oscillates at the 0.1% level;
    the relativistic run has a smaller fractional error."""
    out = {}
    for rel in (False, True):
        gp = _golden("gyration_appB1.json")["relativistic" if rel else "nonrelativistic"]
        v0 = gp["drift_v0"]
        b = wl.gyration(relativistic=rel, v0=v0)
        g, p = orc.grid_of(b), orc.params_of(b)
        x, v = wl.absolute_positions(b), b.p.astype(np.float64)
        E = orc.field_prep(g, p, b.rho, b.mom, b.B, np.zeros((4, b.ncell)))
        C = b.C
        G0 = 1.0 / math.sqrt(1.0 - v0 * v0 / (C * C))
        rng = np.random.default_rng(1)
        ek = []
        for _ in range(400):
            dt = gp["dt_mean"] + gp["dt_amp"] * math.cos(rng.uniform(0, 2 * math.pi))
            orc.push(g, p, dt, x, v, E, b.B, None, None)
            vv = v[:, 0]
            gam = math.sqrt(1.0 + vv @ vv / (C * C))
            ek.append((G0 * (gam - v0 * vv[1] / (C * C)) - 1.0) * C * C)
        ek = np.array(ek)
        out[rel] = (ek.max() - ek.min()) / 2.0 / ek.mean()
    level = _golden("gyration_appB1.json")["nonrelativistic"]["energy_oscillation_with_drift"]
    assert level / 3.0 < out[False] < level * 3.0
    assert out[True] < out[False]


# ---------------------------------------------------------------------------
# moments (Appendix A.1) and feedback / conservation (Section 2.1, App. A.3)
# ---------------------------------------------------------------------------

def test_charge_sum_and_uniform_beam_current():
    b = wl.periodic_thermal_2d(nx=16, ny=12, ppc=5)
    g, p = orc.grid_of(b), orc.params_of(b)
    x = wl.absolute_positions(b)
    v = np.zeros((3, b.np))
    v[0], v[1], v[2] = 30.0, -4.0, 7.0          # one common four-velocity
    md = orc.deposit_moments(g, p, x, v, b.ncell)
    dV = 1.0
    assert abs(md[0].sum() * dV - b.qm_cr * b.m_cr * b.np) < 1e-13 * b.qm_cr * b.m_cr * b.np
    gam = math.sqrt(1.0 + (v[:, 0] @ v[:, 0]) / b.C ** 2)
    for d in range(3):
        np.testing.assert_allclose(md[1 + d], md[0] * v[d, 0] / gam, rtol=1e-13, atol=0)


def test_moments_after_push_equal_standalone_deposit():
    b = wl.periodic_thermal_2d(nx=12, ny=10, ppc=4, dv_amp=0.2)
    st = orc.State(b, wl.absolute_positions(b), b.p.astype(np.float64))
    corr, md = st.push_only(b.dt)
    md2 = orc.deposit_moments(st.g, st.p, st.x, st.v, b.ncell)
    np.testing.assert_allclose(md, md2, rtol=1e-13, atol=1e-18)


@pytest.mark.parametrize("hall", [0, 1])
def test_total_momentum_and_energy_conserved(hall):
    """Gas + CR momentum and energy are unchanged by a step (Newton's third law,
    eq:eng), to roundoff, with a non-zero electric field."""
    b = wl.periodic_thermal_2d(nx=10, ny=8, ppc=6, dv_amp=0.5, pmag=10.0)
    b.hall = hall
    b.m_cr = 0.05       # make the CR share of the totals visible
    # tilt B off the axes so every momentum component is exchanged
    rng = np.random.default_rng(21)
    b.B = np.ascontiguousarray(np.array([[1.0], [0.6], [-0.4]]) + 0.3 * rng.standard_normal(b.B.shape))
    st = orc.State(b, wl.absolute_positions(b), b.p.astype(np.float64))
    t0 = st.totals()
    for _ in range(5):
        st.step(b.dt)
    t1 = st.totals()
    P0, P1 = t0[0:3] + t0[4:7], t1[0:3] + t1[4:7]
    scaleP = np.abs(st.mom).sum() + b.m_cr * np.abs(st.v).sum()
    assert np.abs(P1 - P0).max() < 1e-13 * scaleP
    assert abs((t1[3] + t1[7]) - (t0[3] + t0[7])) < 1e-13 * (t0[3] + t0[7])
    # the exchange is real: every component of the CR share changed by much
    # more than roundoff
    assert np.abs(t1[4:7] - t0[4:7]).min() > 1e-6 * scaleP
    assert abs(t1[7] - t0[7]) > 1e-6 * t0[7]


def test_feedback_applies_corrector_and_resets():
    g = orc.make_grid(2, (3, 2, 1), dx=(2.0, 0.5, 3.0))
    corr = np.arange(24, dtype=np.float64).reshape(4, 6) - 5.0
    mom = np.ones((3, 6))
    egas = np.full(6, 4.0)
    expect_m = mom + corr[:3] / 3.0
    expect_e = egas + corr[3] / 3.0
    orc.apply_feedback(g, mom, egas, corr)
    np.testing.assert_allclose(mom, expect_m, rtol=1e-15)
    np.testing.assert_allclose(egas, expect_e, rtol=1e-15)
    assert not corr.any()


def test_hall_field_identities():
    """With the CR-Hall term: E = -[(1-R) v_g + R u_CR] x B (eq:emfcr1), and the
    energy identities of eq:eng: v_g.F = (1-R) J.E0 = J.E, where F = n_g (E0 - E)."""
    rng = np.random.default_rng(5)
    g = orc.make_grid(2, (7, 5, 1))
    nc = 35
    rho = rng.uniform(0.5, 2.0, nc)
    vel = rng.normal(0, 1, (3, nc))
    mom = rho * vel
    B = rng.normal(0, 1, (3, nc))
    md = np.empty((4, nc))
    md[0] = rng.uniform(0.01, 0.2, nc)
    md[1:] = rng.normal(0, 0.3, (3, nc))
    p1 = orc.make_params(1.0, 1.3, 100.0, 1.0, 1)
    p0 = orc.make_params(1.0, 1.3, 100.0, 1.0, 0)
    E = orc.field_prep(g, p1, rho, mom, B, md)
    E0 = orc.field_prep(g, p0, rho, mom, B, md)
    np.testing.assert_allclose(E0, -np.cross(vel.T, B.T).T, rtol=1e-13, atol=1e-15)
    ng = 1.3 * rho
    n, J = md[0], md[1:]
    R = n / (ng + n)
    adv = (1.0 - R) * vel + R * (J / n)
    np.testing.assert_allclose(E, -np.cross(adv.T, B.T).T, rtol=1e-12, atol=1e-14)
    F = ng * (E0 - E)
    lhs = (vel * F).sum(0)
    mid = (1.0 - R) * (J * E0).sum(0)
    rhs = (J * E).sum(0)
    np.testing.assert_allclose(lhs, mid, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(rhs, mid, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("bmag,axis", [(2.0, True), (1.0, True), (0.25, True), (1.0, False)])
def test_parallel_field_is_cleaned_before_the_kick(bmag, axis):
    """A field with E parallel to B at the particle does no work (App. A.2
    cleaning), whatever |B| (cleaning applies for every |B| > 0)."""
    g = orc.make_grid(3, (4, 4, 4))
    p = orc.make_params(1.0, 1.0, 50.0, 1.0, 0)
    u = np.array([1.0, 0.0, 0.0]) if axis else np.array([1.0, -2.0, 2.0]) / 3.0
    E, B = _uniform_fields((4, 4, 4), 3, E=tuple(0.7 * u), B=tuple(bmag * u))
    x = np.array([[1.3], [2.2], [0.7]])
    v = np.array([[3.0], [1.0], [-2.0]])
    ek0 = orc.kinetic_energy(v[:, 0], 50.0)
    for _ in range(10):
        orc.push(g, p, 0.05, x, v, E, B, None, None)
    assert abs(orc.kinetic_energy(v[:, 0], 50.0) - ek0) < 1e-13 * ek0


def test_gamma_and_kinetic_energy_forms():
    """gamma = sqrt(C^2+v^2)/C = C/sqrt(C^2-u^2); E_k = (gamma-1)C^2 (eq:parEk)."""
    for C in (10.0, 300.0):
        for v in ([1.0, 2.0, 3.0], [100.0, -50.0, 20.0], [1e-3, 0.0, 0.0]):
            v = np.array(v)
            g = orc.gamma(v, C)
            u = v / g
            assert abs(g - C / math.sqrt(C * C - u @ u)) < 1e-13 * g
            ek = orc.kinetic_energy(v, C)
            # (gamma - 1) C^2 itself carries a rounding error of order eps*gamma*C^2
            assert abs(ek - (g - 1.0) * C * C) < 8 * np.finfo(float).eps * g * C * C
            v2 = v @ v
            if v2 < 1e-4 * C * C:   # non-relativistic series v^2/2 - v^4/(8 C^2) + v^6/(16 C^4)
                assert abs(ek - (v2 / 2 - v2 * v2 / (8 * C * C) + v2 ** 3 / (16 * C ** 4))) < 1e-15 * v2


# ---------------------------------------------------------------------------
# sort (the GPU layout; checked against numpy's stable argsort)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,n,brick", [
    (2, (16, 12, 1), (16, 12, 1)),
    (2, (16, 12, 1), (8, 8, 1)),
    (2, (13, 7, 1), (4, 4, 1)),
    (3, (8, 6, 10), (4, 4, 4)),
    (3, (9, 9, 9), (9, 9, 9)),
])
def test_sort_is_a_stable_sort_by_brick_key(ndim, n, brick):
    rng = np.random.default_rng(8)
    g = orc.make_grid(ndim, n)
    nc = int(np.prod(n))
    cells = rng.integers(0, nc, 3000).astype(np.int32)
    cells[:500] = cells[0]     # long run of one cell: stability matters
    perm, counts = orc.sort_cells(g, brick, cells)
    keys = np.array([orc.sort_key(g, brick, int(c)) for c in cells])
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable"))
    np.testing.assert_array_equal(counts, np.bincount(keys, minlength=len(counts)))
    assert len(counts) == orc.sort_nkeys(g, brick)


def test_sort_key_properties():
    """Whole-grid brick gives the linear cell; otherwise keys of one brick form one
    contiguous block ordered x fastest, and distinct cells get distinct keys."""
    g = orc.make_grid(3, (8, 4, 6))
    for c in range(8 * 4 * 6):
        assert orc.sort_key(g, (8, 4, 6), c) == c
    brick = (4, 2, 3)
    vol = 24
    seen = {}
    for k in range(6):
        for j in range(4):
            for i in range(8):
                key = orc.sort_key(g, brick, (k * 4 + j) * 8 + i)
                assert key not in seen
                seen[key] = (i, j, k)
                bid = key // vol
                assert bid == ((k // 3) * 2 + j // 2) * 2 + i // 4
                r = key % vol
                assert r == ((k % 3) * 2 + j % 2) * 4 + i % 4


def test_cells_of_positions():
    g = orc.make_grid(2, (10, 7, 1), dx=(0.5, 2.0, 1.0), x0=(-1.0, 3.0, 0.0))
    x = np.array([[-1.0, -0.51, 3.99, 0.0], [3.0, 4.99, 16.99, 5.0]])
    np.testing.assert_array_equal(orc.cells_of(g, x), [0, 0 + 10 * 0 + 0 * 0 + 0, 9 + 60, 2 + 10])


def test_energy_change_equals_the_definition_in_high_precision():
    """The corrector's dE_k equals E_k(v^(n+1)) - E_k(v^(n)) (eq:parEk,
    App. A.3) evaluated with 50-digit decimals from the stored FP64 states, to
    the rounding of those states."""
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    rng = np.random.default_rng(17)
    g = orc.make_grid(3, (6, 6, 6), dx=(1.0, 1.0, 1.0))
    p = orc.make_params(1.0, 1.0, 30.0, 1.0, 0)
    nc = 216
    E = 0.5 * rng.standard_normal((3, nc))
    B = np.array([[1.0], [0.3], [-0.2]]) + 0.2 * rng.standard_normal((3, nc))

    def ek(v, C):
        v2 = sum(Decimal(float(a)) ** 2 for a in v)
        Cd = Decimal(C)
        gam = (Cd * Cd + v2).sqrt() / Cd
        return v2 / (gam + 1)

    checked = 0
    for _ in range(40):
        x = rng.uniform(0.5, 5.5, (3, 1))
        v = rng.standard_normal((3, 1)) * rng.choice([0.5, 5.0, 60.0])
        v0 = v[:, 0].copy()
        corr = np.zeros((4, nc))
        orc.push(g, p, 0.05, x, v, E, B, corr, None)
        dek = -corr[3].sum()                      # m = 1
        exact = float(ek(v[:, 0], 30.0) - ek(v0, 30.0))
        scale = np.finfo(float).eps * (v[:, 0] @ v[:, 0] + v0 @ v0)
        assert abs(dek - exact) < 16 * scale + 1e-15 * abs(exact)
        assert abs(exact) > 1000 * scale          # the check is not vacuous
        checked += 1
    assert checked == 40


# ---------------------------------------------------------------------------
# diagnostics: spectra, E_max (Section 4.3), Lambda (eq:lambda)
# ---------------------------------------------------------------------------

def _v_of_energy(E, C):
    """Four-velocity along x whose kinetic energy per unit mass is E:
    gamma = 1 + E/C^2, v^2 = (gamma^2 - 1) C^2 = E (E + 2 C^2) / C^2."""
    E = np.asarray(E, dtype=np.float64)
    v = np.zeros((3, E.shape[0]))
    v[0] = np.sqrt(E * (E + 2.0 * C * C)) / C
    return v


def test_spectrum_brute_force_edges_and_region():
    """Hand-placed particles: a bin holds edges[b] <= q < edges[b+1], values
    outside [edges[0], edges[-1]) and particles outside the half-open region
    are not counted, and the two sums are the plain power sums."""
    g = orc.make_grid(2, (8, 8, 1))
    p = orc.make_params(1.0, 1.0, 1e6, 1.0, 0)
    speeds = np.array([0.5, 1.0, 1.999, 2.0, 3.0, 4.0, 0.25, 2.5])
    v = np.zeros((3, 8))
    v[1] = speeds                                    # |v| along y
    x = np.array([[0.5, 1.0, 2.0, 3.0, 3.999, 5.0, 6.0, 4.0],
                  [0.5, 0.5, 0.5, 0.5, 7.5, 1.0, 1.0, 0.5]])
    edges = [0.5, 1.0, 2.0, 3.0, 4.0]
    counts, sums = orc.spectrum(g, p, x, v, 1, edges, n_moment=2)
    # 0.5 | 1.0, 1.999 | 2.0, 2.5 | 3.0 ; 4.0 (= last edge) and 0.25 excluded
    np.testing.assert_array_equal(counts, [1, 2, 2, 1])
    inc = np.array([0.5, 1.0, 1.999, 2.0, 3.0, 2.5])
    assert sums[0] == pytest.approx((inc ** 3).sum(), rel=1e-15)
    assert sums[1] == pytest.approx((inc ** 2).sum(), rel=1e-15)
    # region [1, 4) x [0, 1): keeps particles 1, 2, 3 (x = 1.0, 2.0, 3.0; y = 0.5);
    # the one at x = 4.0 sits on the excluded upper face
    counts, sums = orc.spectrum(g, p, x, v, 1, edges, region=[1.0, 4.0, 0.0, 1.0], n_moment=0)
    np.testing.assert_array_equal(counts, [0, 2, 1, 0])
    assert sums[1] == 3.0 and sums[0] == pytest.approx(1.0 + 1.999 + 2.0, rel=1e-15)


def test_spectrum_energy_kind_bins_the_kinetic_energy():
    """Energies placed at bin centres of log-spaced edges come back one per bin
    (E_k = v^2/(gamma+1) = (gamma-1) C^2, eq:parEk, in the relativistic regime)."""
    C = 3.0
    edges = np.geomspace(0.01, 1e4, 13)
    centres = np.sqrt(edges[:-1] * edges[1:])
    g = orc.make_grid(3, (2, 2, 2))
    p = orc.make_params(1.0, 1.0, C, 1.0, 0)
    x = np.full((3, centres.shape[0]), 0.5)
    counts, sums = orc.spectrum(g, p, x, _v_of_energy(centres, C), 0, edges, n_moment=1)
    np.testing.assert_array_equal(counts, np.ones(12, dtype=np.int64))
    assert sums[0] == pytest.approx((centres ** 2).sum(), rel=1e-12)
    assert sums[1] == pytest.approx(centres.sum(), rel=1e-12)


def test_emax_closed_form_of_the_paper():
    """For f(E) ~ E^-m exp(-E/E_cut) the ratio of eq:emax is (n + 1 - m) E_cut
    (Section 4.3).  With m = -1 (a Gamma distribution of shape 2) it is
    (n + 2) E_cut exactly.  Energies at the distribution's quantiles reproduce
    it up to the tail beyond the last quantile, which only lowers the ratio and
    matters more the larger n is."""
    from scipy import stats
    Ecut, C, N = 2.5, 50.0, 200000
    u = (np.arange(N) + 0.5) / N
    E = np.where(u > 0.5, stats.gamma.isf(1.0 - u, a=2.0, scale=Ecut), stats.gamma.ppf(u, a=2.0, scale=Ecut))
    g = orc.make_grid(3, (1, 1, 1))
    p = orc.make_params(1.0, 1.0, C, 1.0, 0)
    x = np.full((3, N), 0.5)
    v = _v_of_energy(E, C)
    edges = [0.0, 1e9]
    for n, tol in ((1, 1e-4), (2, 3e-4)):
        counts, sums = orc.spectrum(g, p, x, v, 0, edges, n_moment=n)
        assert counts[0] == N
        assert sums[0] / sums[1] == pytest.approx((n + 2) * Ecut, rel=tol)
    # the paper's n = 6: 8 E_cut, approached from below
    _, s6 = orc.spectrum(g, p, x, v, 0, edges, n_moment=6)
    assert -0.01 < s6[0] / s6[1] / (8.0 * Ecut) - 1.0 < 0.0


def test_lambda_map_matches_the_hall_field():
    """E - E0 = -R (u_CR - v_g) x B = -v_A Lambda x B: the Lambda map against
    the CR-Hall field of the field preparation (eq:emfcr1 vs eq:emfcr2), and
    Lambda = 0 where the CRs move with the gas."""
    rng = np.random.default_rng(9)
    g = orc.make_grid(3, (3, 4, 2))
    nc = 24
    rho = rng.uniform(0.5, 2.0, nc)
    vel = rng.normal(0, 1, (3, nc))
    B = rng.normal(0, 1, (3, nc))
    md = np.empty((4, nc))
    md[0] = rng.uniform(0.01, 0.2, nc)
    md[1:] = rng.normal(0, 0.3, (3, nc))
    md[1:, :4] = md[0, :4] * vel[:, :4]          # co-moving CRs in four cells
    p1 = orc.make_params(1.0, 0.7, 100.0, 1.0, 1)
    p0 = orc.make_params(1.0, 0.7, 100.0, 1.0, 0)
    lam = orc.lambda_map(g, p1, rho, rho * vel, B, md)
    E = orc.field_prep(g, p1, rho, rho * vel, B, md)
    E0 = orc.field_prep(g, p0, rho, rho * vel, B, md)
    vA = np.sqrt((B * B).sum(0) / rho)
    np.testing.assert_allclose(E - E0, -vA * np.cross(lam.T, B.T).T, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(lam[:, :4], 0.0, atol=1e-15)
    # no field: Lambda is defined as zero
    lam0 = orc.lambda_map(g, p1, rho, rho * vel, np.zeros((3, nc)), md)
    assert not lam0.any()


def test_field_free_box_streams_particles_freely():
    """B = 0 everywhere: E0 = -v x B and the CR-Hall force vanish, so every
    particle keeps its four-velocity exactly, moves by u dt with
    u = v/gamma (periodic wrap), and the corrector deposit is exactly zero."""
    b = wl.periodic_thermal_2d(nx=12, ny=10, ppc=4, dv_amp=0.5, seed=5)
    b.B = np.zeros_like(b.B)
    b.hall = 1
    g, p = orc.grid_of(b), orc.params_of(b)
    x = np.ascontiguousarray(wl.absolute_positions(b))
    v = np.ascontiguousarray(b.p.astype(np.float64))
    x0, v0 = x.copy(), v.copy()
    md = orc.deposit_moments(g, p, x, v, b.ncell)
    E = orc.field_prep(g, p, b.rho, b.mom, b.B, md)
    assert np.all(E == 0.0)
    corr = np.zeros((4, b.ncell))
    dt = b.dt
    orc.push(g, p, dt, x, v, E, b.B, corr, None)
    np.testing.assert_array_equal(v, v0)
    assert np.all(corr == 0.0)
    gam = np.sqrt(1.0 + (v0 ** 2).sum(axis=0) / b.C ** 2)
    for d in range(2):
        L = b.n[d] * b.dx[d]
        want = (x0[d] + v0[d] / gam * dt) % L
        diff = (x[d] - want + L / 2) % L - L / 2
        assert np.abs(diff).max() < 1e-12 * L
