"""Pins of the oracle's open boundary (a conducting wall at x = 0 and an open
upper face, the paper's shock box of Section 5).

Closed forms: with the gas at rest and B along x there is no force along x,
so x(t) = x0 + u_x t and a particle leaves exactly when its half-step or
full-step position reaches the open face; the charge density of the particles
left is qm m N / V; the sort puts removed particles after every cell, in
input order (compared with numpy's stable argsort).
"""
import math

import numpy as np

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl

WALL_OPEN = 2


def _open_box(seed=3, nx=24, ny=6, ppc=5):
    box = wl.periodic_thermal_2d(nx=nx, ny=ny, ppc=ppc, dv_amp=0.0, seed=seed)
    box.bc = (WALL_OPEN, 0, 0)
    box.mom[:] = 0.0
    box.B[:] = 0.0
    box.B[0] = 1.0          # B along x: no force along x
    return box


def test_particles_leave_exactly_when_they_reach_the_open_face():
    box = _open_box()
    x = np.ascontiguousarray(wl.absolute_positions(box).astype(np.float64))
    v = np.ascontiguousarray(box.p.astype(np.float64))
    st = orc.State(box, x, v)
    C = box.C
    gam = np.sqrt(1.0 + (v ** 2).sum(axis=0) / C ** 2)
    ux = v[0] / gam
    L = box.n[0] * box.dx[0]
    dt = 4.0 * box.dt
    nsteps = 12
    E = np.zeros((3, box.ncell))
    corr = np.zeros((4, box.ncell))
    for _ in range(nsteps):
        md = np.zeros((4, box.ncell))
        orc.push(st.g, st.p, dt, st.x, st.v, E, st.B, corr, md)
    dead = np.isnan(st.x[0])
    # reflection at the lower wall turns u_x around: follow it in closed form
    # step by step (half steps), removing at the first half step at or past L
    xs = x[0].copy()
    us = ux.copy()
    gone = np.zeros(box.np, dtype=bool)
    margin = np.full(box.np, np.inf)
    for _ in range(2 * nsteps):
        xs = xs + 0.5 * dt * us
        neg = xs < 0.0
        xs[neg] = -xs[neg]
        us[neg] = -us[neg]
        margin = np.minimum(margin, np.abs(xs - L))
        hit = (xs >= L) & ~gone
        gone |= hit
        xs[gone] = np.nan
    ok = margin > 1e-9
    assert np.array_equal(dead[ok], gone[ok])
    assert 0 < dead.sum() < box.np
    # removed particles carry no four-velocity; the others keep |v_x| (no
    # force along x) and |v| (the field does no work)
    assert np.all(st.v[:, dead] == 0.0)
    np.testing.assert_allclose(np.abs(st.v[0, ~dead]), np.abs(v[0, ~dead]), rtol=1e-15)
    np.testing.assert_allclose((st.v[:, ~dead] ** 2).sum(0), (v[:, ~dead] ** 2).sum(0), rtol=1e-13)
    # the last moments deposit holds exactly the charge of the particles left
    dV = box.dx[0] * box.dx[1] * box.dx[2]
    np.testing.assert_allclose(md[0].sum() * dV, box.qm_cr * box.m_cr * (~dead).sum(), rtol=1e-12)
    # no force along x and no work (E = 0): the x-momentum and energy
    # corrector channels stay exactly zero
    assert np.abs(corr[0]).max() == 0.0 and np.abs(corr[3]).max() == 0.0


def test_removed_particles_sort_after_every_cell_in_input_order():
    box = _open_box(seed=8, nx=20, ny=6, ppc=4)
    g = orc.grid_of(box)
    x = np.ascontiguousarray(wl.absolute_positions(box).astype(np.float64))
    rng = np.random.default_rng(2)
    kill = rng.random(box.np) < 0.3
    x[0, kill] = np.nan
    cell = orc.cells_of(g, x)
    assert np.all(cell[kill] == -1) and np.all(cell[~kill] >= 0)
    brick = (8, 8, 1)
    perm, counts = orc.sort_cells(g, brick, cell)
    nk = orc.sort_nkeys(g, brick)
    key = np.array([nk if c < 0 else orc.sort_key(g, brick, int(c)) for c in cell])
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert counts.sum() == (~kill).sum()


def test_lower_face_is_still_a_reflecting_wall():
    box = _open_box(seed=5)
    g = orc.grid_of(box)
    xp, vp = orc.boundary(g, [-0.25, 1.5], [-3.0, 1.0, 0.0])
    assert xp[0] == 0.25 and vp[0] == 3.0
    xp, vp = orc.boundary(g, [box.n[0] * box.dx[0] + 0.1, 1.5], [3.0, 1.0, 0.0])
    assert xp[0] < box.n[0] * box.dx[0] and vp[0] == 3.0   # held inside, not reflected


def test_deposit_folds_at_the_wall_and_keeps_charge_at_the_open_face():
    """TSC at s = 0.2: (0.32, 0.66, 0.02) on cells -1, 0, 1, the wall
    folding cell -1 onto cell 0; at s = n - 0.2 the weight beyond the open
    face stays in the last cell, so no charge is lost before the particle
    itself leaves."""
    n = 6
    g = orc.make_grid(2, (n, 4, 1), bc=(WALL_OPEN, 0, 0))
    for s, cells in ((0.2, {0: 0.98, 1: 0.02}), (n - 0.2, {n - 1: 0.98, n - 2: 0.02})):
        planes = np.zeros((1, n * 4))
        orc.deposit(g, [s, 1.5], [1.0], planes)
        row = planes.reshape(4, n)[1]
        exp = np.zeros(n)
        for c, w in cells.items():
            exp[c] = 0.75 * w
        np.testing.assert_allclose(row, exp, rtol=0, atol=1e-15)
        assert abs(planes.sum() - 1.0) < 1e-15


# ---------------------------------------------------------------------------
# random numbers, front tracking and injection (Section 5)
# ---------------------------------------------------------------------------

def test_counter_based_words_are_uniform_and_independent():
    """Statistical pins of the counter-based generator: uniform words,
    independent counters and keys, and full avalanche on a counter bit."""
    key = [12345, 678]
    words = np.array([orc.philox([k, 7, 0, 0], key) for k in range(4096)], dtype=np.uint64)
    u = (words.astype(np.float64) + 0.5) / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.005
    hist = np.histogram(u.ravel(), bins=64, range=(0.0, 1.0))[0]
    chi2 = ((hist - hist.mean()) ** 2 / hist.mean()).sum()
    assert chi2 < 120.0                                     # 63 degrees of freedom
    r = np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]
    assert abs(r) < 0.06
    # a different key or call gives a different stream
    assert not np.array_equal(orc.philox([5, 7, 0, 0], key), orc.philox([5, 7, 0, 0], [12346, 678]))
    assert not np.array_equal(orc.philox([5, 7, 0, 0], key), orc.philox([5, 8, 0, 0], key))
    # flipping one counter bit changes about half of the 128 output bits
    flips = []
    for b in range(32):
        a = orc.philox([1000, 3, 0, 0], key)
        c = orc.philox([1000 ^ (1 << b), 3, 0, 0], key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, c)))
    assert 48 < np.mean(flips) < 80


def _shock(nx=256, ny=8, **kw):
    return wl.shock_front_2d(nx=nx, ny=ny, **kw)


def test_front_of_a_sharp_shock_is_the_smoothed_step_crossing():
    """A sharp jump of v_x from 0 to -v0 at the face x = f: smoothed with a
    Gaussian of 4 cells it falls to 0.6 v0 where Phi((x - f)/4) = 0.6, i.e.
    x_s = f + 0.2533 * 4 cells; the pressure step reaches 2/3 P1 where
    Phi = 1/3, x = f - 0.4307 * 4, and x_t is the first cell centre at or
    below that."""
    box = _shock(nx=256, ny=8, front=0.25)
    g = orc.grid_of(box)
    xs, xt, rup, vup = orc.front(g, box.rho, box.mom, box.egas, box.B)
    f = 0.25 * 256
    assert abs(xs - (f + 0.2533 * 4.0)) < 0.02
    xt_expect = np.floor(f - 0.4307 * 4.0 - 0.5) + 0.5
    assert xt == xt_expect
    assert rup == 1.0 and vup == -20.0
    # no front in a uniform inflow
    box.mom[0] = -20.0 * box.rho
    xs2 = orc.front(g, box.rho * 0 + 1.0, np.ascontiguousarray(np.vstack([np.full(box.ncell, -20.0),
                                                                          box.mom[1:]])),
                    box.egas, box.B)[0]
    assert np.isnan(xs2)


def test_injection_conserves_momentum_energy_and_mass_and_places_particles():
    box = _shock(nx=256, ny=8, front=0.25)
    g, p = orc.grid_of(box), orc.params_of(box)
    fr = orc.front(g, box.rho, box.mom, box.egas, box.B)
    rho, mom, egas = box.rho.copy(), box.mom.copy(), box.egas.copy()
    dV = box.dx[0] * box.dx[1] * box.dx[2]
    gas0 = (rho.sum() * dV, mom.sum(axis=1) * dV, egas.sum() * dV)
    eta, fE = 0.2, 10.0
    xn, vn, carry = orc.inject(g, p, fr, np.nan, box.dt, eta, fE, 99, 0, 0.0, 100000, rho, mom, egas)
    N = xn.shape[1]
    assert N > 100
    gam = np.sqrt(1.0 + (vn ** 2).sum(axis=0) / box.C ** 2)
    Ek = (vn ** 2).sum(axis=0) / (gam + 1.0)
    # static front: every particle has E_k = 10 E_sh, E_sh = v_up^2 / 2
    np.testing.assert_allclose(Ek, fE * 0.5 * fr[3] ** 2, rtol=1e-12)
    # at the front, spread over the box in y, isotropic
    assert np.all(xn[0] == fr[0])
    Ly = box.n[1] * box.dx[1]
    assert xn[1].min() >= 0.0 and xn[1].max() < Ly
    u = np.sort(xn[1] / Ly)                       # uniform in y: Kolmogorov-Smirnov at the 0.1% level
    ks = max(np.max(np.arange(1, N + 1) / N - u), np.max(u - np.arange(N) / N))
    assert ks < 1.95 / np.sqrt(N)
    # isotropic: every component of the direction has mean 0 and mean square 1/3
    n_hat = vn / np.sqrt((vn ** 2).sum(axis=0))
    for d in range(3):
        assert abs(n_hat[d].mean()) < 4.0 / np.sqrt(3.0 * N), d
        assert abs((n_hat[d] ** 2).mean() - 1.0 / 3.0) < 4.0 * np.sqrt(4.0 / 45.0 / N), d
    # the gas gives exactly what the particles take
    m = p.m_cr
    np.testing.assert_allclose(rho.sum() * dV, gas0[0] - N * m, rtol=1e-13)
    np.testing.assert_allclose(mom.sum(axis=1) * dV + m * vn.sum(axis=1), gas0[1], rtol=1e-13, atol=1e-9)
    np.testing.assert_allclose(egas.sum() * dV + m * Ek.sum(), gas0[2], rtol=1e-13)
    # the cells that gave are those between x_t and x_s
    changed = np.where(rho != box.rho)[0] % box.n[0]
    xc = changed + 0.5
    assert np.all((xc >= fr[1]) & (xc < fr[0]))


def test_injected_count_follows_the_swept_mass_over_many_calls():
    """N = floor(eta M / m + carry) per call: over many calls the total is the
    floor of eta times the total swept mass over m (the carry is exact)."""
    box = _shock(nx=128, ny=4, front=0.5)
    g, p = orc.grid_of(box), orc.params_of(box)
    fr = orc.front(g, box.rho, box.mom, box.egas, box.B)
    eta = 0.01
    rho, mom, egas = box.rho.copy(), box.mom.copy(), box.egas.copy()
    carry, total = 0.0, 0
    calls = 40
    for call in range(calls):
        xn, vn, carry = orc.inject(g, p, fr, fr[0], box.dt, eta, 10.0, 5, call, carry, 1 << 20, rho, mom, egas)
        total += xn.shape[1]
    A = box.n[1] * box.dx[1] * box.dx[2]
    M = fr[2] * abs(fr[3]) * box.dt * A * calls
    assert total == int(np.floor(eta * M / p.m_cr + 1e-9)) or total == int(np.floor(eta * M / p.m_cr - 1e-9))
    assert 0.0 <= carry < 1.0
    # a front advancing at V into the inflow sweeps rho (|v_up| + V) A per unit time
    V = 5.0
    carry, total = 0.0, 0
    for call in range(calls):
        xn, vn, carry = orc.inject(g, p, fr, fr[0] - V * box.dt, box.dt, eta, 10.0, 5, call, carry, 1 << 20,
                                   rho, mom, egas)
        total += xn.shape[1]
    M = fr[2] * (abs(fr[3]) + V) * box.dt * A * calls
    assert abs(total - eta * M / p.m_cr) < 1.0 + 1e-6


def test_moving_front_boosts_the_injected_particles():
    """With the front moving at V the injection energy holds in the front's
    frame: boosting the four-velocity back by -V gives E_k = 10 E_sh."""
    box = _shock(nx=256, ny=8, front=0.25)
    g, p = orc.grid_of(box), orc.params_of(box)
    fr = orc.front(g, box.rho, box.mom, box.egas, box.B)
    V = 7.0
    xs_prev = fr[0] - V * box.dt
    xn, vn, _ = orc.inject(g, p, fr, xs_prev, box.dt, 0.2, 10.0, 3, 1, 0.0, 100000, box.rho.copy(),
                           box.mom.copy(), box.egas.copy())
    C = box.C
    Vf = (fr[0] - xs_prev) / box.dt
    G = 1.0 / np.sqrt(1.0 - Vf * Vf / C ** 2)
    gam = np.sqrt(1.0 + (vn ** 2).sum(axis=0) / C ** 2)
    vx_rest = G * (vn[0] - Vf * gam)
    vr = np.vstack([vx_rest, vn[1], vn[2]])
    gr = np.sqrt(1.0 + (vr ** 2).sum(axis=0) / C ** 2)
    np.testing.assert_allclose((vr ** 2).sum(axis=0) / (gr + 1.0), 10.0 * 0.5 * fr[3] ** 2, rtol=1e-9)


def test_early_particles_go_exactly_at_twice_their_injection_time():
    """Section 5's removal rule by brute force: t_i < t_early and t >= 2 t_i;
    the boundaries (t = 2 t_i exactly, t_i = t_early) and particles already
    removed or never injected early (t_i NaN / +inf) included."""
    rng = np.random.default_rng(11)
    n = 400
    t_early = 480.0
    x = rng.uniform(0.0, 10.0, (2, n))
    v = rng.normal(size=(3, n))
    t_inj = rng.uniform(0.0, 1000.0, n)
    t = 700.0
    t_inj[:5] = t / 2.0                    # exactly at 2 t_i: removed
    t_inj[5:10] = np.nextafter(t / 2.0, np.inf)   # just after: kept
    t_inj[10:15] = t_early                 # not early
    t_inj[15:20] = np.nextafter(t_early, -np.inf)  # early, but 2 t_i > t
    t_inj[20:25] = np.nan
    t_inj[25:30] = np.inf
    x[0, 30:35] = np.nan                   # already gone
    t_inj[30:35] = 0.0
    x, v = np.ascontiguousarray(x), np.ascontiguousarray(v)
    x0, v0 = x.copy(), v.copy()
    nrem = orc.remove_early(x, v, t_inj, t, t_early)
    want = [j for j in range(n)
            if not math.isnan(x0[0, j]) and t_inj[j] < t_early and t >= 2.0 * t_inj[j]]
    assert nrem == len(want)
    assert set(range(5)) <= set(want) and not set(range(5, 35)) & set(want)
    gone = np.isnan(x[0])
    assert sorted(np.flatnonzero(gone & ~np.isnan(x0[0]))) == want
    assert np.all(v[:, want] == 0.0)
    keep = ~gone
    np.testing.assert_array_equal(x[:, keep], x0[:, keep])
    np.testing.assert_array_equal(v[:, keep], v0[:, keep])
    # past 2 t_early: t_i = t_early stays (strictly earlier only), just below goes
    x2 = np.zeros((1, 3))
    v2 = np.ones((3, 3))
    t2 = np.array([t_early, np.nextafter(t_early, -np.inf), 0.0])
    assert orc.remove_early(x2, v2, t2, 2.0 * t_early + 1.0, t_early) == 2
    assert not math.isnan(x2[0, 0]) and math.isnan(x2[0, 1]) and math.isnan(x2[0, 2])


def test_after_twice_the_threshold_no_early_particle_is_left():
    """Injecting at every step up to t = 1200 and removing at each step's
    end: at any t every particle with t_i < min(t_early, t/2) is gone and the
    others remain, so after 2 t_early only particles injected at or after
    t_early are left."""
    dt, t_early = 10.0, 480.0
    t_inj = np.arange(0.0, 1200.0, dt)
    n = t_inj.size
    x = np.zeros((1, n))
    v = np.ones((3, n))
    t = 0.0
    for _ in range(n):
        t += dt
        orc.remove_early(x, v, t_inj, t, t_early)
        live = ~np.isnan(x[0])
        expect = ~((t_inj < t_early) & (2.0 * t_inj <= t))
        np.testing.assert_array_equal(live, expect)
    assert np.all(np.isnan(x[0][t_inj < t_early]))
    assert not np.any(np.isnan(x[0][t_inj >= t_early]))
