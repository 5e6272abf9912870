"""Pins of the oracle's open boundary (a conducting wall at x = 0 and an open
upper face, the paper's shock box of Section 5).

Closed forms: with the gas at rest and B along x there is no force along x,
so x(t) = x0 + u_x t and a particle leaves exactly when its half-step or
full-step position reaches the open face; the charge density of the particles
left is qm m N / V; the sort puts removed particles after every cell, in
input order (compared with numpy's stable argsort).
"""
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
