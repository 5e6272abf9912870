"""Parity of the sm_103a library with the FP64 oracle (needs a GPU).

Everything goes through the C ABI (ctypes binding).  Tolerances:
  * sort permutation and counts: bit-exact;
  * FP64 path: 1e-12 relative after one step (deposits per channel in
    relative L2, positions and four-velocities element-wise);
  * mixed path: deposits 1e-5 relative L2 per channel, positions 1e-5 cells,
    four-velocities 1e-5 relative.
The oracle is put into the library's sorted particle order with the oracle's
own sort, whose equality with the library's sort is checked first.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl
from tests._parity import (default_brick, mixed_rows, momenta_of, periodic_diff, positions_of, rel_l2,
                           sorted_oracle_state, tilt_B)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402

MIXED, FP64 = m.MHDPIC_PREC_MIXED, m.MHDPIC_PREC_FP64
TOL = {FP64: 1e-12, MIXED: 1e-5}


def _boxes():
    """Small variants of every workload shape: several tiles and a ragged tail."""
    return {
        "thermal2d": lambda: tilt_B(wl.periodic_thermal_2d(nx=29, ny=21, ppc=9, dv_amp=0.4, seed=1), 1),
        "beam3d": lambda: wl.alfvenic_beam_3d(n=14, ppc=6, nmodes=16, seed=2),
        "bell2d_hall": lambda: tilt_B(wl.bell_2d(n=24, ppc=12, seed=3), 3, amp=0.05),
        "shock2d_reflect": lambda: tilt_B(wl.shock_2d(nx=96, ny=10, ppc=8.0, seed=4), 4, amp=0.1),
    }


def _engine(box, prec, **kw):
    return m.Engine([box], precision=prec, **kw)


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("name", list(_boxes()))
def test_sort_matches_oracle_bit_exactly(prec, name):
    box = _boxes()[name]()
    eng = _engine(box, prec)
    # put the unsorted particles back and sort through the ABI
    if prec == MIXED:
        eng.set_particles(box.cell, box.off, box.p)
    else:
        eng.x.copy_(torch.from_numpy(wl.absolute_positions(box)))
        eng.p64.copy_(torch.from_numpy(box.p.astype(np.float64)))
    perm, counts = eng.sort(want_perm=True, want_counts=True)
    g = orc.grid_of(box)
    cells = box.cell if prec == MIXED else orc.cells_of(g, wl.absolute_positions(box))
    operm, ocounts = orc.sort_cells(g, default_brick(box.ndim), cells)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.int64), ocounts)
    # the particle arrays were permuted the same way
    if prec == MIXED:
        np.testing.assert_array_equal(eng.cell.cpu().numpy(), box.cell[operm])
        np.testing.assert_array_equal(eng.p.cpu().numpy(), box.p[:, operm])
    else:
        np.testing.assert_array_equal(eng.p64.cpu().numpy(), box.p.astype(np.float64)[:, operm])
    assert eng.status() == 0
    eng.close()


def _lookahead_cells(box, t, prec, cell=None, off=None, v=None, x=None):
    """The cells the library's look-ahead sort keys particles by, recomputed
    in numpy with the same correctly rounded FP32 operations in the same
    order: per dimension +1 when v > 0 and (a v)^2 >= ((1-o)(1-o)) g2, -1
    when v < 0 and (a v)^2 > (o o) g2, g2 = 1 + v^2 w, a = t/dx rounded to
    float, w = 1/(C C) in float."""
    n = box.n
    if prec == MIXED:
        c = cell.astype(np.int64)
        ci = [c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1])]
        o = [off[d].astype(np.float32) for d in range(box.ndim)]
        vf = v.astype(np.float32)
    else:
        ci, o = [], []
        for d in range(box.ndim):
            sd = (x[d] - box.x0[d]) / box.dx[d]
            f = np.floor(sd)
            vv = np.clip(f, 0, n[d] - 1).astype(np.int64)
            ci.append(vv)
            o.append((sd - vv).astype(np.float32))
        ci.append(np.zeros_like(ci[0]))
        vf = v.astype(np.float32)
    C = np.float32(box.C)
    w = np.float32(1) / (C * C)
    v2 = (vf[0] * vf[0] + vf[1] * vf[1]) + vf[2] * vf[2]
    g2 = np.float32(1) + v2 * w
    out = []
    for d in range(3):
        if d >= box.ndim:
            out.append(ci[d])
            continue
        a = np.float32(t * (1.0 / box.dx[d]))
        av = a * vf[d]
        lhs = av * av
        up = np.float32(1) - o[d]
        ru = (up * up) * g2
        rl = (o[d] * o[d]) * g2
        k = np.where((vf[d] > 0) & (lhs >= ru), 1, np.where((vf[d] < 0) & (lhs > rl), -1, 0)).astype(np.int64)
        cd = ci[d] + k
        cd = np.mod(cd, n[d]) if box.bc[d] == 0 else np.clip(cd, 0, n[d] - 1)
        out.append(cd)
    return ((out[2] * n[1] + out[1]) * n[0] + out[0]).astype(np.int64)


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("name", list(_boxes()))
def test_lookahead_sort_matches_oracle_bit_exactly(prec, name):
    """With a look-ahead of half a step the sort keys each particle by the
    cell of x + u dt/2: the permutation and counts equal the oracle's stable
    sort of those cells, recomputed here."""
    box = _boxes()[name]()
    eng = _engine(box, prec)
    t = 0.5 * box.dt * 7.0   # a face crossed by many particles, so that wraps and clamps occur
    if prec == MIXED:
        eng.set_particles(box.cell, box.off, box.p)
        cells = _lookahead_cells(box, t, prec, cell=box.cell, off=box.off, v=box.p)
    else:
        x = wl.absolute_positions(box)
        eng.x.copy_(torch.from_numpy(x))
        eng.p64.copy_(torch.from_numpy(box.p.astype(np.float64)))
        cells = _lookahead_cells(box, t, prec, v=box.p.astype(np.float64), x=x)
    eng.set_sort_lookahead(t)
    perm, counts = eng.sort(want_perm=True, want_counts=True)
    operm, ocounts = orc.sort_cells(orc.grid_of(box), default_brick(box.ndim), cells)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.int64), ocounts)
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_lookahead_sort_changes_nothing_but_the_order(prec):
    """Graph-replayed steps sorted by the half-step cell or by the current
    cell: deposits, gas, fields and the particle set bit-identical."""
    box = tilt_B(wl.alfvenic_beam_3d(n=12, ppc=6, nmodes=8, seed=45), 45)
    box.hall = 1
    stream = torch.cuda.Stream()
    outs = []
    for ahead in (0.0, 0.5 * box.dt):
        eng = m.Engine([box], precision=prec, stream=stream)
        eng.set_sort_lookahead(ahead)
        eng.run(box.dt, 9, 1)
        stream.synchronize()
        if prec == MIXED:
            rows = mixed_rows(eng)
        else:
            rows = np.vstack([eng.x.cpu().numpy(), eng.p64.cpu().numpy()])
        rows = rows[:, np.lexsort(rows[::-1])]
        outs.append((eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy(), eng.mom.cpu().numpy(),
                     eng.egas.cpu().numpy(), eng.fields().cpu().numpy(), rows, eng.status()))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_sort_stability_with_crowded_cells():
    """Hundreds of particles per cell (segment sorts beyond one warp) stay stable."""
    box = wl.periodic_thermal_2d(nx=6, ny=5, ppc=2, seed=9)
    rng = np.random.default_rng(0)
    npart = 9000
    box.cell = rng.integers(0, 3, npart).astype(np.int32)   # three crowded cells
    box.cell[:1500] = 7
    box.off = rng.random((2, npart)).astype(np.float32)
    box.p = rng.standard_normal((3, npart)).astype(np.float32)
    eng = _engine(box, MIXED, brick=(2, 2, 1))
    eng.cell.copy_(torch.from_numpy(box.cell))
    perm, counts = eng.sort(want_perm=True, want_counts=True)
    operm, ocounts = orc.sort_cells(orc.grid_of(box), (2, 2, 1), box.cell)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.int64), ocounts)
    eng.close()


@pytest.mark.parametrize("per_cell,movers", [(300, 0.0), (300, 0.03), (700, 0.01), (200, 0.2)])
def test_sort_of_large_nearly_sorted_cells(per_cell, movers):
    """Segments of 129..1024 particles made of few runs (the input nearly
    sorted, as after a push) and of many (movers): the permutation is the
    stable sort either way."""
    box = wl.periodic_thermal_2d(nx=6, ny=5, ppc=2, seed=10)
    rng = np.random.default_rng(1)
    npart = 30 * per_cell
    cell = (np.arange(npart) // per_cell).astype(np.int32)
    mv = rng.random(npart) < movers
    cell[mv] = rng.integers(0, 30, mv.sum()).astype(np.int32)
    box.cell = cell
    box.off = rng.random((2, npart)).astype(np.float32)
    box.p = rng.standard_normal((3, npart)).astype(np.float32)
    eng = _engine(box, MIXED, brick=(2, 2, 1))
    eng.cell.copy_(torch.from_numpy(box.cell))
    perm, counts = eng.sort(want_perm=True, want_counts=True)
    operm, ocounts = orc.sort_cells(orc.grid_of(box), (2, 2, 1), box.cell)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)
    np.testing.assert_array_equal(counts.cpu().numpy().astype(np.int64), ocounts)
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("name", list(_boxes()))
def test_initial_moments_and_fields(prec, name):
    box = _boxes()[name]()
    eng = _engine(box, prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    md = eng.deposits(1).cpu().numpy()
    # the mixed path deposits the initial moments as a push would (f32 weights)
    for q in range(4):
        assert rel_l2(md[q], st.mom_dep[q]) < (1e-12 if prec == FP64 else TOL[MIXED]), q
    f = eng.fields().cpu().numpy()
    E = st.fields()
    tol = 1e-12 if prec == FP64 else 1e-6
    for q in range(3):
        assert rel_l2(f[q], E[q], floor=1e-3 * np.linalg.norm(box.B)) < tol, q
        assert rel_l2(f[3 + q], box.B[q], floor=1e-3 * np.linalg.norm(box.B)) < tol, q
    eng.close()


def _compare_step(eng, box, st, corr, md, prec, tol_pos=None):
    tol = TOL[prec]
    gc = eng.deposits(0).cpu().numpy()
    gm = eng.deposits(1).cpu().numpy()
    for q in range(4):
        assert rel_l2(gm[q], md[q]) < tol, ("moments", q, rel_l2(gm[q], md[q]))
    for q in range(4):
        assert rel_l2(gc[q], corr[q]) < tol, ("corrector", q, rel_l2(gc[q], corr[q]))
    xg = positions_of(eng)
    vg = momenta_of(eng)
    for d in range(box.ndim):
        L = box.n[d] * box.dx[d]
        dx = periodic_diff(xg[d], st.x[d], L) if box.bc[d] == 0 else xg[d] - st.x[d]
        lim = (1e-12 * (1.0 + np.abs(st.x[d]))) if prec == FP64 else (tol_pos or 1e-5) * box.dx[d]
        assert np.all(np.abs(dx) <= lim), (d, np.abs(dx).max())
    vscale = np.sqrt((st.v ** 2).sum(0))
    assert np.all(np.abs(vg - st.v) <= tol * vscale + 1e-300), np.abs(vg - st.v).max()


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("name", list(_boxes()))
def test_one_step_matches_oracle(prec, name):
    box = _boxes()[name]()
    eng = _engine(box, prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    corr, md = st.push_only(box.dt)
    eng.interp_push(box.dt, 1)
    _compare_step(eng, box, st, corr, md, prec)
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_crowded_bricks_split_into_interleaved_items(prec):
    """A brick half holding more than one work item's worth of particles
    (4096) is pushed as interleaved items (item t of m takes every m-th
    particle); one push still equals the oracle's.  The thermal recipe with
    12,000 of its particles moved into the 32 cells of one half brick."""
    box = tilt_B(wl.periodic_thermal_2d(nx=32, ny=16, ppc=40, dv_amp=0.3, seed=15), 15)
    rng = np.random.default_rng(15)
    k = rng.choice(box.np, 12000, replace=False)
    box.cell[k] = (rng.integers(0, 8, k.size) + 32 * rng.integers(0, 4, k.size)).astype(np.int32)
    x, y = box.cell % 32, box.cell // 32
    half = (x // 8) * 4 + (y // 8) * 2 + (y % 8) // 4
    assert np.bincount(half).max() > 3 * 4096   # at least four items in that half
    eng = _engine(box, prec)
    _, _, xs, vs = sorted_oracle_state(box)
    st = orc.State(box, xs, vs)
    corr, md = st.push_only(box.dt)
    eng.interp_push(box.dt, 1)
    _compare_step(eng, box, st, corr, md, prec)
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_steps_without_sorting_use_the_global_path(prec):
    """Eight pushes with no sort and no feedback: particles drift out of their
    bricks (up to ~3 cells) and take the global-memory path; the corrector
    accumulated over the eight pushes, the last moments and the particle
    states still equal the oracle's."""
    box = tilt_B(wl.periodic_thermal_2d(nx=33, ny=17, ppc=5, dv_amp=0.3, seed=5), 5)
    eng = _engine(box, prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    E = st.fields()
    corr = np.zeros((4, box.ncell))
    md = np.zeros((4, box.ncell))
    for _ in range(8):
        md[:] = 0.0
        orc.push(st.g, st.p, box.dt, st.x, st.v, E, st.B, corr, md)
        eng.interp_push(box.dt, 1)
    _compare_step(eng, box, st, corr, md, prec, tol_pos=1e-4)
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_subcycling_accumulates_the_corrector(prec):
    box = tilt_B(wl.alfvenic_beam_3d(n=10, ppc=5, nmodes=8, seed=6), 6)
    eng = _engine(box, prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    E = st.fields()
    corr = np.zeros((4, box.ncell))
    md = np.zeros((4, box.ncell))
    for s in range(3):
        md[:] = 0.0
        orc.push(st.g, st.p, box.dt, st.x, st.v, E, st.B, corr, md)
    eng.interp_push(box.dt, 3)
    _compare_step(eng, box, st, corr, md, prec, tol_pos=4e-5)
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_subcycle_resorting_changes_nothing_but_the_order(prec):
    """Five sub-steps with a re-sort after every second one: the same
    deposits bit for bit and the same particle states (as a set) as five
    sub-steps without."""
    box = tilt_B(wl.alfvenic_beam_3d(n=10, ppc=6, nmodes=8, seed=16), 16)
    outs = []
    for every in (0, 2):
        eng = _engine(box, prec)
        eng.set_subcycle_sort(every)
        eng.interp_push(box.dt, 5)
        dep = (eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy())
        if prec == MIXED:
            rows = mixed_rows(eng)
        else:
            rows = np.vstack([eng.x.cpu().numpy(), eng.p64.cpu().numpy()])
        rows = rows[:, np.lexsort(rows[::-1])]
        outs.append((dep[0], dep[1], rows, eng.status()))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    with pytest.raises(m.MhdpicError):
        eng = _engine(box, prec)
        try:
            eng.set_subcycle_sort(-1)
        finally:
            eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_results_do_not_depend_on_the_sort_cadence(prec):
    """Four steps with a sort after every step, or with none: identical
    corrector, moments and gas bit for bit, and the same particles as a set."""
    box = tilt_B(wl.alfvenic_beam_3d(n=12, ppc=7, nmodes=8, seed=17), 17)
    box.hall = 1
    outs = []
    for sort in (True, False):
        eng = _engine(box, prec)
        for _ in range(4):
            eng.interp_push(box.dt, 1)
            eng.apply_feedback()
            if sort:
                eng.sort()
        if prec == MIXED:
            rows = mixed_rows(eng)
        else:
            rows = np.vstack([eng.x.cpu().numpy(), eng.p64.cpu().numpy()])
        rows = rows[:, np.lexsort(rows[::-1])]
        outs.append((eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy(), eng.mom.cpu().numpy(),
                     eng.egas.cpu().numpy(), rows, eng.status()))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_multi_step_with_feedback(prec):
    """Ten full steps (push, feedback, restaging, sort every 2 steps) against
    the oracle; totals conserved."""
    box = tilt_B(wl.periodic_thermal_2d(nx=20, ny=16, ppc=8, dv_amp=0.5, seed=7), 7)
    box.hall = 1
    box.m_cr = 0.02
    eng = _engine(box, prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    t0 = eng.apply_feedback(totals=True)[0]
    o0 = st.totals()
    np.testing.assert_allclose(t0, o0, rtol=1e-12 if prec == FP64 else 1e-6, atol=1e-9)
    for k in range(10):
        st.step(box.dt)
        eng.interp_push(box.dt, 1)
        tg = eng.apply_feedback(totals=True)[0]
        if k % 2 == 1:
            eng.sort()
    to = st.totals()
    mom_scale = np.abs(st.mom).sum() + box.m_cr * np.abs(st.v).sum()
    e_scale = abs(to[3]) + abs(to[7])
    tol = 1e-11 if prec == FP64 else 2e-5
    assert np.abs(tg[4:7] - to[4:7]).max() < tol * mom_scale
    assert abs(tg[7] - to[7]) < tol * e_scale
    # gas state
    gm = eng.mom.cpu().numpy()
    assert rel_l2(gm, st.mom) < (1e-12 if prec == FP64 else 1e-6)
    # conservation of the GPU's own totals
    P0, P1 = t0[0:3] + t0[4:7], tg[0:3] + tg[4:7]
    assert np.abs(P1 - P0).max() < (1e-12 if prec == FP64 else 1e-6) * mom_scale
    E0, E1 = t0[3] + t0[7], tg[3] + tg[7]
    assert abs(E1 - E0) < (1e-12 if prec == FP64 else 1e-6) * e_scale
    assert eng.status() == 0
    eng.close()


def test_deposits_are_bit_identical_run_to_run():
    box = tilt_B(wl.alfvenic_beam_3d(n=12, ppc=8, nmodes=8, seed=8), 8)
    outs = []
    for _ in range(2):
        eng = _engine(box, MIXED)
        eng.interp_push(box.dt, 1)
        outs.append((eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy(), mixed_rows(eng)))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_host_buffers_give_identical_results(prec):
    box = tilt_B(wl.periodic_thermal_2d(nx=18, ny=14, ppc=6, dv_amp=0.3, seed=10), 10)
    res = []
    for mem in (m.MHDPIC_MEM_DEVICE, m.MHDPIC_MEM_HOST, m.MHDPIC_MEM_HOST_GAS):
        eng = _engine(box, prec, memory=mem)
        eng.interp_push(box.dt, 1)
        eng.apply_feedback()
        eng.sort()
        eng.interp_push(box.dt, 1)
        t = eng.apply_feedback(totals=True)
        eng.synchronize()
        parts = momenta_of(eng)
        res.append((t, parts, eng.mom.cpu().numpy()))
        eng.close()
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("between", ["nothing", "sort"])
def test_host_gas_upload_beside_the_push_changes_nothing(between):
    """With the gas in host memory, a feedback that follows a push uploads
    the gas on a second stream while the push runs; several steps of it (and
    of the in-order upload, when a sort comes between) give what device
    buffers give, bit for bit."""
    box = tilt_B(wl.periodic_thermal_2d(nx=20, ny=16, ppc=6, dv_amp=0.3, seed=14), 14)
    res = []
    for mem in (m.MHDPIC_MEM_DEVICE, m.MHDPIC_MEM_HOST_GAS):
        eng = _engine(box, MIXED, memory=mem)
        for step in range(5):
            eng.interp_push(box.dt, 1)
            if between == "sort" and step % 2 == 0:
                eng.sort()
            eng.apply_feedback()
        eng.run(box.dt, 4, 2)
        eng.sync_particles()
        eng.synchronize()
        res.append((mixed_rows(eng), eng.mom.cpu().numpy(), eng.egas.cpu().numpy()))
        assert eng.status() == 0
        eng.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_ensemble_of_boxes_with_an_empty_one():
    boxes = wl.ensemble_2d(nbox=5, seed0=11, max_side=40)
    boxes[2].cell = boxes[2].cell[:0]
    boxes[2].off = np.ascontiguousarray(boxes[2].off[:, :0])
    boxes[2].p = np.ascontiguousarray(boxes[2].p[:, :0])
    for b in boxes:
        tilt_B(b, 12, amp=0.05)
    dt = min(b.dt for b in boxes)
    for prec in (MIXED, FP64):
        eng = m.Engine(boxes, precision=prec)
        eng.interp_push(dt, 1)
        gc = eng.deposits(0).cpu().numpy()
        gm = eng.deposits(1).cpu().numpy()
        c0 = 0
        for b in boxes:
            _, _, x, v = sorted_oracle_state(b)
            st = orc.State(b, x, v)
            corr, md = st.push_only(dt)
            sl = slice(c0, c0 + b.ncell)
            for q in range(4):
                if b.np:
                    assert rel_l2(gc[q, sl], corr[q]) < TOL[prec]
                    assert rel_l2(gm[q, sl], md[q]) < TOL[prec]
                else:
                    assert not gc[q, sl].any() and not gm[q, sl].any()
            c0 += b.ncell
        assert eng.status() == 0
        eng.close()


@pytest.mark.parametrize("n,ndim", [((3, 5, 1), 2), ((3, 3, 3), 3), ((13, 11, 1), 2)])
def test_boxes_smaller_than_a_tile_and_ragged_bricks(n, ndim):
    if ndim == 2:
        box = tilt_B(wl.periodic_thermal_2d(nx=n[0], ny=n[1], ppc=7, dv_amp=0.3, seed=13), 13)
    else:
        box = tilt_B(wl.alfvenic_beam_3d(n=3, ppc=7, nmodes=4, seed=13), 13)
    for prec in (MIXED, FP64):
        eng = _engine(box, prec)
        _, _, x, v = sorted_oracle_state(box)
        st = orc.State(box, x, v)
        corr, md = st.push_only(box.dt)
        eng.interp_push(box.dt, 1)
        _compare_step(eng, box, st, corr, md, prec)
        eng.close()


def test_gyration_phase_exact_on_gpu_fp64():
    """App. B.1, v0 = 0, through the FP64 library path: phase 2 atan(Omega dt/2)
    per step and |v| conserved."""
    box = wl.gyration()
    eng = _engine(box, FP64)
    v0 = eng.p64.cpu().numpy()[:, 0].copy()
    gam = math.sqrt(1.0 + v0 @ v0 / box.C ** 2)
    om = 1.0 / gam
    for _ in range(50):
        eng.interp_push(box.dt, 1)
    v = eng.p64.cpu().numpy()[:, 0]
    phase = math.atan2(v[2], v[1]) - math.atan2(v0[2], v0[1])
    expect = -50 * 2.0 * math.atan(om * box.dt / 2.0)
    assert abs(math.remainder(phase - expect, 2 * math.pi)) < 1e-12
    assert abs(np.linalg.norm(v) - np.linalg.norm(v0)) < 1e-13 * np.linalg.norm(v0)
    eng.close()


def test_fast_mover_sets_a_status_flag_without_faulting():
    box = wl.periodic_thermal_2d(nx=16, ny=16, ppc=2, seed=14)
    eng = _engine(box, MIXED)
    eng.interp_push(box.dt * 40.0, 1)     # particles cross many cells per half step
    flags = eng.status()
    assert flags & 1
    eng.clear_status()
    assert eng.status() == 0
    eng.close()


def test_invalid_calls_are_rejected():
    box = wl.periodic_thermal_2d(nx=8, ny=8, ppc=2, seed=15)
    eng = _engine(box, MIXED)
    with pytest.raises(m.MhdpicError):
        eng.interp_push(-1.0, 1)
    with pytest.raises(m.MhdpicError):
        eng.interp_push(0.1, 0)
    with pytest.raises(m.MhdpicError):
        m.mhdpic_get_deposits(eng.ctx, 5, 0)
    eng.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_graph_replayed_run_equals_eager_steps(k):
    """mhdpic_run replays whole sort cycles from a CUDA graph: the result is
    bit-identical to the same steps issued one call at a time."""
    box = tilt_B(wl.alfvenic_beam_3d(n=12, ppc=6, nmodes=8, seed=40), 40)
    stream = torch.cuda.Stream()
    outs = []
    for mode in ("eager", "graph"):
        eng = m.Engine([box], precision=MIXED, stream=stream)
        nsteps = 2 * k * 2 + 1
        if mode == "eager":
            for s in range(nsteps):
                eng.step(box.dt)
                if (s + 1) % k == 0:
                    eng.sort()
        else:
            eng.run(box.dt, nsteps, k)
        stream.synchronize()
        outs.append((mixed_rows(eng), eng.mom.cpu().numpy(), eng.deposits(1).cpu().numpy(),
                     eng.fields().cpu().numpy()))
        assert eng.status() == 0
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("k", [1, 3])
def test_run_sorts_look_ahead_over_the_whole_cycle(k):
    """With a look-ahead t set, mhdpic_run's sorts every k steps look k t
    ahead: its steps equal, bit for bit and in the same particle order, eager
    steps sorted by mhdpic_sort with a look-ahead of k t."""
    box = tilt_B(wl.alfvenic_beam_3d(n=12, ppc=6, nmodes=8, seed=46), 46)
    stream = torch.cuda.Stream()
    t = 0.5 * box.dt
    outs = []
    for mode in ("eager", "graph"):
        eng = m.Engine([box], precision=MIXED, stream=stream)
        nsteps = 2 * k * 2 + 1
        if mode == "eager":
            eng.set_sort_lookahead(k * t)
            for s in range(nsteps):
                eng.step(box.dt)
                if (s + 1) % k == 0:
                    eng.sort()
        else:
            eng.set_sort_lookahead(t)
            eng.run(box.dt, nsteps, k)
        stream.synchronize()
        outs.append((mixed_rows(eng), eng.mom.cpu().numpy(), eng.deposits(1).cpu().numpy(),
                     eng.fields().cpu().numpy()))
        assert eng.status() == 0
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("fail_at", [1, 2, 5])
def test_failed_graph_capture_leaves_the_context_as_it_was(fail_at):
    """A launch failure injected on the host inside the graph capture of
    mhdpic_run (nothing captured runs): the call reports the error, the
    context keeps the state it had before the capture, and the steps issued
    afterwards are bit-identical to those of a context that never failed."""
    box = tilt_B(wl.alfvenic_beam_3d(n=12, ppc=6, nmodes=8, seed=43), 43)
    stream = torch.cuda.Stream()
    outs = []
    for mode in ("clean", "failed"):
        eng = m.Engine([box], precision=MIXED, stream=stream)
        eng.run(box.dt, 1, 1)           # one eager step, ending on a pending sort
        if mode == "failed":
            m.mhdpic_debug_fail_launch(eng.ctx, fail_at)
            with pytest.raises(m.MhdpicError, match="failure injected"):
                eng.run(box.dt, 2, 1)   # the capture of a two-step cycle (at least 6 launches) fails
            m.mhdpic_debug_fail_launch(eng.ctx, 0)
        for s in range(3):
            eng.step(box.dt)
            eng.sort()
        stream.synchronize()
        outs.append((mixed_rows(eng), eng.mom.cpu().numpy(), eng.deposits(1).cpu().numpy(),
                     eng.fields().cpu().numpy()))
        assert eng.status() == 0
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_run_tunes_the_sort_cadence():
    box = wl.periodic_thermal_2d(nx=48, ny=40, ppc=8, seed=41)
    stream = torch.cuda.Stream()
    eng = m.Engine([box], precision=MIXED, stream=stream)
    assert eng.sort_cadence() == 0
    eng.run(box.dt, 16, 0)
    assert eng.sort_cadence() in (1, 2, 3, 4)
    t = eng.apply_feedback(totals=True)[0]
    assert np.all(np.isfinite(t)) and eng.status() == 0
    eng.close()


def test_mixed_conservation_over_1000_steps():
    """Total gas + CR momentum and energy drift by <= 1e-6 over 1000 mixed
    steps (graph-replayed, sort every 2 steps), with a substantial CR share."""
    box = tilt_B(wl.periodic_thermal_2d(nx=32, ny=24, ppc=8, dv_amp=0.5, seed=42), 42)
    box.hall = 1
    box.m_cr = 0.05
    stream = torch.cuda.Stream()
    eng = m.Engine([box], precision=MIXED, stream=stream)
    t0 = eng.apply_feedback(totals=True)[0]
    eng.run(box.dt, 1000, 2)
    t1 = eng.apply_feedback(totals=True)[0]
    assert eng.status() == 0
    mom = eng.mom.cpu().numpy()
    scaleP = np.abs(mom).sum() + box.m_cr * np.abs(eng.p.cpu().numpy().astype(np.float64)).sum()
    dP = np.abs((t1[0:3] + t1[4:7]) - (t0[0:3] + t0[4:7])).max()
    dE = abs((t1[3] + t1[7]) - (t0[3] + t0[7]))
    assert dP <= 1e-6 * scaleP, (dP / scaleP)
    assert dE <= 1e-6 * abs(t0[3] + t0[7]), (dE / abs(t0[3] + t0[7]))
    # the CR and gas shares really exchanged momentum and energy
    assert np.abs(t1[4:7] - t0[4:7]).max() > 1e-3 * box.m_cr * box.np
    eng.close()


def test_mixed_conservation_of_the_3d_beam_over_1000_steps():
    """The benchmark's 3-D Alfvenic-beam recipe at 64^3 x 32 CRs (8,388,608),
    graph-replayed with a sort every step: total gas + CR momentum along every
    axis and the total energy drift by <= 1e-6 over 1000 mixed steps (App.
    A.3: the corrector's exchange is exact).  The beam (|v| ~ 100 along B)
    hands momentum to the gas every step, which a one-word FP32 four-velocity
    could not hold to this bound; the two-word record does."""
    box = wl.alfvenic_beam_3d(n=64, ppc=32, seed=44)
    stream = torch.cuda.Stream()
    eng = m.Engine([box], precision=MIXED, stream=stream)
    t0 = eng.apply_feedback(totals=True)[0]
    eng.run(box.dt, 1000, 1)
    t1 = eng.apply_feedback(totals=True)[0]
    assert eng.status() == 0
    scaleP = np.abs(eng.mom.cpu().numpy()).sum() + box.m_cr * np.abs(momenta_of(eng)).sum()
    dP = np.abs((t1[0:3] + t1[4:7]) - (t0[0:3] + t0[4:7]))
    dE = abs((t1[3] + t1[7]) - (t0[3] + t0[7])) / abs(t0[3] + t0[7])
    assert np.all(dP <= 1e-6 * scaleP), dP / scaleP
    assert dE <= 1e-6, dE
    # the beam really gave the gas momentum along B over the run
    assert abs(t1[4] - t0[4]) > 1e3 * dP[0]
    eng.close()


def test_full_size_bench_configuration_sampled():
    """The bench's workload and launch configuration (128^3 x 32 = 67,108,864
    CRs, mixed): 4096 sampled particles after one push match the oracle's push
    of the same particles in the same fields, the charge deposit sums to
    (q/mc) m N / dV, and the corrector momentum equals minus the particles'
    momentum change."""
    box = wl.alfvenic_beam_3d()          # the bench workload, seed 0
    eng = m.Engine([box], precision=MIXED)
    rng = np.random.default_rng(43)
    idx = np.sort(rng.choice(box.np, 4096, replace=False))
    cell0 = eng.cell.cpu().numpy()
    off0 = eng.off.cpu().numpy()
    p0 = momenta_of(eng)
    eng.interp_push(box.dt, 1)
    cell1 = eng.cell.cpu().numpy()
    off1 = eng.off.cpu().numpy()
    p1 = momenta_of(eng)
    corr = eng.deposits(0).cpu().numpy()
    mdep = eng.deposits(1).cpu().numpy()
    assert eng.status() == 0
    eng.close()
    # oracle push of the sampled particles (fields from the same gas)
    n = box.n[0]

    def absx(cell, off, sel):
        c = cell[sel].astype(np.int64)
        co = [c % n, (c // n) % n, c // (n * n)]
        return np.stack([co[d] + off[d, sel].astype(np.float64) for d in range(3)])

    g, p = orc.grid_of(box), orc.params_of(box)
    E = orc.field_prep(g, p, box.rho, box.mom, box.B, np.zeros((4, box.ncell)))
    x = np.ascontiguousarray(absx(cell0, off0, idx))
    v = np.ascontiguousarray(p0[:, idx].astype(np.float64))
    orc.push(g, p, box.dt, x, v, E, box.B, None, None)
    xg = absx(cell1, off1, idx)
    dx = periodic_diff(xg, x, float(n))
    assert np.abs(dx).max() < 1e-5
    vg = p1[:, idx].astype(np.float64)
    assert np.all(np.abs(vg - v) <= 1e-5 * np.sqrt((v ** 2).sum(0)))
    # whole-grid invariants
    qn = box.qm_cr * box.m_cr
    # each particle's three f32 TSC weights per dimension sum to 1 within a few
    # ulps, so the total charge agrees to f32 precision
    assert abs(mdep[0].sum() - qn * box.np) < 1e-6 * qn * box.np
    # the two-word four-velocities change by exactly what the corrector
    # deposits, up to one rounding at 2^-35 of |v| per particle and the
    # fixed-point quantisation of the deposit
    dpart = box.m_cr * (p1 - p0).sum(axis=1)
    gross = box.m_cr * np.abs(p1 - p0).sum(axis=1)
    assert np.all(np.abs(corr[:3].sum(axis=1) + dpart) <= 1e-9 * gross), (corr[:3].sum(axis=1) + dpart) / gross


# --- a sort applied by the next push -------------------------------------------

def _lazy_box(name):
    if name == "thermal2d":
        return tilt_B(wl.periodic_thermal_2d(nx=40, ny=36, ppc=12, dv_amp=0.6, seed=21), 21)
    return wl.alfvenic_beam_3d(seed=22, n=12, ppc=9)


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("name", ["thermal2d", "beam3d"])
def test_sort_applied_by_the_push_matches_sort_applied_at_once(prec, name):
    """The push that reads its particles through a pending permutation leaves
    the same particles, in the same order, and the same deposits, as a sort
    whose permutation was applied before the push."""
    box = _lazy_box(name)
    outs = []
    for at_once in (False, True):
        eng = _engine(box, prec)
        for _ in range(3):
            eng.interp_push(box.dt, 1)
            eng.apply_feedback()
            eng.sort()
            if at_once:
                eng.sync_particles()
        eng.interp_push(box.dt, 2)   # the first sub-step applies the sort
        t = eng.apply_feedback(totals=True)
        dep = (eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy())
        outs.append((momenta_of(eng), positions_of(eng), dep[0], dep[1], t, eng.status()))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_repeated_sorts_and_the_permutation_seen_by_the_caller():
    """A second sort supersedes a pending one; a permutation asked for is
    relative to the order the caller saw, so after a sort it is the identity."""
    box = _lazy_box("thermal2d")
    eng = _engine(box, MIXED)
    eng.interp_push(box.dt, 1)
    eng.apply_feedback()
    ref = _engine(box, MIXED)
    ref.interp_push(box.dt, 1)
    ref.apply_feedback()
    eng.sort()
    eng.sort()
    ref.sort()
    perm, _ = eng.sort(want_perm=True)
    np.testing.assert_array_equal(perm.cpu().numpy(), np.arange(box.np))
    for e in (eng, ref):
        e.interp_push(box.dt, 1)
    np.testing.assert_array_equal(mixed_rows(eng), mixed_rows(ref))
    np.testing.assert_array_equal(eng.deposits(1).cpu().numpy(), ref.deposits(1).cpu().numpy())
    eng.close()
    ref.close()


# --- the standalone charge/current deposit ------------------------------------

@pytest.mark.parametrize("name", ["thermal2d", "beam3d"])
def test_standalone_deposit_reproduces_the_push_moments_bit_for_bit(name):
    """mhdpic_deposit at the positions a push left gives the integers the
    push deposited there: right after the push (the call sorts), with a sort
    pending, and after three pushes without a sort (particles out of their
    bricks take the global path in both)."""
    box = _lazy_box(name)
    eng = _engine(box, MIXED)
    dt = box.dt
    eng.interp_push(dt, 1)
    eng.apply_feedback()
    for case in ("after push", "sort pending", "unsorted"):
        if case == "sort pending":
            eng.interp_push(dt, 1)
            eng.apply_feedback()
            eng.sort()
        elif case == "unsorted":
            for _ in range(3):
                eng.interp_push(dt, 1)
                eng.apply_feedback()
        md_push = eng.deposits(1).cpu().numpy().copy()
        eng.deposit()
        md_dep = eng.deposits(1).cpu().numpy()
        np.testing.assert_array_equal(md_dep, md_push, err_msg=case)
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("name", ["thermal2d", "beam3d"])
def test_standalone_deposit_matches_oracle(prec, name):
    """After two steps and a sort, mhdpic_deposit against the oracle's
    deposit at the engine's positions; the particle state is unchanged."""
    box = _lazy_box(name)
    eng = _engine(box, prec)
    dt = box.dt
    for _ in range(2):
        eng.interp_push(dt, 1)
        eng.apply_feedback()
    eng.sort()
    x, v = positions_of(eng).copy(), momenta_of(eng).copy()
    eng.deposit()
    np.testing.assert_array_equal(positions_of(eng), x)
    np.testing.assert_array_equal(momenta_of(eng), v)
    md = orc.deposit_moments(orc.grid_of(box), orc.params_of(box), np.ascontiguousarray(x),
                             np.ascontiguousarray(v), box.ncell)
    gm = eng.deposits(1).cpu().numpy()
    for q in range(4):
        assert rel_l2(gm[q], md[q]) < TOL[prec], q
    assert eng.status() == 0
    eng.close()


def test_standalone_deposit_with_host_buffers_and_open_face():
    """Host-memory buffers and removed particles: the deposit skips particles
    that left and leaves the caller's arrays as they were."""
    box = wl.shock_front_2d(nx=96, ny=8, ppc=6.0, front=0.4, seed=9)
    eng = m.Engine([box], precision=MIXED, memory=m.MHDPIC_MEM_HOST)
    for _ in range(3):
        eng.interp_push(3.0 * box.dt, 1)
        eng.apply_feedback()
    cell = eng.cell.cpu().numpy().copy()
    x = positions_of(eng)
    v = momenta_of(eng)
    eng.deposit()
    np.testing.assert_array_equal(eng.cell.cpu().numpy(), cell)
    live = cell >= 0
    md = orc.deposit_moments(orc.grid_of(box), orc.params_of(box), np.ascontiguousarray(x[:, live]),
                             np.ascontiguousarray(v[:, live]), box.ncell)
    gm = eng.deposits(1).cpu().numpy()
    for q in range(4):
        assert rel_l2(gm[q], md[q]) < TOL[MIXED], q
    assert eng.status() == 0
    eng.close()


# --- degenerate inputs ------------------------------------------------------------

@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_field_free_box_streams_particles_freely(prec):
    """B = 0: no force, so the four-velocities come back bit for bit, the
    corrector deposit is exactly zero and the positions follow the oracle's
    free streaming."""
    box = wl.periodic_thermal_2d(nx=20, ny=18, ppc=6, dv_amp=0.5, seed=6)
    box.B = np.zeros_like(box.B)
    box.hall = 1
    eng = _engine(box, prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    v_before = momenta_of(eng).copy()
    corr, md = st.push_only(box.dt)
    eng.interp_push(box.dt, 1)
    np.testing.assert_array_equal(momenta_of(eng), v_before)
    assert np.all(eng.deposits(0).cpu().numpy() == 0.0)
    _compare_step(eng, box, st, corr, md, prec)
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_context_without_particles(prec):
    """A box with no particles at all goes through every call: zero moments,
    zero corrector, the gas totals unchanged, an empty spectrum."""
    box = wl.periodic_thermal_2d(nx=16, ny=16, ppc=2, seed=7)
    box.cell = box.cell[:0]
    box.off = np.ascontiguousarray(box.off[:, :0])
    box.p = np.ascontiguousarray(box.p[:, :0])
    eng = _engine(box, prec)
    t0 = eng.apply_feedback(totals=True)[0]
    for _ in range(3):
        eng.interp_push(box.dt, 1)
        eng.apply_feedback()
        eng.sort()
    eng.deposit()
    eng.run(box.dt, 6, 2)
    t1 = eng.apply_feedback(totals=True)[0]
    np.testing.assert_array_equal(t1, t0)
    assert not t1[4:].any()
    assert not eng.deposits(0).cpu().numpy().any() and not eng.deposits(1).cpu().numpy().any()
    counts, _ = eng.spectrum(m.MHDPIC_SPEC_ENERGY, np.array([0.0, 1.0, 10.0]))
    assert int(np.asarray(counts).sum()) == 0
    assert eng.live_particles() == 0
    assert eng.status() == 0
    eng.close()


def test_standalone_deposit_then_graph_replay_changes_nothing():
    """A standalone deposit leaves a sort pending; graph-replayed steps from
    there give the same particles (as a set) and the same deposits, bit for
    bit, as the same steps without it."""
    box = _lazy_box("beam3d")
    dt = box.dt
    outs = []
    for with_deposit in (False, True):
        stream = torch.cuda.Stream()
        eng = m.Engine([box], precision=MIXED, stream=stream)
        if with_deposit:
            eng.deposit()
        eng.run(dt, 8, 2)
        rows = np.vstack([positions_of(eng), momenta_of(eng)])
        rows = rows[:, np.lexsort(rows[::-1])]
        outs.append((rows, eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy(), eng.mom.cpu().numpy()))
        assert eng.status() == 0
        eng.close()
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
