"""Open inflow face, front tracking and CR injection on the GPU (Section 5)
against the FP64 oracle, through the C ABI.

Tolerances: FP64 path 1e-12 relative, mixed path 1e-5 (particles compared as
sets, since the sort orders them); counts exact.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl
from tests._parity import momenta_of, positions_of, rel_l2, sorted_oracle_state, tilt_B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402

MIXED, FP64 = m.MHDPIC_PREC_MIXED, m.MHDPIC_PREC_FP64
TOL = {FP64: 1e-12, MIXED: 1e-5}


def _live_rows_gpu(eng):
    x = positions_of(eng)
    v = momenta_of(eng)
    if eng.x is not None:
        live = ~np.isnan(eng.x.cpu().numpy()[0])
    else:
        live = eng.cell.cpu().numpy() >= 0
    rows = np.vstack([x[:, live], v[:, live]])
    return rows[:, np.lexsort(rows[::-1])]


def _live_rows_oracle(x, v):
    live = ~np.isnan(x[0])
    rows = np.vstack([x[:, live], v[:, live]])
    return rows[:, np.lexsort(rows[::-1])]


def _box(seed=1):
    box = wl.shock_front_2d(nx=128, ny=8, ppc=6.0, front=0.4, seed=seed)
    return tilt_B(box, seed, amp=0.05)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_particles_leave_through_the_open_face_as_the_oracle_says(prec):
    box = _box()
    eng = m.Engine([box], precision=prec)
    _, _, x, v = sorted_oracle_state(box)
    st = orc.State(box, x, v)
    dt = 3.0 * box.dt
    n0 = eng.live_particles()
    assert n0 == int((box.cell >= 0).sum())
    for s in range(6):
        st.step(dt)
        eng.interp_push(dt, 1)
        eng.apply_feedback()
        if s % 2 == 1:
            eng.sort()
    live_o = int((~np.isnan(st.x[0])).sum())
    assert live_o < n0                      # some left
    if prec == FP64:
        assert eng.live_particles() == live_o
        a, b = _live_rows_gpu(eng), _live_rows_oracle(st.x, st.v)
        assert a.shape == b.shape
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    else:
        # a particle within f32 rounding of the face may go the other way
        assert abs(eng.live_particles() - live_o) <= 2
    gm = eng.mom.cpu().numpy()
    for q in range(3):
        assert rel_l2(gm[q] - box.mom[q], st.mom[q] - box.mom[q], floor=1e-300) < TOL[prec] * 10, q
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_injection_matches_the_oracle(prec):
    box = _box(seed=2)
    eng = m.Engine([box], precision=prec)
    g, p = orc.grid_of(box), orc.params_of(box)
    rho, mom, egas = box.rho.copy(), box.mom.copy(), box.egas.copy()
    x0 = wl.absolute_positions(box)
    v0 = box.p.astype(np.float64)
    live0 = ~np.isnan(x0[0])
    free = int((~live0).sum())
    eta, fE, seed = 0.05, 10.0, 1234
    carry = 0.0
    xs_prev = np.nan
    rows_o = [np.vstack([x0[:, live0], v0[:, live0]])]
    for call in range(2):
        fr = orc.front(g, rho, mom, egas, box.B)
        xn, vn, carry = orc.inject(g, p, fr, xs_prev, box.dt, eta, fE, seed, call, carry, free, rho, mom, egas)
        free -= xn.shape[1]
        xs_prev = fr[0]
        n, xs, xt = eng.inject(box.dt, eta, fE, 5.0 / 3.0, seed)
        assert n == xn.shape[1] and n > 0
        assert abs(xs - fr[0]) <= 1e-12 * abs(fr[0]) and xt == fr[1]
        rows_o.append(np.vstack([xn, vn]))
    # every particle, old and injected, as a set
    ro = np.concatenate(rows_o, axis=1)
    ro = ro[:, np.lexsort(ro[::-1])]
    rg = _live_rows_gpu(eng)
    assert rg.shape == ro.shape
    if prec == FP64:
        np.testing.assert_allclose(rg, ro, rtol=1e-12, atol=1e-12)
    else:
        scale = np.abs(ro).max(axis=1, keepdims=True)
        assert np.all(np.abs(rg - ro) <= 1e-6 * scale)
    # the gas gave what the particles took
    tol = 1e-12 if prec == FP64 else 1e-6
    np.testing.assert_allclose(eng.rho.cpu().numpy(), rho, rtol=tol)
    for q in range(3):
        d_g = eng.mom.cpu().numpy()[q] - box.mom[q]
        d_o = mom[q] - box.mom[q]
        assert rel_l2(d_g, d_o, floor=1e-300) < tol, q
    assert rel_l2(eng.egas.cpu().numpy() - box.egas, egas - box.egas, floor=1e-300) < tol
    assert eng.live_particles() == int(live0.sum()) + sum(r.shape[1] for r in rows_o[1:])
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_injection_conserves_gas_plus_cr_momentum_and_energy(prec):
    box = _box(seed=3)
    eng = m.Engine([box], precision=prec)
    t0 = eng.apply_feedback(totals=True)[0]
    for _ in range(3):
        n, _, _ = eng.inject(box.dt, 0.05, 10.0, 5.0 / 3.0, 7)
        assert n > 0
    t1 = eng.apply_feedback(totals=True)[0]
    scale = np.abs(t0).max() + np.abs(t1[4:]).max()
    assert np.abs((t1[:3] + t1[4:7]) - (t0[:3] + t0[4:7])).max() < 1e-12 * scale
    assert abs((t1[3] + t1[7]) - (t0[3] + t0[7])) < 1e-12 * scale
    # and the injected particles push on like the others
    for _ in range(3):
        eng.interp_push(box.dt, 1)
        eng.apply_feedback()
        eng.sort()
    assert eng.status() == 0
    eng.close()


def test_injection_stops_at_the_free_slots_and_is_checked():
    box = _box(seed=4)
    eng = m.Engine([box], precision=MIXED)
    free = int((box.cell < 0).sum())
    n, _, _ = eng.inject(box.dt, 1e4, 10.0, 5.0 / 3.0, 1)
    assert n == free
    assert eng.live_particles() == box.np
    assert m.status_names(eng.status()) == ["INJECT_CAP"]
    with pytest.raises(m.MhdpicError):
        eng.inject(-1.0, 0.1)
    eng.close()
    per = wl.periodic_thermal_2d(nx=16, ny=16, ppc=2, seed=1)
    eng = m.Engine([per], precision=MIXED)
    with pytest.raises(m.MhdpicError):
        eng.inject(per.dt, 0.1)
    eng.close()


def _pow2_dt(box):
    """A step that is a power of two (clock sums exact) within the box's limit."""
    return 2.0 ** math.floor(math.log2(box.dt))


def _early_times(n, dt, seed):
    """Distinct injection times: half early-ish in [0, 3 dt), half late."""
    rng = np.random.default_rng(seed)
    t = np.where(rng.random(n) < 0.5, rng.uniform(0.0, 3.0 * dt, n), rng.uniform(1e3, 2e3, n))
    return np.ascontiguousarray(t)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_early_particles_are_removed_at_twice_their_injection_time(prec):
    """Section 5's removal (t_i < t_early goes at t = 2 t_i) on the GPU against
    the oracle: the same particles go (identified by their distinct t_i), the
    survivors' states, the moments of the survivors and the gas match."""
    box = _box(seed=5)
    dt = _pow2_dt(box)
    t_early = 2.5 * dt
    eng = m.Engine([box], precision=prec)
    _, _, x, v = sorted_oracle_state(box)
    t_inj = _early_times(box.np, dt, 5)
    eng.set_injection_times(t_inj, 0.0, t_early)
    st = orc.State(box, x, v)
    t = 0.0
    removed = 0
    for s in range(6):
        corr, _ = st.push_only(dt)
        t += dt
        removed += orc.remove_early(st.x, st.v, t_inj, t, t_early)
        st.mom_dep = orc.deposit_moments(st.g, st.p, st.x, st.v, st.nc)
        orc.apply_feedback(st.g, st.mom, st.egas, corr)
        eng.interp_push(dt, 1)
        eng.apply_feedback()
        if s % 2 == 1:
            eng.sort()
    assert removed > 0
    tg, clock = eng.injection_times()
    assert clock == t
    live_g = (~np.isnan(eng.x.cpu().numpy()[0])) if prec == FP64 else eng.cell.cpu().numpy() >= 0
    live_o = ~np.isnan(st.x[0])
    set_g, set_o = set(tg[live_g].tolist()), set(t_inj[live_o].tolist())
    early_gone = set(t_inj[(t_inj < t_early) & (2.0 * t_inj <= t)].tolist())
    assert not early_gone & set_g
    if prec == FP64:
        assert set_g == set_o
        rg = np.vstack([positions_of(eng)[:, live_g], momenta_of(eng)[:, live_g], tg[live_g]])
        ro = np.vstack([st.x[:, live_o], st.v[:, live_o], t_inj[live_o]])
        rg, ro = rg[:, np.argsort(rg[-1])], ro[:, np.argsort(ro[-1])]
        np.testing.assert_allclose(rg, ro, rtol=1e-12, atol=1e-12)
    else:
        # only a particle within f32 rounding of the open face may differ
        assert len(set_g ^ set_o) <= 2
    md = eng.deposits(1).cpu().numpy()
    for q in range(4):
        assert rel_l2(md[q], st.mom_dep[q], floor=1e-300) < TOL[prec] * 10, q
    gm = eng.mom.cpu().numpy()
    for q in range(3):
        assert rel_l2(gm[q] - box.mom[q], st.mom[q] - box.mom[q], floor=1e-300) < TOL[prec] * 10, q
    assert eng.status() == 0
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_injected_particles_carry_the_clock_and_leave_at_twice_it(prec):
    box = _box(seed=6)
    dt = _pow2_dt(box)
    eng = m.Engine([box], precision=prec)
    n0 = eng.live_particles()
    t0 = 2.0 * dt
    eng.set_injection_times(None, t0, 100.0 * dt)      # the initial particles stay
    n, _, _ = eng.inject(dt, 0.05, 10.0, 5.0 / 3.0, 9)
    assert n > 0
    tg, clock = eng.injection_times()
    assert clock == t0
    assert int((tg == t0).sum()) == n and np.all(np.isinf(tg) | (tg == t0))
    live = [eng.live_particles()]
    for _ in range(3):
        eng.interp_push(dt, 1)
        eng.apply_feedback()
        live.append(eng.live_particles())
    # the injected ones go at the end of the push that reaches 2 t0 = t0 + 2 dt
    # (others may leave through the open face meanwhile)
    assert live[0] == n0 + n
    gone = [live[i] - live[i + 1] for i in range(3)]
    assert gone[1] >= n
    assert gone[0] < n and gone[2] < n
    tg, clock = eng.injection_times()
    assert clock == t0 + 3 * dt
    eng.sort()
    tg, _ = eng.injection_times()
    live_g = (~np.isnan(eng.x.cpu().numpy()[0])) if prec == FP64 else eng.cell.cpu().numpy() >= 0
    assert not np.any(tg[live_g] == t0)
    assert eng.status() == 0
    eng.close()


def test_removal_through_graph_replay_matches_eager_steps_bit_for_bit():
    box = _box(seed=7)
    dt = _pow2_dt(box)
    t_inj = _early_times(box.np, dt, 7)
    outs = []
    for graphs in (False, True):
        eng = m.Engine([box], precision=MIXED)
        eng.set_injection_times(t_inj, 0.0, 2.5 * dt)
        if graphs:
            eng.run(dt, 8, 2)
        else:
            for s in range(8):
                eng.interp_push(dt, 1)
                eng.apply_feedback()
                if s % 2 == 1:
                    eng.sort()
        tg, clock = eng.injection_times()
        live = eng.cell.cpu().numpy() >= 0
        rows = np.vstack([tg[live], positions_of(eng)[:, live], momenta_of(eng)[:, live]])
        md = eng.deposits(1).cpu().numpy()
        outs.append((clock, rows[:, np.argsort(rows[0])], eng.mom.cpu().numpy().copy(), md))
        assert eng.status() == 0
        eng.close()
    (c0, r0, m0, d0), (c1, r1, m1, d1) = outs
    assert c0 == c1 == 8 * dt
    np.testing.assert_array_equal(r0, r1)
    np.testing.assert_array_equal(m0, m1)
    np.testing.assert_array_equal(d0, d1)


def test_injection_times_need_tracking_and_valid_arguments():
    box = _box(seed=8)
    eng = m.Engine([box], precision=MIXED)
    with pytest.raises(m.MhdpicError):
        eng.injection_times()
    with pytest.raises(m.MhdpicError):
        eng.set_injection_times(None, float("nan"), 1.0)
    with pytest.raises(m.MhdpicError):
        eng.set_injection_times(None, 0.0, float("nan"))
    eng.set_injection_times(None, 1.5, float("-inf"))
    tg, clock = eng.injection_times()
    assert clock == 1.5 and np.all(np.isinf(tg))
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
def test_removal_inside_sub_cycled_pushes(prec):
    """Each sub-step advances the clock: four sub-steps in one call remove
    the same particles, at the same clock, as four single pushes in the same
    staged fields (no feedback in between)."""
    box = _box(seed=10)
    dt = _pow2_dt(box)
    t_inj = _early_times(box.np, dt, 10)
    res = []
    for split in (False, True):
        eng = m.Engine([box], precision=prec)
        eng.set_injection_times(t_inj, 0.0, 2.5 * dt)
        if split:
            for _ in range(4):
                eng.interp_push(dt, 1)
        else:
            eng.interp_push(dt, 4)
        tg, clock = eng.injection_times()
        live = (~np.isnan(eng.x.cpu().numpy()[0])) if prec == FP64 else eng.cell.cpu().numpy() >= 0
        rows = np.vstack([tg[live], positions_of(eng)[:, live], momenta_of(eng)[:, live]])
        res.append((clock, rows[:, np.argsort(rows[0])]))
        assert eng.status() == 0
        eng.close()
    (c0, r0), (c1, r1) = res
    assert c0 == c1 == 4 * dt
    np.testing.assert_array_equal(r0[0], r1[0])          # the same particles left
    np.testing.assert_allclose(r0, r1, rtol=0, atol=1e-12 if prec == FP64 else 1e-6)
    gone = (t_inj < 2.5 * dt) & (2.0 * t_inj <= 4 * dt)
    assert gone.any() and not set(t_inj[gone].tolist()) & set(r0[0].tolist())
