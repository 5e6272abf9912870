"""Parity at the benchmark's full sizes (every workload the benchmark times:
the 3-D beam, the 2-D Bell box, the two shock boxes and the 96-box
ensemble), one push in the engine's default launch configuration, on sampled
outputs the oracle computes one by one.

* Sampled particles: 4096 particles per box, read after the engine's initial
  sort, pushed by the oracle in the fields of the same gas (with the CR-Hall
  term from the oracle's own deposit of every particle where the box has it
  on): positions within 1e-5 cells, momenta within 1e-5 relative.
* Sampled cells: the corrector (at x^(n+1/2)) and the charge/current moments
  (at x^(n+1)) of 32 cells per box, against the oracle's push of every
  particle that starts within 3 cells of a sampled cell (a particle moves
  less than a cell per step, so no contributor is missed); relative L2 over
  the sampled cells <= 1e-5 per channel.  The oracle's inputs are the
  generator's arrays, not the engine's.
* Whole grid: the charge deposit sums to (q/mc) m N_live / dV.
"""
import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl
from tests._parity import periodic_diff, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402

TOL = 1e-5
NSAMPLE = 4096
NCELLS = 32
REACH = 3


def _abs_positions(box, cell, off):
    n = box.n
    c = cell.astype(np.int64)
    co = [c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1])]
    return np.stack([box.x0[d] + (co[d] + off[d].astype(np.float64)) * box.dx[d] for d in range(box.ndim)])


def _fields(box):
    g, p = orc.grid_of(box), orc.params_of(box)
    md = np.zeros((4, box.ncell))
    if box.hall:
        x = np.ascontiguousarray(wl.absolute_positions(box))
        v = np.ascontiguousarray(box.p.astype(np.float64))
        md = orc.deposit_moments(g, p, x, v, box.ncell)
    return orc.field_prep(g, p, box.rho, box.mom, box.B, md)


def _check_particles(box, E, dt, before, after, rng):
    cell0, off0, p0 = before
    cell1, off1, p1 = after
    live = np.flatnonzero(cell0 >= 0)
    idx = np.sort(rng.choice(live, min(NSAMPLE, live.size), replace=False))
    g, p = orc.grid_of(box), orc.params_of(box)
    x = np.ascontiguousarray(_abs_positions(box, cell0[idx], off0[:, idx]))
    v = np.ascontiguousarray(p0[:, idx].astype(np.float64))
    orc.push(g, p, dt, x, v, E, box.B, None, None)
    stay = ~np.isnan(x[0])                      # left through an open face
    assert np.array_equal(cell1[idx] >= 0, stay)
    xg = _abs_positions(box, cell1[idx[stay]], off1[:, idx[stay]])
    for d in range(box.ndim):
        L = box.n[d] * box.dx[d]
        dd = periodic_diff(xg[d], x[d, stay], L) if box.bc[d] == 0 else xg[d] - x[d, stay]
        assert np.abs(dd).max() < TOL * box.dx[d], d
    vg = p1[:, idx[stay]].astype(np.float64)
    vo = v[:, stay]
    assert np.all(np.abs(vg - vo) <= TOL * np.sqrt((vo ** 2).sum(0)))


def _check_cells(box, E, dt, corr_g, md_g, rng):
    """Oracle push of every particle within REACH cells of the sampled cells."""
    n = box.n
    nc = box.ncell
    cells = rng.choice(nc, NCELLS, replace=False)
    near = np.zeros(nc, dtype=bool)
    co = [cells % n[0], (cells // n[0]) % n[1], cells // (n[0] * n[1])]
    rngs = []
    for d in range(3):
        if d < box.ndim:
            off = np.arange(-REACH, REACH + 1)
            r = co[d][:, None] + off[None, :]
            r = r % n[d] if box.bc[d] == 0 else np.clip(r, 0, n[d] - 1)
        else:
            r = np.zeros((NCELLS, 1), dtype=np.int64)
        rngs.append(r)
    for k in range(NCELLS):
        ii, jj, kk = np.meshgrid(rngs[0][k], rngs[1][k], rngs[2][k], indexing="ij")
        near[((kk * n[1] + jj) * n[0] + ii).ravel()] = True
    sel = np.flatnonzero((box.cell >= 0) & near[np.maximum(box.cell, 0)])
    g, p = orc.grid_of(box), orc.params_of(box)
    x = np.ascontiguousarray(wl.absolute_positions(box)[:, sel])
    v = np.ascontiguousarray(box.p[:, sel].astype(np.float64))
    corr = np.zeros((4, nc))
    md = np.zeros((4, nc))
    orc.push(g, p, dt, x, v, E, box.B, corr, md)
    for q in range(4):
        assert rel_l2(corr_g[q, cells], corr[q, cells], floor=1e-300) < TOL, ("corrector", q)
        assert rel_l2(md_g[q, cells], md[q, cells], floor=1e-300) < TOL, ("moments", q)


def _run(boxes, check_boxes, seed):
    dt = min(b.dt for b in boxes)
    eng = m.Engine(boxes, precision=m.MHDPIC_PREC_MIXED)
    before = (eng.cell.cpu().numpy(), eng.off.cpu().numpy(), eng.p.cpu().numpy())
    eng.interp_push(dt, 1)
    after = (eng.cell.cpu().numpy(), eng.off.cpu().numpy(), eng.p.cpu().numpy())
    corr = eng.deposits(0).cpu().numpy()
    md = eng.deposits(1).cpu().numpy()
    assert eng.status() == 0
    starts = eng.box_start.copy()
    eng.close()
    rng = np.random.default_rng(seed)
    c0 = np.concatenate([[0], np.cumsum([b.ncell for b in boxes])])
    for bi in check_boxes:
        box = boxes[bi]
        s, e = starts[bi], starts[bi + 1]
        cs = slice(c0[bi], c0[bi + 1])
        E = _fields(box)
        _check_particles(box, E, dt, tuple(a[..., s:e] for a in before), tuple(a[..., s:e] for a in after), rng)
        _check_cells(box, E, dt, corr[:, cs], md[:, cs], rng)
        qn = box.qm_cr * box.m_cr / (box.dx[0] * box.dx[1] * box.dx[2])
        nlive = int((after[0][s:e] >= 0).sum())
        assert abs(md[0, cs].sum() - qn * nlive) < 1e-6 * qn * max(nlive, 1)


def test_bell_2d_full_size_with_the_hall_term():
    """1024^2 x 64 CRs (67,108,864), CR-Hall term on."""
    box = wl.bell_2d()
    assert box.hall and box.np == 1024 * 1024 * 64
    _run([box], [0], 51)


def test_shock_2d_full_size_load_imbalance_and_walls():
    """16384 x 128, 40 CRs per cell average with 80% near the reflecting wall."""
    box = wl.shock_2d()
    _run([box], [0], 52)


def test_shock_front_2d_full_size_open_face():
    """The open-face shock box with free slots, as the bench builds it."""
    box = wl.shock_front_2d(nx=16384, ny=128, ppc=40.0, front=0.25)
    _run([box], [0], 53)


def test_ensemble_2d_full_size_96_boxes():
    """96 boxes advanced together at their common dt; the largest, the
    smallest and two others checked."""
    boxes = wl.ensemble_2d(nbox=96)
    sizes = [b.ncell for b in boxes]
    pick = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 17, 60})
    _run(boxes, pick, 54)


def test_alfvenic_beam_3d_full_size_cells():
    """128^3 x 32 CRs (67,108,864), the default benchmark box: the sampled
    cells' deposits as well as the sampled particles."""
    box = wl.alfvenic_beam_3d()
    _run([box], [0], 55)
