"""Diagnostics through the C ABI against the oracle: particle spectra with the
E_max sums (Section 4.3, eq:dpdE, eq:emax) and the Lambda map (eq:lambda).

Spectrum bins are integer decisions taken in IEEE double on both sides, so the
counts must agree exactly on the same particle state; the sums are compared
within 1e-12 (summation order differs).  The Lambda map is compared with the
oracle evaluated on the oracle's own charge/current deposit of the same
positions."""
import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import mhdpic as m
from paper_1412_1087_gb300 import workloads as wl

from _parity import rel_l2, tilt_B

pytestmark = pytest.mark.gpu

MIXED, FP64 = m.MHDPIC_PREC_MIXED, m.MHDPIC_PREC_FP64


def _boxes():
    return {
        "thermal2d": lambda: tilt_B(wl.periodic_thermal_2d(nx=40, ny=36, ppc=12, dv_amp=0.6, seed=31), 31),
        "beam3d": lambda: wl.alfvenic_beam_3d(seed=32, n=12, ppc=9),
        "bell2d": lambda: wl.bell_2d(seed=33, n=32, ppc=16),
        "shock2d": lambda: wl.shock_2d(seed=34, nx=256, ny=8),
    }


def _oracle_spectrum(box, kind, edges, region, n_moment):
    x = wl.absolute_positions(box)
    v = box.p.astype(np.float64)
    return orc.spectrum(orc.grid_of(box), orc.params_of(box), x, v, kind, edges, region, n_moment)


def _edges(kind):
    if kind == m.MHDPIC_SPEC_ENERGY:
        return np.concatenate([[0.0], np.geomspace(1e-3, 1e5, 97)])
    return np.concatenate([[0.0], np.geomspace(1e-2, 1e5, 65)])


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("kind", [m.MHDPIC_SPEC_ENERGY, m.MHDPIC_SPEC_MOMENTUM])
@pytest.mark.parametrize("name", list(_boxes()))
def test_spectrum_matches_oracle(prec, kind, name):
    box = _boxes()[name]()
    eng = m.Engine([box], precision=prec)
    edges = _edges(kind)
    L = [box.n[d] * box.dx[d] for d in range(box.ndim)]
    regions = [None, [box.x0[d] + f * L[d] for d in range(box.ndim) for f in (0.25, 0.6)]]
    for region in regions:
        counts, sums = eng.spectrum(kind, edges, region, n_moment=6)
        oc, os_ = _oracle_spectrum(box, kind, edges, region, 6)
        np.testing.assert_array_equal(counts[0], oc)
        np.testing.assert_allclose(sums[0], os_, rtol=1e-12)
        assert counts.sum() > 0
    eng.close()


def test_spectrum_ensemble_per_box_and_empty_box():
    boxes = wl.ensemble_2d(nbox=4, seed0=41, max_side=48)
    boxes[1].cell = boxes[1].cell[:0]
    boxes[1].off = np.ascontiguousarray(boxes[1].off[:, :0])
    boxes[1].p = np.ascontiguousarray(boxes[1].p[:, :0])
    eng = m.Engine(boxes, precision=MIXED)
    edges = _edges(m.MHDPIC_SPEC_MOMENTUM)
    counts, sums = eng.spectrum(m.MHDPIC_SPEC_MOMENTUM, edges, None, n_moment=2)
    for b, box in enumerate(boxes):
        oc, os_ = _oracle_spectrum(box, m.MHDPIC_SPEC_MOMENTUM, edges, None, 2)
        np.testing.assert_array_equal(counts[b], oc)
        np.testing.assert_allclose(sums[b], os_, rtol=1e-12)
    assert counts[1].sum() == 0 and not sums[1].any()
    eng.close()


def test_spectrum_after_steps_counts_every_particle_and_is_repeatable():
    """After pushes, sorts and a pending sort the spectrum still counts every
    particle once, and two calls on the same state agree exactly."""
    box = _boxes()["beam3d"]()
    eng = m.Engine([box], precision=MIXED)
    for _ in range(3):
        eng.interp_push(box.dt, 1)
        eng.apply_feedback()
        eng.sort()
    edges = np.array([0.0, 1e30])
    c1, s1 = eng.spectrum(m.MHDPIC_SPEC_ENERGY, edges, None, 6)
    c2, s2 = eng.spectrum(m.MHDPIC_SPEC_ENERGY, edges, None, 6)
    assert c1[0, 0] == box.np
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(s1, s2)
    eng.close()


@pytest.mark.parametrize("prec", [MIXED, FP64])
@pytest.mark.parametrize("name", ["thermal2d", "beam3d", "bell2d"])
def test_lambda_map_matches_oracle(prec, name):
    box = _boxes()[name]()
    eng = m.Engine([box], precision=prec)      # init deposits n, J at the initial positions
    lam = eng.lambda_map().cpu().numpy()
    g, p = orc.grid_of(box), orc.params_of(box)
    x = wl.absolute_positions(box)
    md = orc.deposit_moments(g, p, x, box.p.astype(np.float64), box.ncell)
    olam = orc.lambda_map(g, p, box.rho, box.mom, box.B, md)
    tol = 1e-5 if prec == MIXED else 1e-12
    for d in range(3):
        assert rel_l2(lam[d], olam[d], floor=1e-30) <= tol, (d, rel_l2(lam[d], olam[d], floor=1e-30))
    eng.close()


def test_lambda_map_host_gas_mode_is_identical():
    box = _boxes()["thermal2d"]()
    box.hall = 1
    outs = []
    for mem in (m.MHDPIC_MEM_DEVICE, m.MHDPIC_MEM_HOST_GAS, m.MHDPIC_MEM_HOST):
        eng = m.Engine([box], precision=MIXED, memory=mem)
        eng.interp_push(box.dt, 1)
        eng.apply_feedback()
        outs.append(eng.lambda_map().cpu().numpy())
        eng.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


def test_spectrum_rejects_bad_arguments():
    box = _boxes()["thermal2d"]()
    eng = m.Engine([box], precision=MIXED)
    for edges in (np.array([1.0]), np.array([0.0, 2.0, 1.0]), np.array([0.0, np.inf]),
                  np.zeros(m.MHDPIC_SPEC_MAX_BINS + 2)):
        with pytest.raises(m.MhdpicError):
            eng.spectrum(m.MHDPIC_SPEC_ENERGY, edges)
    with pytest.raises(m.MhdpicError):
        eng.spectrum(7, np.array([0.0, 1.0]))
    with pytest.raises(m.MhdpicError):
        eng.spectrum(m.MHDPIC_SPEC_ENERGY, np.array([0.0, 1.0]), n_moment=65)
    # the context stays usable
    c, _ = eng.spectrum(m.MHDPIC_SPEC_ENERGY, np.array([0.0, 1e30]))
    assert c[0, 0] == box.np
    eng.close()
