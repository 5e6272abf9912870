"""FP64 CPU oracle of the MHD-PIC cosmic-ray particle update (arXiv:1412.1087).

TEST INFRASTRUCTURE ONLY.  A plain, slow, double-precision implementation of
what the CUDA path computes, written from the paper (Sections 2.1-2.2, 3 and
Appendices A.1-A.3).  It is used by the test-suite, by the smoke check and by
the benchmark's CPU-baseline leg; the product library never imports it and
shares no code with it.

The arithmetic lives in ``mhdpic_oracle.c`` (compiled here with gcc and
``-ffp-contract=off`` so that x86-64 and aarch64 give identical bits); this
module only marshals numpy arrays.  Every function cites the passage it
follows in the C file.

Parity status: every function is pinned by the ``-m "not gpu"`` tests against
closed forms or invariants (gyration radius, phase and energy; E x B drift;
TSC moments; conservation; charge sum; Hall identities; brute-force sort).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhdpic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("dx", ctypes.c_double * 3),
                ("x0", ctypes.c_double * 3), ("bc", ctypes.c_int32 * 3)]


class Params(ctypes.Structure):
    _fields_ = [("qm_cr", ctypes.c_double), ("qm_gas", ctypes.c_double), ("C", ctypes.c_double),
                ("m_cr", ctypes.c_double), ("hall", ctypes.c_int32)]


_P = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            G = ctypes.POINTER(Grid)
            Pp = ctypes.POINTER(Params)
            lib.orc_gamma.restype = ctypes.c_double
            lib.orc_gamma.argtypes = [_P, ctypes.c_double]
            lib.orc_kinetic_energy.restype = ctypes.c_double
            lib.orc_kinetic_energy.argtypes = [_P, ctypes.c_double]
            lib.orc_tsc_weights.argtypes = [ctypes.c_double, _P, _P]
            lib.orc_gather.argtypes = [G, _P, _P, ctypes.c_int, _P]
            lib.orc_deposit.argtypes = [G, _P, _P, ctypes.c_int, _P]
            lib.orc_boundary.argtypes = [G, _P, _P]
            lib.orc_field_prep.argtypes = [G, Pp, _P, _P, _P, _P, _P]
            lib.orc_deposit_moments.argtypes = [G, Pp, ctypes.c_int64, _P, _P, _P]
            lib.orc_push.argtypes = [G, Pp, ctypes.c_double, ctypes.c_int64, _P, _P, _P, _P, _P, _P]
            lib.orc_apply_feedback.argtypes = [G, _P, _P, _P]
            lib.orc_totals.argtypes = [G, Pp, ctypes.c_int64, _P, _P, _P, _P]
            lib.orc_step.argtypes = [G, Pp, ctypes.c_double, ctypes.c_int64, _P, _P, _P, _P, _P,
                                     _P, _P, _P, _P]
            lib.orc_sort_nkeys.restype = ctypes.c_int64
            lib.orc_sort_nkeys.argtypes = [G, _P]
            lib.orc_sort_key.restype = ctypes.c_int64
            lib.orc_sort_key.argtypes = [G, _P, ctypes.c_int64]
            lib.orc_cells_of.argtypes = [G, ctypes.c_int64, _P, _P]
            lib.orc_sort_cells.argtypes = [G, _P, ctypes.c_int64, _P, _P, _P]
            lib.orc_spectrum.argtypes = [G, Pp, ctypes.c_int64, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P,
                                         ctypes.c_int, _P, _P]
            lib.orc_lambda_map.argtypes = [G, Pp, _P, _P, _P, _P, _P]
            lib.orc_philox.argtypes = [_P, _P, _P]
            lib.orc_front.argtypes = [G, _P, _P, _P, _P, ctypes.c_double, _P]
            lib.orc_inject.restype = ctypes.c_int64
            lib.orc_inject.argtypes = [G, Pp, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, _P, ctypes.c_int64,
                                       _P, _P, _P, _P, _P]
            lib.orc_remove_early.restype = ctypes.c_int64
            lib.orc_remove_early.argtypes = [ctypes.c_int, ctypes.c_int64, _P, _P, _P, ctypes.c_double,
                                             ctypes.c_double]
            lib.orc_gas_rhs.argtypes = [G, ctypes.c_int, _P, _P, _P, _P, _P, _P]
            lib.orc_gas_predict.argtypes = [G, Pp, ctypes.c_int, ctypes.c_double] + [_P] * 13
            lib.orc_gas_correct.argtypes = [G, Pp, ctypes.c_int, ctypes.c_double] + [_P] * 11
            _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _pad3(xp) -> np.ndarray:
    out = np.zeros(3, dtype=np.float64)
    xp = np.asarray(xp, dtype=np.float64).reshape(-1)
    out[: xp.shape[0]] = xp
    return out


def make_grid(ndim: int, n: Sequence[int], dx=(1.0, 1.0, 1.0), x0=(0.0, 0.0, 0.0),
              bc=(0, 0, 0)) -> Grid:
    g = Grid()
    g.ndim = ndim
    for d in range(3):
        g.n[d] = int(n[d]) if d < len(n) else 1
        g.dx[d] = float(dx[d])
        g.x0[d] = float(x0[d])
        g.bc[d] = int(bc[d])
    return g


def make_params(qm_cr: float, qm_gas: float, C: float, m_cr: float, hall: int) -> Params:
    p = Params()
    p.qm_cr, p.qm_gas, p.C, p.m_cr, p.hall = float(qm_cr), float(qm_gas), float(C), float(m_cr), int(hall)
    return p


def grid_of(box) -> Grid:
    return make_grid(box.ndim, box.n, box.dx, box.x0, box.bc)


def params_of(box) -> Params:
    return make_params(box.qm_cr, box.qm_gas, box.C, box.m_cr, box.hall)


# ---------------------------------------------------------------------------
# thin wrappers
# ---------------------------------------------------------------------------

def gamma(v, C: float) -> float:
    v = _f64(v)
    return _load().orc_gamma(_ptr(v), C)


def kinetic_energy(v, C: float) -> float:
    v = _f64(v)
    return _load().orc_kinetic_energy(_ptr(v), C)


def tsc_weights(s: float):
    i = np.zeros(1, dtype=np.int64)
    w = np.zeros(3, dtype=np.float64)
    _load().orc_tsc_weights(float(s), _ptr(i), _ptr(w))
    return int(i[0]), w


def gather(g: Grid, xp, planes: np.ndarray) -> np.ndarray:
    planes = _f64(planes)
    nq = planes.shape[0]
    xp = _pad3(xp)
    out = np.zeros(nq, dtype=np.float64)
    _load().orc_gather(ctypes.byref(g), _ptr(xp), _ptr(planes), nq, _ptr(out))
    return out


def deposit(g: Grid, xp, q, planes: np.ndarray) -> None:
    assert planes.dtype == np.float64 and planes.flags["C_CONTIGUOUS"]
    q = _f64(q)
    xp = _pad3(xp)
    _load().orc_deposit(ctypes.byref(g), _ptr(xp), _ptr(q), len(q), _ptr(planes))


def boundary(g: Grid, xp, v):
    xp = _pad3(xp)
    v = _f64(v).copy()
    _load().orc_boundary(ctypes.byref(g), _ptr(xp), _ptr(v))
    return xp[: g.ndim], v


def field_prep(g: Grid, p: Params, rho, mom, B, mom_dep) -> np.ndarray:
    rho, mom, B, mom_dep = _f64(rho), _f64(mom), _f64(B), _f64(mom_dep)
    E = np.zeros_like(B)
    _load().orc_field_prep(ctypes.byref(g), ctypes.byref(p), _ptr(rho), _ptr(mom), _ptr(B),
                           _ptr(mom_dep), _ptr(E))
    return E


def deposit_moments(g: Grid, p: Params, x, v, ncell: int) -> np.ndarray:
    x, v = _f64(x), _f64(v)
    out = np.zeros((4, ncell), dtype=np.float64)
    _load().orc_deposit_moments(ctypes.byref(g), ctypes.byref(p), v.shape[1], _ptr(x), _ptr(v),
                                _ptr(out))
    return out


def push(g: Grid, p: Params, dt: float, x: np.ndarray, v: np.ndarray, E, B,
         corr: Optional[np.ndarray], mom_dep: Optional[np.ndarray]) -> None:
    """In-place push of x (ndim, np) and v (3, np); deposits accumulate."""
    for a in (x, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    E, B = _f64(E), _f64(B)
    _load().orc_push(ctypes.byref(g), ctypes.byref(p), float(dt), v.shape[1], _ptr(x), _ptr(v),
                     _ptr(E), _ptr(B), _ptr(corr), _ptr(mom_dep))


def apply_feedback(g: Grid, mom: np.ndarray, egas: np.ndarray, corr: np.ndarray) -> None:
    _load().orc_apply_feedback(ctypes.byref(g), _ptr(mom), _ptr(egas), _ptr(corr))


def totals(g: Grid, p: Params, v, mom, egas) -> np.ndarray:
    v, mom, egas = _f64(v), _f64(mom), _f64(egas)
    out = np.zeros(8, dtype=np.float64)
    _load().orc_totals(ctypes.byref(g), ctypes.byref(p), v.shape[1], _ptr(v), _ptr(mom), _ptr(egas),
                       _ptr(out))
    return out


def sort_nkeys(g: Grid, brick) -> int:
    b = np.asarray(brick, dtype=np.int32)
    return int(_load().orc_sort_nkeys(ctypes.byref(g), _ptr(b)))


def sort_key(g: Grid, brick, cell: int) -> int:
    b = np.asarray(brick, dtype=np.int32)
    return int(_load().orc_sort_key(ctypes.byref(g), _ptr(b), int(cell)))


def cells_of(g: Grid, x) -> np.ndarray:
    x = _f64(x)
    out = np.zeros(x.shape[1], dtype=np.int32)
    _load().orc_cells_of(ctypes.byref(g), x.shape[1], _ptr(x), _ptr(out))
    return out


def sort_cells(g: Grid, brick, cell) -> tuple:
    """Stable sort by brick-major cell key: returns (perm, counts)."""
    b = np.asarray(brick, dtype=np.int32)
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    perm = np.zeros(cell.shape[0], dtype=np.int64)
    counts = np.zeros(sort_nkeys(g, brick), dtype=np.int64)
    _load().orc_sort_cells(ctypes.byref(g), _ptr(b), cell.shape[0], _ptr(cell), _ptr(perm),
                           _ptr(counts))
    return perm, counts


def spectrum(g: Grid, p: Params, x, v, kind: int, edges, region=None, n_moment: int = 6) -> tuple:
    """Counts per bin and (sum q^(n+1), sum q^n) of the particles inside region
    (Section 4.3, eq:dpdE, eq:emax); kind 0 bins E_k, kind 1 bins |v|."""
    x = _f64(x)
    v = _f64(v)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nb = edges.shape[0] - 1
    reg = None if region is None else np.ascontiguousarray(region, dtype=np.float64)
    counts = np.zeros(nb, dtype=np.int64)
    sums = np.zeros(2, dtype=np.float64)
    _load().orc_spectrum(ctypes.byref(g), ctypes.byref(p), v.shape[1], _ptr(x), _ptr(v), int(kind), nb,
                         _ptr(edges), _ptr(reg), int(n_moment), _ptr(counts), _ptr(sums))
    return counts, sums


def lambda_map(g: Grid, p: Params, rho, mom, B, mom_dep) -> np.ndarray:
    """Lambda = R (u_CR - v_g) / v_A per cell, planes (3, ncell) (eq:lambda)."""
    rho, mom, B, mom_dep = _f64(rho), _f64(mom), _f64(B), _f64(mom_dep)
    out = np.zeros((3, rho.shape[0]), dtype=np.float64)
    _load().orc_lambda_map(ctypes.byref(g), ctypes.byref(p), _ptr(rho), _ptr(mom), _ptr(B), _ptr(mom_dep),
                           _ptr(out))
    return out


def gas_rhs(g: Grid, model: int, rho, mom, B, H=None) -> tuple:
    """Gas right-hand side of the coupled step's model (no CR sources):
    (dmom, dB), each (3, ncell)."""
    rho, mom, B = _f64(rho), _f64(mom), _f64(B)
    H = _f64(H) if H is not None else None
    dmom = np.zeros_like(mom)
    dB = np.zeros_like(B)
    _load().orc_gas_rhs(ctypes.byref(g), int(model), _ptr(rho), _ptr(mom), _ptr(B), _ptr(H), _ptr(dmom), _ptr(dB))
    return dmom, dB


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 words of a 4-word counter under a 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def front(g: Grid, rho, mom, egas, B, gamma_gas: float = 5.0 / 3.0) -> np.ndarray:
    """Shock front along x: (x_s, x_t, rho_up, v_up), x_s NaN without a front."""
    rho, mom, egas, B = _f64(rho), _f64(mom), _f64(egas), _f64(B)
    out = np.zeros(4)
    _load().orc_front(ctypes.byref(g), _ptr(rho), _ptr(mom), _ptr(egas), _ptr(B), float(gamma_gas), _ptr(out))
    return out


def inject(g: Grid, p: Params, fr, xs_prev: float, dt: float, eta: float, energy_factor: float, seed: int,
           call: int, carry: float, cap: int, rho: np.ndarray, mom: np.ndarray, egas: np.ndarray) -> tuple:
    """CR injection at the front fr (orc_front's output); the gas arrays are
    updated in place.  Returns (x_new (ndim, N), v_new (3, N), carry)."""
    fr = _f64(fr)
    c = np.array([carry], dtype=np.float64)
    xn = np.zeros((g.ndim, max(cap, 1)))
    vn = np.zeros((3, max(cap, 1)))
    for a in (rho, mom, egas):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    n = _load().orc_inject(ctypes.byref(g), ctypes.byref(p), _ptr(fr), float(xs_prev), float(dt), float(eta),
                           float(energy_factor), int(seed), int(call) & 0xffffffff, _ptr(c), int(cap), _ptr(xn),
                           _ptr(vn), _ptr(rho), _ptr(mom), _ptr(egas))
    return xn[:, :n].copy(), vn[:, :n].copy(), float(c[0])


def remove_early(x: np.ndarray, v: np.ndarray, t_inj, t: float, t_early: float) -> int:
    """Early-particle removal at time t (in place): live particles with
    t_inj < t_early and t >= 2 t_inj are removed.  Returns the count."""
    t_inj = _f64(t_inj)
    assert x.dtype == np.float64 and v.dtype == np.float64 and x.flags["C_CONTIGUOUS"] and v.flags["C_CONTIGUOUS"]
    assert t_inj.shape == (v.shape[1],)
    return int(_load().orc_remove_early(int(x.shape[0]), int(v.shape[1]), _ptr(x), _ptr(v), _ptr(t_inj),
                                        float(t), float(t_early)))


class State:
    """A box advanced by the oracle: FP64 particles, gas and deposit planes."""

    def __init__(self, box, x: Optional[np.ndarray] = None, v: Optional[np.ndarray] = None):
        self.g = grid_of(box)
        self.p = params_of(box)
        self.nc = box.ncell
        self.x = _f64(x).copy() if x is not None else None
        self.v = _f64(v).copy() if v is not None else None
        self.rho = _f64(box.rho).copy()
        self.mom = _f64(box.mom).copy()
        self.egas = _f64(box.egas).copy()
        self.B = _f64(box.B).copy()
        self.corr = np.zeros((4, self.nc))
        self.E = np.zeros((3, self.nc))
        self.mom_dep = deposit_moments(self.g, self.p, self.x, self.v, self.nc)

    def fields(self) -> np.ndarray:
        return field_prep(self.g, self.p, self.rho, self.mom, self.B, self.mom_dep)

    def step(self, dt: float) -> None:
        _load().orc_step(ctypes.byref(self.g), ctypes.byref(self.p), float(dt), self.v.shape[1],
                         _ptr(self.x), _ptr(self.v), _ptr(self.rho), _ptr(self.mom), _ptr(self.egas),
                         _ptr(self.B), _ptr(self.mom_dep), _ptr(self.corr), _ptr(self.E))

    def push_only(self, dt: float):
        """One particle step without applying feedback; returns (corr, new moments)."""
        E = self.fields()
        corr = np.zeros((4, self.nc))
        md = np.zeros((4, self.nc))
        push(self.g, self.p, dt, self.x, self.v, E, self.B, corr, md)
        return corr, md

    def totals(self) -> np.ndarray:
        return totals(self.g, self.p, self.v, self.mom, self.egas)

    def predict(self, dt: float, model: int):
        """Predictor of the coupled step (eq:scheme): returns the half state
        (rho, mom, egas, B) and the cell-centred E of it for the push."""
        nc = self.nc
        half = (np.zeros(nc), np.zeros((3, nc)), np.zeros(nc), np.zeros((3, nc)))
        E = np.zeros((3, nc))
        H, dm, dB = np.zeros((3, nc)), np.zeros((3, nc)), np.zeros((3, nc))
        _load().orc_gas_predict(ctypes.byref(self.g), ctypes.byref(self.p), int(model), float(dt), _ptr(self.rho),
                                _ptr(self.mom), _ptr(self.egas), _ptr(self.B), _ptr(self.mom_dep), _ptr(half[0]),
                                _ptr(half[1]), _ptr(half[2]), _ptr(half[3]), _ptr(E), _ptr(H), _ptr(dm), _ptr(dB))
        return half, E

    def correct(self, dt: float, model: int, half) -> None:
        """Corrector of the coupled step: applies self.corr and the gas model at
        the half state; self.corr is zeroed."""
        nc = self.nc
        H, dm, dB = np.zeros((3, nc)), np.zeros((3, nc)), np.zeros((3, nc))
        _load().orc_gas_correct(ctypes.byref(self.g), ctypes.byref(self.p), int(model), float(dt), _ptr(self.rho),
                                _ptr(self.mom), _ptr(self.egas), _ptr(self.B), _ptr(half[0]), _ptr(half[1]),
                                _ptr(half[3]), _ptr(self.corr), _ptr(H), _ptr(dm), _ptr(dB))

    def coupled_step(self, dt: float, model: int) -> None:
        """One step of the paper's predictor-corrector (eq:scheme): gas half
        step with the CR sources of the moments at x^n, particle step in the
        half-step fields (corrector deposit at x^(n+1/2), moments at
        x^(n+1)), gas full step with the corrector deposit."""
        half, E = self.predict(dt, model)
        self.mom_dep[:] = 0.0
        push(self.g, self.p, dt, self.x, self.v, E, half[3], self.corr, self.mom_dep)
        self.correct(dt, model, half)
