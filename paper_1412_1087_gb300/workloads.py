"""Seeded synthetic workloads for the cosmic-ray particle update.

This module only draws random numbers and lays out arrays: it contains none of
the particle update's arithmetic (no interpolation, push or deposit).  Both the
CUDA path and the FP64 CPU oracle are fed from it, so they start from
bit-identical states.

Units are the paper's code units (Section 5): rho0 = B0 = (q/mc) = 1, so the
Alfven speed is 1, and the factor c is absorbed into E and J (Section 2.2).

Layout of one box (all arrays are numpy, C-contiguous; a particle slot with
cell -1 is free, for boxes with an open face):

* cells are numbered ``c = (k*ny + j)*nx + i`` (x fastest);
* gas: ``rho[nc]``, ``mom[3, nc]`` (momentum density rho*v), ``egas[nc]``
  (total energy density), ``B[3, nc]`` (cell-centred field), all float64;
* particles, quantised once so that both sides read the same numbers:
  ``cell[np]`` int32 (linear cell), ``off[ndim, np]`` float32 offsets inside
  the cell in [0, 1), ``p[3, np]`` float32 four-velocity ``v = gamma*u``.
  The exact FP64 position is ``x0 + (cell_d + off_d) * dx`` (see
  :func:`absolute_positions`); it is exact because both terms are short.

The recipes follow the paper's workloads: the gyration test of Appendix B.1,
a periodic thermal-CR box, an Alfvenic-turbulence box with a drifting CR beam,
a Bell-instability box (CR current along B), a shock-shaped load (upstream
inflow against a conducting wall, Section 5), and an ensemble of independent
boxes.  Where the paper leaves a value open, the value chosen is stated in the
recipe's docstring.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

PERIODIC = 0
REFLECT = 1
WALL_OPEN = 2   # conducting wall at the lower face, open upper face

# Particles are drawn in fixed-size chunks so that large boxes do not need a
# full set of float64 temporaries; the chunk size is part of the recipe.
_CHUNK = 1 << 22


@dataclasses.dataclass
class Box:
    """One simulation box: grid, gas state, quantised particles, parameters."""

    ndim: int
    n: Tuple[int, int, int]
    dx: Tuple[float, float, float]
    x0: Tuple[float, float, float]
    bc: Tuple[int, int, int]
    rho: np.ndarray
    mom: np.ndarray
    egas: np.ndarray
    B: np.ndarray
    cell: np.ndarray
    off: np.ndarray
    p: np.ndarray
    qm_cr: float
    qm_gas: float
    C: float
    m_cr: float
    hall: int
    dt: float
    nsteps: int
    name: str = ""

    @property
    def ncell(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def np(self) -> int:
        return int(self.cell.shape[0])

    def copy(self) -> "Box":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            kw[f.name] = v.copy() if isinstance(v, np.ndarray) else v
        return Box(**kw)


# ---------------------------------------------------------------------------
# small helpers (distributions and layout only)
# ---------------------------------------------------------------------------

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic_dirs(rng: np.random.Generator, m: int) -> np.ndarray:
    """Unit vectors uniform on the sphere, shape (3, m)."""
    g = rng.standard_normal((3, m))
    nrm = np.sqrt((g * g).sum(axis=0))
    nrm[nrm == 0.0] = 1.0
    return g / nrm


def _quantise_positions(s: np.ndarray, n: Tuple[int, int, int], ndim: int):
    """Split positions in cell units (ndim, m) into (linear cell, f32 offset)."""
    m = s.shape[1]
    idx = np.floor(s).astype(np.int64)
    off = (s - idx).astype(np.float32)
    # a float64 offset just below 1 may round to 1.0f: move it to the next cell
    up = off >= np.float32(1.0)
    off[up] = np.float32(0.0)
    idx[up] += 1
    for d in range(ndim):
        idx[d] %= n[d]
    cell = idx[0].copy()
    if ndim >= 2:
        cell += n[0] * idx[1]
    if ndim == 3:
        cell += n[0] * n[1] * idx[2]
    return cell.astype(np.int32), off.reshape(ndim, m)


def absolute_positions(box: Box) -> np.ndarray:
    """Exact FP64 positions (ndim, np) of the quantised particles."""
    nx, ny, _ = box.n
    c = box.cell.astype(np.int64)
    coords = [c % nx]
    if box.ndim >= 2:
        coords.append((c // nx) % ny)
    if box.ndim == 3:
        coords.append(c // (nx * ny))
    x = np.empty((box.ndim, box.np), dtype=np.float64)
    for d in range(box.ndim):
        x[d] = box.x0[d] + (coords[d].astype(np.float64) + box.off[d].astype(np.float64)) * box.dx[d]
    x[0, c < 0] = np.nan   # a free slot (cell -1): no particle
    return x


def cell_coordinates(box: Box) -> np.ndarray:
    """Integer cell coordinates (ndim, np) of the quantised particles."""
    nx, ny, _ = box.n
    c = box.cell.astype(np.int64)
    out = [c % nx]
    if box.ndim >= 2:
        out.append((c // nx) % ny)
    if box.ndim == 3:
        out.append(c // (nx * ny))
    return np.stack(out)


def _cell_centres(n, dx, x0, ndim):
    """Cell-centre coordinates as 1-D arrays per dimension."""
    return [x0[d] + (np.arange(n[d], dtype=np.float64) + 0.5) * dx[d] for d in range(3)]


def _gas(n, rho0: float, v0, B_of_cells: np.ndarray, P0: float, gamma_gas: float,
         dv: Optional[np.ndarray] = None):
    """Uniform gas of density rho0 and pressure P0 moving at v0 (+ dv per cell)."""
    nc = n[0] * n[1] * n[2]
    rho = np.full(nc, rho0, dtype=np.float64)
    vel = np.empty((3, nc), dtype=np.float64)
    for d in range(3):
        vel[d] = v0[d]
    if dv is not None:
        vel += dv
    mom = rho * vel
    B = B_of_cells
    egas = P0 / (gamma_gas - 1.0) + 0.5 * rho * (vel * vel).sum(axis=0) + 0.5 * (B * B).sum(axis=0)
    return rho, mom, egas, B


def _alfvenic_modes(rng, n, ndim, nmodes: int, dB_rms: float, polar_z: bool):
    """Random-phase superposition of nmodes transverse modes, rms amplitude dB_rms.

    Wave vectors are integer multiples of the box wavenumbers with components
    in [-4, 4] (drawn without replacement, zero excluded).  In 3-D the
    polarisation is along k x x_hat (a random direction perpendicular to x_hat
    when k is parallel to x_hat); with ``polar_z`` (2-D boxes) it is z_hat.
    Each mode is div-free because its polarisation is perpendicular to k.
    Returns dB with shape (3, ncell).
    """
    nc = n[0] * n[1] * n[2]
    dB = np.zeros((3, nc), dtype=np.float64)
    if dB_rms == 0.0 or nmodes == 0:
        return dB
    if ndim == 3:
        grid = np.array([(a, b, c) for a in range(-4, 5) for b in range(-4, 5)
                         for c in range(-4, 5) if (a, b, c) != (0, 0, 0)])
    else:
        grid = np.array([(a, b, 0) for a in range(-4, 5) for b in range(-4, 5)
                         if (a, b) != (0, 0)])
    pick = rng.choice(len(grid), size=nmodes, replace=False)
    amp = dB_rms / math.sqrt(nmodes / 2.0)
    xs = _cell_centres(n, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), ndim)
    for m in range(nmodes):
        nv = grid[pick[m]].astype(np.float64)
        k = 2.0 * np.pi * nv / np.array([n[0], n[1], n[2]], dtype=np.float64)
        if polar_z:
            e = np.array([0.0, 0.0, 1.0])
        else:
            e = np.cross(k, np.array([1.0, 0.0, 0.0]))
            if np.linalg.norm(e) == 0.0:
                th = rng.uniform(0.0, 2.0 * np.pi)
                e = np.array([0.0, math.cos(th), math.sin(th)])
            e = e / np.linalg.norm(e)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        # separable complex exponential evaluated at the cell centres
        ex = np.exp(1j * k[0] * xs[0])
        ey = np.exp(1j * k[1] * xs[1])
        ez = np.exp(1j * k[2] * xs[2]) if ndim == 3 else np.ones(1, dtype=complex)
        wave = (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).reshape(-1)
        wave = np.real(wave * np.exp(1j * phase))
        for d in range(3):
            if e[d] != 0.0:
                dB[d] += amp * e[d] * wave
    return dB


def _boost_x(p: np.ndarray, V: float, C: float) -> np.ndarray:
    """Lorentz boost of four-velocities p (3, m) by speed V along x.

    For a particle of Lorentz factor gamma = sqrt(1 + p^2/C^2) the boosted
    x component is Gamma*(p_x + V*gamma); transverse components are unchanged.
    """
    if V == 0.0:
        return p
    G = 1.0 / math.sqrt(1.0 - V * V / (C * C))
    gam = np.sqrt(1.0 + (p * p).sum(axis=0) / (C * C))
    q = p.copy()
    q[0] = G * (p[0] + V * gam)
    return q


def _momenta(rng, m: int, kind: str, C: float, pmag: float = 0.0,
             prange: Tuple[float, float] = (1.0, 1.0), V: float = 0.0) -> np.ndarray:
    """Draw m four-velocities (float64, (3, m)).

    kind = "mono":  isotropic with |p| = pmag;
    kind = "power": isotropic with dN/dp proportional to p^-2 on prange, i.e.
    a 3-D distribution function f(p) proportional to p^-4, sampled by inverse
    CDF p = 1/(1/pmin - U (1/pmin - 1/pmax)).
    The result is boosted by V along x (the drift frame moves at V).
    """
    d = _isotropic_dirs(rng, m)
    if kind == "mono":
        mag = np.full(m, pmag)
    elif kind == "power":
        lo, hi = prange
        u = rng.random(m)
        mag = 1.0 / (1.0 / lo - u * (1.0 / lo - 1.0 / hi))
    else:
        raise ValueError(kind)
    return _boost_x(d * mag, V, C)


def _particles_uniform(rng, n, ndim, npart: int, lo=None, hi=None, **mom_kw):
    """npart particles uniform in the box (or in [lo, hi) along x), quantised."""
    cells, offs, ps = [], [], []
    left = npart
    while left > 0:
        m = min(left, _CHUNK)
        s = np.empty((ndim, m), dtype=np.float64)
        for d in range(ndim):
            if d == 0 and lo is not None:
                s[d] = lo + (hi - lo) * rng.random(m)
            else:
                s[d] = n[d] * rng.random(m)
        c, o = _quantise_positions(s, n, ndim)
        p = _momenta(rng, m, **mom_kw).astype(np.float32)
        cells.append(c)
        offs.append(o)
        ps.append(p)
        left -= m
    return (np.concatenate(cells), np.ascontiguousarray(np.concatenate(offs, axis=1)),
            np.ascontiguousarray(np.concatenate(ps, axis=1)))


def choose_dt(p32: np.ndarray, C: float, qm_cr: float, Bmax: float, dx: float,
              cfl: float = 0.4, upsilon: float = 0.3) -> float:
    """One fixed time step per workload (Appendix A.4 constraints).

    dt = min(cfl*dx / max_{j,d} |u_{j,d}|, upsilon * min_j gamma_j / (qm*Bmax)):
    particles move at most ``cfl`` cells per step (the paper allows two) and
    the Larmor frequency satisfies Omega_L dt <= upsilon (the paper uses 0.3).
    """
    p = p32.astype(np.float64)
    gam = np.sqrt(1.0 + (p * p).sum(axis=0) / (C * C))
    umax = float(np.abs(p / gam).max()) if p.shape[1] else 1.0
    gmin = float(gam.min()) if p.shape[1] else 1.0
    dt1 = cfl * dx / umax if umax > 0 else np.inf
    dt2 = upsilon * gmin / (qm_cr * Bmax) if Bmax > 0 else np.inf
    return float(min(dt1, dt2))


def _mass(ratio_cr_gas: float, qm_gas: float, rho: float, dV: float, qm_cr: float, ppc: float):
    """CR particle mass so that n_CR / n_gas = ratio at the mean particle density.

    n_gas = qm_gas*rho (Appendix A.1) and each particle carries charge
    qm_cr*m_cr per cell volume, so m_cr = ratio*qm_gas*rho*dV / (qm_cr*ppc).
    """
    return ratio_cr_gas * qm_gas * rho * dV / (qm_cr * ppc)


def _make_box(name, ndim, n, bc, gas, part, qm_cr, qm_gas, C, m_cr, hall, dt, nsteps):
    rho, mom, egas, B = gas
    cell, off, p = part
    return Box(ndim=ndim, n=tuple(int(v) for v in n), dx=(1.0, 1.0, 1.0), x0=(0.0, 0.0, 0.0),
               bc=tuple(bc), rho=rho, mom=np.ascontiguousarray(mom), egas=egas,
               B=np.ascontiguousarray(B), cell=cell, off=off, p=p, qm_cr=qm_cr, qm_gas=qm_gas,
               C=C, m_cr=m_cr, hall=hall, dt=dt, nsteps=nsteps, name=name)


# ---------------------------------------------------------------------------
# workload recipes
# ---------------------------------------------------------------------------

def periodic_thermal_2d(seed: int = 0, nx: int = 64, ny: int = 64, ppc: int = 16,
                        pmag: float = 10.0, C: float = 100.0, dv_amp: float = 0.0,
                        nsteps: int = 100) -> Box:
    """2-D periodic box, uniform gas (rho=1, v=0, P=1), B = (1, 0, 0).

    ``ppc`` CRs per cell at uniform random positions with isotropic |p| = pmag,
    C = 100, q/m = 1, n_CR/n_gas = 1e-3 (reading: the paper fixes no ratio
    here).  ``dv_amp`` > 0 adds a seeded random cell-wise gas velocity so that
    the ideal electric field -v x B is non-zero (used by parity tests).
    Default: 64 x 64 cells, 16 per cell (65,536 particles), 100 steps.
    """
    rng = _rng(seed)
    n = (nx, ny, 1)
    nc = nx * ny
    B = np.zeros((3, nc))
    B[0] = 1.0
    dv = None
    if dv_amp > 0.0:
        dv = dv_amp * rng.standard_normal((3, nc))
    gas = _gas(n, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0, dv)
    part = _particles_uniform(rng, n, 2, nc * ppc, kind="mono", C=C, pmag=pmag)
    dt = choose_dt(part[2], C, 1.0, float(np.sqrt((B * B).sum(0)).max()), 1.0)
    return _make_box("periodic_thermal_2d", 2, n, (PERIODIC,) * 3, gas, part, 1.0, 1.0, C,
                     _mass(1e-3, 1.0, 1.0, 1.0, 1.0, ppc), 0, dt, nsteps)


def alfvenic_beam_3d(seed: int = 0, n: int = 128, ppc: int = 32, nsteps: int = 200,
                     dB_rms: float = 0.1, nmodes: int = 64, hall: int = 0) -> Box:
    """3-D periodic n^3 box, uniform gas plus a random-phase Alfvenic perturbation.

    B = x_hat + dB with dB/B0 = 0.1 (rms) from 64 Fourier modes, dv = -dB/sqrt(rho).
    CR beam: isotropic |p| = 100 in the beam frame, boosted by V = 10 v_A along
    B (x), C = 300, n_CR/n_gas = 1e-3, ``ppc`` per cell (32 -> 67,108,864 CRs at
    n = 128).  Gas pressure P = 1, gamma_gas = 5/3.
    """
    rng = _rng(seed)
    nn = (n, n, n)
    nc = n ** 3
    B = np.zeros((3, nc))
    B[0] = 1.0
    dB = _alfvenic_modes(rng, nn, 3, nmodes, dB_rms, polar_z=False)
    B += dB
    gas = _gas(nn, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0, -dB)
    C = 300.0
    part = _particles_uniform(rng, nn, 3, nc * ppc, kind="mono", C=C, pmag=100.0, V=10.0)
    dt = choose_dt(part[2], C, 1.0, float(np.sqrt((B * B).sum(0)).max()), 1.0)
    return _make_box("alfvenic_beam_3d", 3, nn, (PERIODIC,) * 3, gas, part, 1.0, 1.0, C,
                     _mass(1e-3, 1.0, 1.0, 1.0, 1.0, ppc), hall, dt, nsteps)


def bell_2d(seed: int = 0, n: int = 1024, ppc: int = 64, nsteps: int = 500) -> Box:
    """2-D periodic n^2 box for the Bell instability with the CR-Hall term on.

    Uniform gas at rest, B = x_hat; CRs with dN/dp ~ p^-2 on [10, 1e4]
    (f(p) ~ p^-4), isotropic in a frame drifting at 0.5 v_A along x; C = 300
    (reading), n_CR/n_gas = 1e-3.  1024^2 x 64 = 67,108,864 CRs.
    """
    rng = _rng(seed)
    nn = (n, n, 1)
    nc = n * n
    B = np.zeros((3, nc))
    B[0] = 1.0
    gas = _gas(nn, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0)
    C = 300.0
    part = _particles_uniform(rng, nn, 2, nc * ppc, kind="power", C=C, prange=(10.0, 1e4), V=0.5)
    dt = choose_dt(part[2], C, 1.0, 1.0, 1.0)
    return _make_box("bell_2d", 2, nn, (PERIODIC,) * 3, gas, part, 1.0, 1.0, C,
                     _mass(1e-3, 1.0, 1.0, 1.0, 1.0, ppc), 1, dt, nsteps)


def shock_2d(seed: int = 0, nx: int = 16384, ny: int = 128, ppc: float = 40.0,
             dense_frac_cells: float = 0.05, dense_frac_parts: float = 0.8,
             nsteps: int = 1000) -> Box:
    """Shock-shaped load: 2-D nx x ny, conducting wall at x = 0, upstream inflow.

    Gas rho = 1, v = (-20, 0, 0), P = 1, B = x_hat (parallel shock, so the
    ideal field -v x B vanishes).  Average ``ppc`` CRs per cell with 80% of
    them in the 5% of cells nearest the wall; dN/dp ~ p^-2 on [1, 1e5], C = 200.
    x boundaries reflect (the far inflow boundary also reflects so the particle
    count stays fixed: a stated deviation); y is periodic.
    At the default size: 83,886,080 CRs, 67,108,864 of them in x < 819.2.
    """
    rng = _rng(seed)
    nn = (nx, ny, 1)
    nc = nx * ny
    B = np.zeros((3, nc))
    B[0] = 1.0
    gas = _gas(nn, 1.0, (-20.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0)
    C = 200.0
    total = int(round(ppc * nc))
    n_dense = int(round(dense_frac_parts * total))
    xw = dense_frac_cells * nx
    a = _particles_uniform(rng, nn, 2, n_dense, lo=0.0, hi=xw, kind="power", C=C, prange=(1.0, 1e5))
    b = _particles_uniform(rng, nn, 2, total - n_dense, lo=xw, hi=float(nx), kind="power", C=C,
                           prange=(1.0, 1e5))
    part = (np.concatenate([a[0], b[0]]), np.ascontiguousarray(np.concatenate([a[1], b[1]], axis=1)),
            np.ascontiguousarray(np.concatenate([a[2], b[2]], axis=1)))
    dt = choose_dt(part[2], C, 1.0, 1.0, 1.0)
    return _make_box("shock_2d", 2, nn, (REFLECT, PERIODIC, PERIODIC), gas, part, 1.0, 1.0, C,
                     _mass(1e-3, 1.0, 1.0, 1.0, 1.0, ppc), 0, dt, nsteps)


def shock_front_2d(seed: int = 0, nx: int = 1024, ny: int = 32, ppc: float = 8.0, front: float = 0.25,
                   v0: float = 20.0, free_frac: float = 0.25, nsteps: int = 100) -> Box:
    """The shock box with open inflow (Section 5) and a shocked gas profile.

    2-D nx x ny, conducting wall at x = 0 and an open (inflow) face at
    x = nx (MHDPIC_BC_WALL_OPEN along x), y periodic.  Upstream of the front
    (x >= front nx) the gas is rho0 = 1, v = (-v0, 0, 0), P0 = 1; downstream it
    is the strong-shock state of eq:rh in the downstream frame: rho1 = 4,
    v = 0, P1 = (4/3) rho0 v0^2 (gamma = 5/3, r = 4).  B = x_hat.  CRs as in
    the shock-shaped load (dN/dp ~ p^-2 on [1, 1e5], C = 200), ppc per cell on
    average with 80% in the 5% of cells nearest the wall; a fraction free_frac
    of the particle slots (at the end) is free for injected particles.
    """
    rng = _rng(seed)
    nn = (nx, ny, 1)
    nc = nx * ny
    B = np.zeros((3, nc))
    B[0] = 1.0
    xf = front * nx
    xc = np.tile(np.arange(nx, dtype=np.float64) + 0.5, ny)
    down = xc < xf
    dv = np.zeros((3, nc))
    dv[0] = np.where(down, 0.0, -v0)
    rho, mom, egas, Bc = _gas(nn, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0, dv=dv)
    rho = np.where(down, 4.0, 1.0)
    mom = np.ascontiguousarray(rho * dv)
    P = np.where(down, 4.0 / 3.0 * v0 * v0, 1.0)
    egas = P / (5.0 / 3.0 - 1.0) + 0.5 * rho * (dv * dv).sum(axis=0) + 0.5 * (Bc * Bc).sum(axis=0)
    C = 200.0
    total = int(round(ppc * nc))
    n_dense = int(round(0.8 * total))
    xw = 0.05 * nx
    a = _particles_uniform(rng, nn, 2, n_dense, lo=0.0, hi=xw, kind="power", C=C, prange=(1.0, 1e5))
    b = _particles_uniform(rng, nn, 2, total - n_dense, lo=xw, hi=float(nx), kind="power", C=C,
                           prange=(1.0, 1e5))
    cell = np.concatenate([a[0], b[0]])
    off = np.concatenate([a[1], b[1]], axis=1)
    p = np.concatenate([a[2], b[2]], axis=1)
    nfree = int(round(free_frac * total))
    cell = np.concatenate([cell, np.full(nfree, -1, dtype=np.int32)])
    off = np.ascontiguousarray(np.concatenate([off, np.zeros((2, nfree), dtype=np.float32)], axis=1))
    p = np.ascontiguousarray(np.concatenate([p, np.zeros((3, nfree), dtype=np.float32)], axis=1))
    dt = choose_dt(p[:, :total], C, 1.0, 1.0, 1.0)
    return _make_box("shock_front_2d", 2, nn, (WALL_OPEN, PERIODIC, PERIODIC), (rho, mom, egas, Bc),
                     (cell, off, p), 1.0, 1.0, C, _mass(1e-3, 1.0, 1.0, 1.0, 1.0, ppc), 0, dt, nsteps)


def ensemble_2d(nbox: int = 96, seed0: int = 0, side_lo: int = 32, side_span: float = 16.0,
                ppc_lo: int = 4, ppc_hi: int = 64, dB_max: float = 0.3,
                nsteps: int = 500, max_side: Optional[int] = None) -> List[Box]:
    """Ensemble of independent 2-D periodic boxes (box b seeded b + seed0).

    Side n_b = round(32 * 16^U) (log-uniform in [32, 512]), ppc_b uniform in
    [4, 64], dB/B0 uniform in [0, 0.3] from 64 modes with in-plane k and z_hat
    polarisation, Alfvenic gas velocity dv = -dB/sqrt(rho) (reading), |p| = 10,
    C = 100, n_CR/n_gas = 1e-3.  ``max_side`` clips the side (small test runs).
    """
    boxes = []
    for b in range(nbox):
        rng = _rng(seed0 + b)
        side = int(round(side_lo * side_span ** rng.random()))
        if max_side is not None:
            side = min(side, max_side)
        ppc = int(rng.integers(ppc_lo, ppc_hi + 1))
        amp = float(dB_max * rng.random())
        nn = (side, side, 1)
        nc = side * side
        B = np.zeros((3, nc))
        B[0] = 1.0
        dB = _alfvenic_modes(rng, nn, 2, min(64, 80), amp, polar_z=True)
        B += dB
        gas = _gas(nn, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0, -dB)
        C = 100.0
        part = _particles_uniform(rng, nn, 2, nc * ppc, kind="mono", C=C, pmag=10.0)
        dt = choose_dt(part[2], C, 1.0, float(np.sqrt((B * B).sum(0)).max()), 1.0)
        boxes.append(_make_box("ensemble_2d[%d]" % b, 2, nn, (PERIODIC,) * 3, gas, part, 1.0, 1.0,
                               C, _mass(1e-3, 1.0, 1.0, 1.0, 1.0, ppc), 0, dt, nsteps))
    return boxes


def gyration(relativistic: bool = False, v0: float = 0.0, C: float = 10.0, n: int = 4) -> Box:
    """Single-particle gyration test of Appendix B.1.

    Gas moving at v0 y_hat through B0 = x_hat (q/mc = B0 = 1); in the gas
    frame the particle has v_par = 0 and v_perp = 1 (C = 10, R_L = 1,
    Omega_L = 1) or v_perp = 100 (relativistic, gamma_1 ~ 10, R_L = 100,
    Omega_L ~ 0.1).  In the gas frame its perpendicular four-velocity points
    along z; the lab-frame four-velocity is that vector boosted by v0 along y,
    i.e. (0, Gamma_0 gamma_1 v0, v_perp).  The box is 3-D periodic with n^3
    large cells (width 64 or 128) so the y-z orbit is tracked and stays inside;
    the particle starts at the box centre.  dt is the paper's mean step (0.5 or
    5); tests that use the random step draw it themselves.
    """
    vperp = 100.0 if relativistic else 1.0
    dxv = 128.0 if relativistic else 64.0
    nn = (n, n, n)
    nc = n ** 3
    B = np.zeros((3, nc))
    B[0] = 1.0
    gas = _gas(nn, 1.0, (0.0, v0, 0.0), B, 1.0, 5.0 / 3.0)
    c = n // 2
    cell = np.array([(c * n + c) * n + c], dtype=np.int32)
    off = np.zeros((3, 1), dtype=np.float32)
    g1 = math.sqrt(C * C + vperp * vperp) / C
    G0 = 1.0 / math.sqrt(1.0 - v0 * v0 / (C * C))
    p = np.array([[0.0], [G0 * g1 * v0], [vperp]], dtype=np.float64)
    bx = Box(ndim=3, n=nn, dx=(dxv, dxv, dxv), x0=(0.0, 0.0, 0.0), bc=(PERIODIC,) * 3,
             rho=gas[0], mom=gas[1], egas=gas[2], B=gas[3], cell=cell, off=off,
             p=p.astype(np.float32), qm_cr=1.0, qm_gas=1.0, C=C, m_cr=1e-6, hall=0,
             dt=5.0 if relativistic else 0.5, nsteps=100, name="gyration")
    return bx


def bell_linear(eps: float = 0.5, Lambda: float = 0.0, nx: int = 32, ny: int = 4, amp: float = 1e-3,
                cfl: float = 0.4, ppc: int = 1) -> Box:
    """Linear growth of the Bell instability, Appendix B.2.

    A 2-D periodic box of nx x ny square cells, one most unstable wavelength
    lambda = 1 along x (B0 = rho0 = 1, so v_A = 1), uniform in y.  Cold CRs,
    ppc per cell spread evenly along x and placed at the cell centre in y,
    drift at U_s = v_A/eps along x; q/mc = 1e-6 k0 makes their own motion
    negligible, so they carry a constant current J = n_CR U_s along x, and
    C = 100 U_s.

    Without the CR-Hall term (Lambda = 0) the box wavenumber is k0 = J/(2 B0)
    (J = 4 pi) and the gas starts on the eigenvector of eq:eigenvect.  With it,
    R = Lambda eps (Lambda = R U_s / v_A, eq:lambda), the box wavenumber is the
    most unstable k_m = k0/f with f = 1 + (Lambda/2)^2, so J = 2 f k_m, and the
    gas starts on eq:eigenvect2; qm_gas is set so that n_CR/(n_g + n_CR) = R.
    The perturbation amplitude is amp (times B0).  dt puts both the CRs and
    an Alfven wave at cfl cells per step.
    """
    k = 2.0 * math.pi
    dxv = 1.0 / nx
    n = (nx, ny, 1)
    nc = nx * ny
    f = 1.0 + 0.25 * Lambda * Lambda
    k0 = f * k
    J = 2.0 * k0
    U = 1.0 / eps
    ncr = J / U
    qm_cr = 1e-6 * k0
    C = 100.0 * U
    hall = 1 if Lambda > 0.0 else 0
    if hall:
        R = Lambda * eps
        qm_gas = ncr * (1.0 - R) / R
    else:
        qm_gas = 1.0
    xc = (np.arange(nx, dtype=np.float64) + 0.5) * dxv
    ph = np.tile(k * xc, ny)
    B = np.zeros((3, nc))
    B[0] = 1.0
    B[1] = amp * np.cos(ph)
    B[2] = amp * np.sin(ph)
    dv = np.zeros((3, nc))
    if hall:
        sf = math.sqrt(f)
        dv[1] = amp * (0.5 * Lambda * np.cos(ph) + sf * np.sin(ph))
        dv[2] = amp * (0.5 * Lambda * np.sin(ph) - sf * np.cos(ph))
    else:
        th = math.asin(eps)
        dv[1] = amp * np.sin(ph - th)
        dv[2] = -amp * np.cos(ph - th)
    rho, mom, egas, Bc = _gas(n, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0, dv=dv)
    # particles: ppc per cell, evenly spaced in x, at the cell centre in y
    npart = nc * ppc
    ci = np.repeat(np.arange(nc, dtype=np.int64), ppc)
    sub = np.tile(np.arange(ppc, dtype=np.float64), nc)
    s = np.empty((2, npart))
    s[0] = (ci % nx) + (sub + 0.5) / ppc
    s[1] = (ci // nx) + 0.5
    cell, off = _quantise_positions(s, n, 2)
    gam = 1.0 / math.sqrt(1.0 - (U / C) ** 2)
    p = np.zeros((3, npart), dtype=np.float32)
    p[0] = np.float32(gam * U)
    dV = dxv * dxv
    m_cr = J * dV / (ppc * qm_cr * U)
    dt = cfl * dxv / max(1.0, U)
    return Box(ndim=2, n=n, dx=(dxv, dxv, 1.0), x0=(0.0, 0.0, 0.0), bc=(PERIODIC,) * 3, rho=rho,
               mom=np.ascontiguousarray(mom), egas=egas, B=np.ascontiguousarray(Bc), cell=cell, off=off, p=p,
               qm_cr=qm_cr, qm_gas=qm_gas, C=C, m_cr=m_cr, hall=hall, dt=dt,
               nsteps=int(math.ceil(3.0 / (k * dt))), name="bell_linear")


def scaled(box_fn, **kw) -> Box:
    """Call a recipe with overridden size arguments (small parity-test variants)."""
    return box_fn(**kw)
