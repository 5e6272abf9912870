"""The synthetic inputs against their recipes (small sizes of each workload).

Each generator is checked for what its recipe fixes: particle counts and
where they sit, momentum magnitudes and distributions (undoing the drift
boost), the gas and field state, boundaries, free slots, and that a seed
gives the same box every time.
"""
import numpy as np

from paper_1412_1087_gb300 import workloads as wl

PERIODIC, REFLECT, WALL_OPEN = 0, 1, 2
KS999 = 1.95   # Kolmogorov-Smirnov critical value at the 0.1% level, times sqrt(n)


def _gamma(p, C):
    return np.sqrt(1.0 + (p ** 2).sum(axis=0) / C ** 2)


def _unboost_x(p, V, C):
    """Four-velocities in the frame moving at V along x."""
    p = p.astype(np.float64)
    G = 1.0 / np.sqrt(1.0 - V * V / C ** 2)
    q = p.copy()
    q[0] = G * (p[0] - V * _gamma(p, C))
    return q


def _uniform_ks(u):
    """Kolmogorov-Smirnov distance of samples u in [0, 1] from uniform."""
    u = np.sort(u)
    n = u.size
    return max(np.max(np.arange(1, n + 1) / n - u), np.max(u - np.arange(n) / n))


def test_thermal_box_recipe():
    b = wl.periodic_thermal_2d(seed=0)
    assert b.n == (64, 64, 1) and b.np == 64 * 64 * 16 and b.bc == (PERIODIC,) * 3
    assert b.C == 100.0 and b.hall == 0
    pm = np.sqrt((b.p.astype(np.float64) ** 2).sum(axis=0))
    np.testing.assert_allclose(pm, 10.0, rtol=1e-6)
    # isotropic: each component has mean 0 and mean square 100/3
    assert np.abs(b.p.astype(np.float64).mean(axis=1)).max() < 4 * 10.0 / np.sqrt(3 * b.np)
    np.testing.assert_allclose((b.p.astype(np.float64) ** 2).mean(axis=1), 100.0 / 3.0, rtol=0.03)
    # isotropic to fourth order as well: <n_d^4> = 1/5 on the sphere (a cube's
    # normalised points share the first two moments but give ~0.18)
    n4 = ((b.p.astype(np.float64) / 10.0) ** 4).mean(axis=1)
    assert np.all(np.abs(n4 - 0.2) < 4.0 * np.sqrt(16.0 / 225.0 / b.np))
    # positions uniform: across the box and inside the cells, cell counts Poisson(16)
    xy = wl.absolute_positions(b)
    for d in range(2):
        assert _uniform_ks(xy[d] / (b.n[d] * b.dx[d])) < KS999 / np.sqrt(b.np)
        assert _uniform_ks(b.off[d].astype(np.float64)) < KS999 / np.sqrt(b.np)
    counts = np.bincount(b.cell, minlength=b.ncell)
    assert abs(counts.mean() - 16.0) < 1e-12 and abs(counts.var() / 16.0 - 1.0) < 0.1
    assert np.all(b.rho == 1.0) and np.all(b.mom == 0.0)
    np.testing.assert_array_equal(b.B, np.vstack([np.ones(b.ncell), np.zeros(b.ncell), np.zeros(b.ncell)]))


def test_alfvenic_beam_recipe():
    n = 16
    b = wl.alfvenic_beam_3d(seed=0, n=n, ppc=32)
    assert b.n == (n, n, n) and b.np == n ** 3 * 32 and b.C == 300.0 and b.bc == (PERIODIC,) * 3
    dB = b.B.copy()
    dB[0] -= 1.0
    rms = np.sqrt((dB ** 2).sum(axis=0).mean())
    assert abs(rms - 0.1) < 0.01
    # divergence-free perturbation (spectral divergence of the cell-centred field)
    k = 2 * np.pi * np.fft.fftfreq(n)
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    planes = [np.fft.fftn(dB[d].reshape(n, n, n).transpose(2, 1, 0)) for d in range(3)]
    div = kx * planes[0] + ky * planes[1] + kz * planes[2]
    assert np.abs(div).max() < 1e-9 * np.abs(planes[1]).max()
    # Alfvenic gas velocity dv = -dB (rho = 1)
    np.testing.assert_allclose(b.mom, -dB, atol=1e-12)
    # the beam: |p| = 100 in the frame drifting at 10 along x
    q = _unboost_x(b.p, 10.0, b.C)
    np.testing.assert_allclose(np.sqrt((q ** 2).sum(axis=0)), 100.0, rtol=1e-5)


def test_bell_box_recipe():
    n = 32
    b = wl.bell_2d(seed=0, n=n)
    assert b.n == (n, n, 1) and b.np == n * n * 64 and b.hall == 1 and b.C == 300.0
    q = _unboost_x(b.p, 0.5, b.C)
    pm = np.sqrt((q ** 2).sum(axis=0))
    assert pm.min() >= 10.0 * (1 - 1e-5) and pm.max() <= 1e4 * (1 + 1e-5)
    # dN/dp ~ p^-2 on [10, 1e4]: 1/p is uniform on [1e-4, 0.1]
    u = (0.1 - 1.0 / pm) / (0.1 - 1e-4)
    assert _uniform_ks(np.clip(u, 0.0, 1.0)) < KS999 / np.sqrt(b.np)
    assert np.all(b.mom == 0.0) and np.all(b.B[0] == 1.0) and np.all(b.B[1:] == 0.0)


def test_shock_load_recipe():
    nx, ny = 2048, 8
    b = wl.shock_2d(seed=0, nx=nx, ny=ny, ppc=40.0)
    total = 40 * nx * ny
    assert b.np == total and b.bc == (REFLECT, PERIODIC, PERIODIC) and b.C == 200.0
    x = b.cell % nx + b.off[0].astype(np.float64)
    assert int((x < 0.05 * nx).sum()) == round(0.8 * total)
    pm = np.sqrt((b.p.astype(np.float64) ** 2).sum(axis=0))
    assert pm.min() >= 1.0 * (1 - 1e-5) and pm.max() <= 1e5 * (1 + 1e-5)
    u = (1.0 - 1.0 / pm) / (1.0 - 1e-5)
    assert _uniform_ks(np.clip(u, 0.0, 1.0)) < KS999 / np.sqrt(b.np)
    np.testing.assert_allclose(b.mom[0], -20.0 * b.rho)
    assert np.all(b.mom[1:] == 0.0)


def test_shock_front_box_recipe():
    nx, ny, ppc = 256, 8, 8.0
    b = wl.shock_front_2d(seed=0, nx=nx, ny=ny, ppc=ppc, front=0.25, v0=20.0, free_frac=0.25)
    total = int(ppc * nx * ny)
    nfree = round(0.25 * total)
    assert b.np == total + nfree and b.bc == (WALL_OPEN, PERIODIC, PERIODIC)
    assert np.all(b.cell[total:] == -1) and np.all(b.p[:, total:] == 0.0)
    assert np.all(b.cell[:total] >= 0)
    xc = np.tile(np.arange(nx) + 0.5, ny)
    down = xc < 0.25 * nx
    np.testing.assert_array_equal(b.rho, np.where(down, 4.0, 1.0))
    v = b.mom / b.rho
    np.testing.assert_array_equal(v[0], np.where(down, 0.0, -20.0))
    P = (5.0 / 3.0 - 1.0) * (b.egas - 0.5 * b.rho * (v ** 2).sum(axis=0) - 0.5 * (b.B ** 2).sum(axis=0))
    np.testing.assert_allclose(P, np.where(down, 4.0 / 3.0 * 400.0, 1.0), rtol=1e-12)


def test_ensemble_recipe_and_seeding():
    boxes = wl.ensemble_2d(nbox=6, seed0=0, max_side=36)
    for b in boxes:
        assert 32 <= b.n[0] <= 36 and b.n[0] == b.n[1] and b.bc == (PERIODIC,) * 3
        ppc = b.np // b.ncell
        assert b.np == ppc * b.ncell and 4 <= ppc <= 64
        dB = b.B.copy()
        dB[0] -= 1.0
        assert np.all(dB[:2] == 0.0)                       # z-polarised
        # plane waves with integer wave numbers in [-4, 4] only; nominal
        # amplitude at most 0.3, which a +k/-k pair of modes can raise by
        # up to sqrt(2) on the grid
        side = b.n[0]
        F = np.fft.fft2(dB[2].reshape(side, side))
        kk = np.abs(np.fft.fftfreq(side) * side)
        outside = (kk[:, None] > 4) | (kk[None, :] > 4)
        assert np.abs(F[outside]).max() < 1e-9 * np.abs(F).max()
        assert np.sqrt((dB[2] ** 2).mean()) <= 0.3 * np.sqrt(2.0)
        np.testing.assert_allclose(np.sqrt((b.p.astype(np.float64) ** 2).sum(axis=0)), 10.0, rtol=1e-6)
    # box b is seeded seed0 + b, on its own
    again = wl.ensemble_2d(nbox=3, seed0=3, max_side=36)
    for b0, b1 in zip(boxes[3:], again):
        np.testing.assert_array_equal(b0.cell, b1.cell)
        np.testing.assert_array_equal(b0.p, b1.p)
        np.testing.assert_array_equal(b0.B, b1.B)


def test_a_seed_gives_the_same_box_and_another_seed_another():
    a = wl.bell_2d(seed=7, n=16)
    b = wl.bell_2d(seed=7, n=16)
    c = wl.bell_2d(seed=8, n=16)
    for name in ("cell", "off", "p", "rho", "mom", "egas", "B"):
        np.testing.assert_array_equal(getattr(a, name), getattr(b, name))
    assert not np.array_equal(a.p, c.p) and not np.array_equal(a.off, c.off)
