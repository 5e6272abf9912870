"""Shared helpers of the GPU parity tests (not a test module)."""
import numpy as np

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl


def default_brick(ndim):
    return (4, 4, 4) if ndim == 3 else (8, 8, 1)


def tilt_B(box, seed=0, amp=0.2):
    """Tilt B off the axes (plus small noise) so every deposit channel carries signal."""
    rng = np.random.default_rng(seed)
    B = box.B + np.array([[0.0], [0.45], [-0.35]]) + amp * rng.standard_normal(box.B.shape)
    box.B = np.ascontiguousarray(B)
    return box


def sorted_oracle_state(box, brick=None):
    """Oracle particle arrays in the library's cell-sorted order."""
    brick = brick or default_brick(box.ndim)
    g = orc.grid_of(box)
    perm, counts = orc.sort_cells(g, brick, box.cell)
    x = np.ascontiguousarray(wl.absolute_positions(box)[:, perm])
    v = np.ascontiguousarray(box.p.astype(np.float64)[:, perm])
    return perm, counts, x, v


def rel_l2(a, b, floor=0.0):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor, 1e-300))


def positions_of(eng):
    """Absolute FP64 positions of the engine's particles, (ndim, np), per box."""
    if eng.x is not None:
        return eng.x.cpu().numpy()
    cell = eng.cell.cpu().numpy().astype(np.int64)
    off = eng.off.cpu().numpy().astype(np.float64)
    out = np.empty((eng.ndim, eng.np))
    for bi, b in enumerate(eng.boxes):
        s, e = eng.box_start[bi], eng.box_start[bi + 1]
        c = cell[s:e]
        co = [c % b.n[0], (c // b.n[0]) % b.n[1], c // (b.n[0] * b.n[1])]
        for d in range(eng.ndim):
            out[d, s:e] = b.x0[d] + (co[d] + off[d, s:e]) * b.dx[d]
    return out


def momenta_of(eng):
    """Four-velocities (3, np) as float64: the exact value of the mixed
    precision's two-word records, or the FP64 state."""
    return eng.velocities().cpu().numpy()


def mixed_rows(eng):
    """The mixed-precision state as rows (cell, offsets, leading words,
    residual word), one column per particle, for comparisons bit for bit."""
    vel = eng.vel.cpu().numpy()
    return np.vstack([eng.cell.cpu().numpy().astype(np.float64)[None], eng.off.cpu().numpy(),
                      vel[:, :3].T.astype(np.float64), vel[:, 3].view(np.uint32).astype(np.float64)[None]])


def periodic_diff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)
