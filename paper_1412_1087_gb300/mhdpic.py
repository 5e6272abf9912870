"""Thin ctypes binding of the sm_103a library ``libmhdpic.so`` (include/mhdpic.h).

Argument marshalling only: every step of the particle update runs in the
library's CUDA kernels.  PyTorch provides device memory and the stream.  If the
library is missing the import of any entry point raises; there is no CPU
fallback.

The functions carry the C names (``mhdpic_init``, ``mhdpic_sort``,
``mhdpic_interp_push``, ``mhdpic_deposit``, ``mhdpic_apply_feedback`` ...) and
raise :class:`MhdpicError` on a non-zero return code.  :class:`Engine` wraps a
context around a list of :class:`workloads.Box` objects.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhdpic.so")

MHDPIC_OK = 0
MHDPIC_BC_PERIODIC = 0
MHDPIC_BC_REFLECT = 1
MHDPIC_BC_WALL_OPEN = 2
MHDPIC_SHAPE_TSC = 2
MHDPIC_PREC_FP64 = 0
MHDPIC_PREC_MIXED = 1
MHDPIC_MEM_DEVICE = 0
MHDPIC_MEM_HOST = 1
MHDPIC_MEM_HOST_GAS = 2
MHDPIC_SPEC_ENERGY = 0
MHDPIC_SPEC_MOMENTUM = 1
MHDPIC_SPEC_MAX_BINS = 2048
MHDPIC_GAS_SOURCES = 0
MHDPIC_GAS_LINEAR_X = 1
STATUS_NAMES = {1: "FAST_MOVER", 2: "NONFINITE", 4: "OVERFLOW", 8: "SORT_CAP", 16: "CELL_RANGE", 32: "INJECT_CAP",
                64: "BARRIER", 128: "COPY_TIMEOUT"}


class MhdpicError(RuntimeError):
    pass


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("dx", ctypes.c_double * 3),
                ("x0", ctypes.c_double * 3), ("bc", ctypes.c_int32 * 3)]


class Params(ctypes.Structure):
    _fields_ = [("qm_cr", ctypes.c_double), ("qm_gas", ctypes.c_double), ("C", ctypes.c_double),
                ("m_cr", ctypes.c_double), ("hall", ctypes.c_int32), ("shape", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("memory", ctypes.c_int32), ("brick", ctypes.c_int32 * 3),
                ("reserved", ctypes.c_int32 * 8)]


class Particles(ctypes.Structure):
    # mixed precision: pos = mhdpic_pos[np] (int32 cell, 3 f32 offsets) and
    # vel = mhdpic_vel[np] (3 f32 leading words, packed residuals), 16 bytes each
    _fields_ = [("np", ctypes.c_int64), ("box_start", ctypes.POINTER(ctypes.c_int64)),
                ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("p64", ctypes.c_void_p)]


class Gas(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_void_p), ("mom", ctypes.c_void_p), ("egas", ctypes.c_void_p),
                ("B", ctypes.c_void_p)]


# every symbol the header declares, with its ctypes signature
_V = ctypes.c_void_p
SIGNATURES = {
    "mhdpic_init": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int32, ctypes.POINTER(Grid),
                                   ctypes.POINTER(Params), ctypes.POINTER(Options),
                                   ctypes.POINTER(Particles), ctypes.POINTER(Gas), _V]),
    "mhdpic_sort": (ctypes.c_int, [_V, _V, _V]),
    "mhdpic_interp_push": (ctypes.c_int, [_V, ctypes.c_double, ctypes.c_int32]),
    "mhdpic_deposit": (ctypes.c_int, [_V]),
    "mhdpic_apply_feedback": (ctypes.c_int, [_V, _V]),
    "mhdpic_live_particles": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_int64)]),
    "mhdpic_inject": (ctypes.c_int, [_V, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_uint64, _V, ctypes.POINTER(ctypes.c_int64)]),
    "mhdpic_set_injection_times": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_double]),
    "mhdpic_get_injection_times": (ctypes.c_int, [_V, _V, ctypes.POINTER(ctypes.c_double)]),
    "mhdpic_gas_predict": (ctypes.c_int, [_V, ctypes.c_double, ctypes.c_int32]),
    "mhdpic_gas_correct": (ctypes.c_int, [_V, ctypes.c_double, ctypes.c_int32, _V]),
    "mhdpic_run": (ctypes.c_int, [_V, ctypes.c_double, ctypes.c_int32, ctypes.c_int32]),
    "mhdpic_sync_particles": (ctypes.c_int, [_V]),
    "mhdpic_set_subcycle_sort": (ctypes.c_int, [_V, ctypes.c_int32]),
    "mhdpic_set_sort_lookahead": (ctypes.c_int, [_V, ctypes.c_double]),
    "mhdpic_spectrum": (ctypes.c_int, [_V, ctypes.c_int32, ctypes.c_int32, _V, _V, ctypes.c_int32, _V, _V]),
    "mhdpic_lambda_map": (ctypes.c_int, [_V, _V]),
    "mhdpic_sort_cadence": (ctypes.c_int32, [_V]),
    "mhdpic_set_step_fusion": (ctypes.c_int, [_V, ctypes.c_int32]),
    "mhdpic_step_fusion": (ctypes.c_int32, [_V]),
    "mhdpic_debug_set_barrier_limit": (ctypes.c_int, [_V, ctypes.c_int64]),
    "mhdpic_debug_set_copy_limit": (ctypes.c_int, [_V, ctypes.c_int64]),
    "mhdpic_set_field_tma": (ctypes.c_int, [_V, ctypes.c_int32]),
    "mhdpic_field_tma": (ctypes.c_int32, [_V]),
    "mhdpic_get_deposits": (ctypes.c_int, [_V, ctypes.c_int32, _V]),
    "mhdpic_get_fields": (ctypes.c_int, [_V, _V]),
    "mhdpic_get_velocities": (ctypes.c_int, [_V, _V]),
    "mhdpic_num_keys": (ctypes.c_int64, [_V]),
    "mhdpic_get_status": (ctypes.c_int, [_V, ctypes.POINTER(ctypes.c_uint32)]),
    "mhdpic_clear_status": (ctypes.c_int, [_V]),
    "mhdpic_launch_count": (ctypes.c_int64, [_V]),
    "mhdpic_debug_fail_launch": (ctypes.c_int, [_V, ctypes.c_int64]),
    "mhdpic_destroy": (ctypes.c_int, [_V]),
    "mhdpic_deposit_moments_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Params), ctypes.c_int32,
                                                       ctypes.c_int64, _V, _V, _V, _V, _V, _V]),
    "mhdpic_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mhdpic_last_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (built by ``paper_1412_1087_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise MhdpicError("CUDA library %s is missing: run __graft_entry__.build() "
                                  "(there is no CPU fallback)" % path)
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int) -> None:
    if rc != MHDPIC_OK:
        lib = load()
        raise MhdpicError("%s (%d): %s" % (lib.mhdpic_strerror(rc).decode(), rc,
                                           lib.mhdpic_last_error().decode()))


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------

def mhdpic_init(nbox, grids, params, options, particles, gas, stream) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().mhdpic_init(ctypes.byref(ctx), nbox, grids, params, ctypes.byref(options),
                              ctypes.byref(particles), ctypes.byref(gas), stream))
    return ctx


def mhdpic_sort(ctx, perm_out: int = 0, counts_out: int = 0) -> None:
    _check(load().mhdpic_sort(ctx, perm_out or None, counts_out or None))


def mhdpic_interp_push(ctx, dt: float, nsub: int = 1) -> None:
    _check(load().mhdpic_interp_push(ctx, float(dt), int(nsub)))


def mhdpic_deposit(ctx) -> None:
    _check(load().mhdpic_deposit(ctx))


def mhdpic_apply_feedback(ctx, totals_out: Optional[np.ndarray] = None) -> None:
    ptr = None
    if totals_out is not None:
        assert totals_out.dtype == np.float64 and totals_out.flags["C_CONTIGUOUS"]
        ptr = totals_out.ctypes.data_as(ctypes.c_void_p)
    _check(load().mhdpic_apply_feedback(ctx, ptr))


def mhdpic_live_particles(ctx) -> int:
    n = ctypes.c_int64(0)
    _check(load().mhdpic_live_particles(ctx, ctypes.byref(n)))
    return int(n.value)


def mhdpic_inject(ctx, dt: float, eta: float, energy_factor: float = 10.0, gamma_gas: float = 5.0 / 3.0,
                  seed: int = 0) -> tuple:
    fr = np.zeros(2, dtype=np.float64)
    n = ctypes.c_int64(0)
    _check(load().mhdpic_inject(ctx, float(dt), float(eta), float(energy_factor), float(gamma_gas),
                                int(seed) & 0xffffffffffffffff, fr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    return int(n.value), float(fr[0]), float(fr[1])


def mhdpic_set_injection_times(ctx, t_inj: Optional[np.ndarray], t_now: float, t_early: float) -> None:
    ptr = None
    if t_inj is not None:
        assert t_inj.dtype == np.float64 and t_inj.flags["C_CONTIGUOUS"]
        ptr = t_inj.ctypes.data_as(ctypes.c_void_p)
    _check(load().mhdpic_set_injection_times(ctx, ptr, float(t_now), float(t_early)))


def mhdpic_get_injection_times(ctx, np_: int) -> tuple:
    t_inj = np.zeros(max(np_, 1), dtype=np.float64)
    t = ctypes.c_double(0.0)
    _check(load().mhdpic_get_injection_times(ctx, t_inj.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t)))
    return t_inj[:np_], float(t.value)


def mhdpic_gas_predict(ctx, dt: float, model: int) -> None:
    _check(load().mhdpic_gas_predict(ctx, float(dt), int(model)))


def mhdpic_gas_correct(ctx, dt: float, model: int, totals_out: Optional[np.ndarray] = None) -> None:
    ptr = None
    if totals_out is not None:
        assert totals_out.dtype == np.float64 and totals_out.flags["C_CONTIGUOUS"]
        ptr = totals_out.ctypes.data_as(ctypes.c_void_p)
    _check(load().mhdpic_gas_correct(ctx, float(dt), int(model), ptr))


def mhdpic_run(ctx, dt: float, nsteps: int, sort_every: int = 0) -> None:
    _check(load().mhdpic_run(ctx, float(dt), int(nsteps), int(sort_every)))


def mhdpic_set_subcycle_sort(ctx, every: int) -> None:
    _check(load().mhdpic_set_subcycle_sort(ctx, int(every)))


def mhdpic_set_sort_lookahead(ctx, t: float) -> None:
    _check(load().mhdpic_set_sort_lookahead(ctx, float(t)))


def mhdpic_sync_particles(ctx) -> None:
    _check(load().mhdpic_sync_particles(ctx))


def mhdpic_spectrum(ctx, kind: int, edges: np.ndarray, region: Optional[np.ndarray], n_moment: int,
                    counts_out: np.ndarray, sums_out: Optional[np.ndarray]) -> None:
    """Host arrays: edges float64[nbins+1], region float64[6] or None,
    counts_out int64[nbox*nbins], sums_out float64[2*nbox] or None."""
    for a, dt in ((edges, np.float64), (region, np.float64), (counts_out, np.int64), (sums_out, np.float64)):
        if a is not None:
            assert a.dtype == dt and a.flags["C_CONTIGUOUS"]
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
    _check(load().mhdpic_spectrum(ctx, int(kind), int(edges.shape[0] - 1), ptr(edges), ptr(region), int(n_moment),
                                  ptr(counts_out), ptr(sums_out)))


def mhdpic_lambda_map(ctx, out_ptr: int) -> None:
    _check(load().mhdpic_lambda_map(ctx, out_ptr))


def mhdpic_sort_cadence(ctx) -> int:
    return int(load().mhdpic_sort_cadence(ctx))


def mhdpic_set_step_fusion(ctx, enable: bool) -> None:
    _check(load().mhdpic_set_step_fusion(ctx, 1 if enable else 0))


def mhdpic_step_fusion(ctx) -> int:
    return int(load().mhdpic_step_fusion(ctx))


def mhdpic_set_field_tma(ctx, enable: bool) -> None:
    _check(load().mhdpic_set_field_tma(ctx, 1 if enable else 0))


def mhdpic_field_tma(ctx) -> int:
    return int(load().mhdpic_field_tma(ctx))


def mhdpic_debug_set_barrier_limit(ctx, ns: int) -> None:
    _check(load().mhdpic_debug_set_barrier_limit(ctx, int(ns)))


def mhdpic_debug_set_copy_limit(ctx, ns: int) -> None:
    _check(load().mhdpic_debug_set_copy_limit(ctx, int(ns)))


def mhdpic_get_deposits(ctx, which: int, out_ptr: int) -> None:
    _check(load().mhdpic_get_deposits(ctx, int(which), out_ptr))


def mhdpic_get_fields(ctx, out_ptr: int) -> None:
    _check(load().mhdpic_get_fields(ctx, out_ptr))


def mhdpic_get_velocities(ctx, out_ptr: int) -> None:
    _check(load().mhdpic_get_velocities(ctx, out_ptr))


def mhdpic_num_keys(ctx) -> int:
    return int(load().mhdpic_num_keys(ctx))


def mhdpic_get_status(ctx) -> int:
    f = ctypes.c_uint32(0)
    _check(load().mhdpic_get_status(ctx, ctypes.byref(f)))
    return int(f.value)


def mhdpic_clear_status(ctx) -> None:
    _check(load().mhdpic_clear_status(ctx))


def mhdpic_launch_count(ctx) -> int:
    return int(load().mhdpic_launch_count(ctx))


def mhdpic_debug_fail_launch(ctx, n: int) -> None:
    _check(load().mhdpic_debug_fail_launch(ctx, int(n)))


def mhdpic_destroy(ctx) -> None:
    _check(load().mhdpic_destroy(ctx))


def mhdpic_deposit_moments_noalloc(grid: Grid, params: Params, precision: int, np_: int, pos=0, vel=0,
                                   x=0, p64=0, out=0, stream=None) -> None:
    """Allocation-free charge/current deposit of one box (device pointers as ints)."""
    _check(load().mhdpic_deposit_moments_noalloc(ctypes.byref(grid), ctypes.byref(params), int(precision),
                                                 int(np_), pos or None, vel or None, x or None,
                                                 p64 or None, out or None, stream))


def pack_records_arrays(cell, off, p):
    """Mixed-precision particle records from SoA arrays: pos (np, 4) int32 =
    cell plus the offsets' bits (unused dimensions 0), vel (np, 4) float32 =
    the four-velocity with a zero residual word."""
    n = cell.shape[0]
    pos = np.zeros((n, 4), dtype=np.int32)
    pos[:, 0] = cell
    pos.view(np.float32)[:, 1:1 + off.shape[0]] = off.T
    vel = np.zeros((n, 4), dtype=np.float32)
    vel[:, :3] = p.T
    return pos, vel


def pack_records(boxes):
    """pack_records_arrays over the concatenated particles of a batch of boxes."""
    cat = np.concatenate
    return pack_records_arrays(cat([b.cell for b in boxes]).astype(np.int32),
                               cat([b.off for b in boxes], axis=1).astype(np.float32),
                               cat([b.p for b in boxes], axis=1).astype(np.float32))


def status_names(flags: int) -> List[str]:
    return [name for bit, name in STATUS_NAMES.items() if flags & bit]


# ---------------------------------------------------------------------------
# Engine: a context over a batch of boxes held in torch tensors
# ---------------------------------------------------------------------------

class Engine:
    """Owns torch buffers for a batch of boxes and one library context.

    ``precision``: MHDPIC_PREC_MIXED or MHDPIC_PREC_FP64.
    ``memory``: MHDPIC_MEM_DEVICE (buffers on cuda), MHDPIC_MEM_HOST (pinned
    host buffers; every call copies through the library) or MHDPIC_MEM_HOST_GAS
    (particles on cuda, gas in pinned host buffers copied by each call).
    """

    def __init__(self, boxes: Sequence, precision: int = MHDPIC_PREC_MIXED,
                 memory: int = MHDPIC_MEM_DEVICE, brick: Sequence[int] = (0, 0, 0),
                 device: str = "cuda:0", stream=None,
                 x64: Optional[np.ndarray] = None, v64: Optional[np.ndarray] = None):
        import torch

        self.torch = torch
        self.boxes = list(boxes)
        self.precision = precision
        self.memory = memory
        nb = len(self.boxes)
        self.ndim = self.boxes[0].ndim
        counts = [b.np for b in self.boxes]
        self.box_start = np.zeros(nb + 1, dtype=np.int64)
        self.box_start[1:] = np.cumsum(counts)
        self.np = int(self.box_start[-1])
        self.nc = int(sum(b.ncell for b in self.boxes))
        self.device = torch.device(device)
        def on_device(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(self.device)

        def pinned(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()

        if memory not in (MHDPIC_MEM_DEVICE, MHDPIC_MEM_HOST, MHDPIC_MEM_HOST_GAS):
            raise ValueError("unknown memory kind %r" % (memory,))
        mk = pinned if memory == MHDPIC_MEM_HOST else on_device
        mk_gas = on_device if memory == MHDPIC_MEM_DEVICE else pinned
        cat = np.concatenate
        if precision == MHDPIC_PREC_MIXED:
            self._pos, self._vel = (mk(a, a.dtype) for a in pack_records(self.boxes))
            self._x = self._p64 = None
        else:
            from . import workloads as wl
            if x64 is None:
                x64 = cat([wl.absolute_positions(b) for b in self.boxes], axis=1)
            if v64 is None:
                v64 = cat([b.p.astype(np.float64) for b in self.boxes], axis=1)
            self._x = mk(x64, np.float64)
            self._p64 = mk(v64, np.float64)
            self._pos = self._vel = None
        self.rho = mk_gas(cat([b.rho for b in self.boxes]), np.float64)
        self.mom = mk_gas(cat([b.mom for b in self.boxes], axis=1), np.float64)
        self.egas = mk_gas(cat([b.egas for b in self.boxes]), np.float64)
        self.B = mk_gas(cat([b.B for b in self.boxes], axis=1), np.float64)

        G = (Grid * nb)()
        P = (Params * nb)()
        for i, b in enumerate(self.boxes):
            G[i].ndim = b.ndim
            for d in range(3):
                G[i].n[d] = b.n[d]
                G[i].dx[d] = b.dx[d]
                G[i].x0[d] = b.x0[d]
                G[i].bc[d] = b.bc[d]
            P[i].qm_cr, P[i].qm_gas, P[i].C, P[i].m_cr = b.qm_cr, b.qm_gas, b.C, b.m_cr
            P[i].hall, P[i].shape = b.hall, MHDPIC_SHAPE_TSC
        self._G, self._P = G, P
        opt = Options()
        opt.precision, opt.memory = precision, memory
        for d in range(3):
            opt.brick[d] = int(brick[d])
        self._opt = opt
        parts = Particles()
        parts.np = self.np
        parts.box_start = self.box_start.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))

        def ptr(t):
            return t.data_ptr() if t is not None else None

        parts.pos, parts.vel = ptr(self._pos), ptr(self._vel)
        parts.x, parts.p64 = ptr(self._x), ptr(self._p64)
        gas = Gas(ptr(self.rho), ptr(self.mom), ptr(self.egas), ptr(self.B))
        self._parts, self._gas = parts, gas
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        with torch.cuda.device(self.device):
            self.ctx = mhdpic_init(nb, G, P, opt, parts, gas, ctypes.c_void_p(stream.cuda_stream))

    # -- the caller's particle buffers ------------------------------------
    # The particle state alternates between these buffers and the library's
    # second set; reading an attribute first brings it back here
    # (mhdpic_sync_particles) and orders torch's current stream after it.
    def sync_particles(self) -> None:
        mhdpic_sync_particles(self.ctx)
        if self.memory == MHDPIC_MEM_HOST:
            # host buffers: the library's copies back are asynchronous
            self.stream.synchronize()
            return
        cur = self.torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def _synced(self, t):
        if t is not None and getattr(self, "ctx", None):
            self.sync_particles()
        return t

    # mixed precision: views into the 16-byte records (writable in place);
    # p holds the FP32 leading words of the two-word four-velocity, whose
    # exact value velocities() returns
    pos = property(lambda self: self._synced(self._pos))
    vel = property(lambda self: self._synced(self._vel))
    cell = property(lambda self: None if self._pos is None else self._synced(self._pos[:, 0]))
    off = property(lambda self: None if self._pos is None
                   else self._synced(self._pos.view(self.torch.float32)[:, 1:1 + self.ndim].t()))
    p = property(lambda self: None if self._vel is None else self._synced(self._vel[:, :3].t()))
    x = property(lambda self: self._synced(self._x))
    p64 = property(lambda self: self._synced(self._p64))

    def set_particles(self, cell, off, p) -> None:
        """Overwrite the mixed-precision state in the caller's order: cell
        (np,), off (ndim, np), p (3, np); the residual words become 0."""
        torch = self.torch
        self.sync_particles()
        pos, vel = pack_records_arrays(np.asarray(cell), np.asarray(off), np.asarray(p))
        self._pos.copy_(torch.from_numpy(pos))
        self._vel.copy_(torch.from_numpy(vel))

    def velocities(self):
        """The current four-velocities as float64 (3, np): the exact value of
        each two-word record (mixed) or a copy of p64."""
        out = self.torch.empty((3, max(self.np, 1)), dtype=self.torch.float64, device=self.device)
        mhdpic_get_velocities(self.ctx, out.data_ptr())
        return out[:, :self.np]

    # -- the step ---------------------------------------------------------
    def sort(self, want_perm: bool = False, want_counts: bool = False):
        torch = self.torch
        perm = torch.empty(max(self.np, 1), dtype=torch.int64, device=self.device) if want_perm else None
        counts = (torch.empty(max(self.num_keys(), 1), dtype=torch.int32, device=self.device)
                  if want_counts else None)
        mhdpic_sort(self.ctx, perm.data_ptr() if perm is not None else 0,
                    counts.data_ptr() if counts is not None else 0)
        return perm, counts

    def interp_push(self, dt: float, nsub: int = 1) -> None:
        mhdpic_interp_push(self.ctx, dt, nsub)

    def deposit(self) -> None:
        mhdpic_deposit(self.ctx)

    def apply_feedback(self, totals: bool = False) -> Optional[np.ndarray]:
        if totals:
            out = np.zeros(8 * len(self.boxes), dtype=np.float64)
            mhdpic_apply_feedback(self.ctx, out)
            return out.reshape(len(self.boxes), 8)
        mhdpic_apply_feedback(self.ctx, None)
        return None

    def step(self, dt: float, nsub: int = 1) -> None:
        self.interp_push(dt, nsub)
        self.apply_feedback(False)

    def live_particles(self) -> int:
        return mhdpic_live_particles(self.ctx)

    def inject(self, dt: float, eta: float, energy_factor: float = 10.0, gamma_gas: float = 5.0 / 3.0,
               seed: int = 0) -> tuple:
        """Front tracking and CR injection (Section 5): returns (n, x_s, x_t)."""
        return mhdpic_inject(self.ctx, dt, eta, energy_factor, gamma_gas, seed)

    def set_injection_times(self, t_inj=None, t_now: float = 0.0, t_early: float = float("inf")) -> None:
        """Early-particle removal (Section 5): particles with injection time
        t_i < t_early are removed at t = 2 t_i.  t_inj (np,) in the order of
        the particle attributes (None: never removed); t_now sets the clock."""
        arr = None if t_inj is None else np.ascontiguousarray(t_inj, dtype=np.float64)
        mhdpic_set_injection_times(self.ctx, arr, t_now, t_early)

    def injection_times(self) -> tuple:
        """(t_inj (np,), clock) in the order of the particle attributes."""
        return mhdpic_get_injection_times(self.ctx, self.np)

    def gas_predict(self, dt: float, model: int) -> None:
        mhdpic_gas_predict(self.ctx, dt, model)

    def gas_correct(self, dt: float, model: int, totals: bool = False) -> Optional[np.ndarray]:
        if totals:
            out = np.zeros(8 * len(self.boxes), dtype=np.float64)
            mhdpic_gas_correct(self.ctx, dt, model, out)
            return out.reshape(len(self.boxes), 8)
        mhdpic_gas_correct(self.ctx, dt, model, None)
        return None

    def coupled_step(self, dt: float, model: int, nsub: int = 1, totals: bool = False):
        """One step of the paper's predictor-corrector (eq:scheme): gas half
        step and field staging, nsub particle sub-steps in the half-step
        fields, gas full step with the corrector deposit."""
        self.gas_predict(dt * nsub, model)
        self.interp_push(dt, nsub)
        return self.gas_correct(dt * nsub, model, totals)

    def run(self, dt: float, nsteps: int, sort_every: int = 0) -> None:
        """nsteps full steps replayed from a CUDA graph (sort cadence tuned when 0)."""
        mhdpic_run(self.ctx, dt, nsteps, sort_every)

    def sort_cadence(self) -> int:
        return mhdpic_sort_cadence(self.ctx)

    def set_step_fusion(self, enable: bool) -> None:
        """One kernel launch per step of run() where the context allows it (default on)."""
        mhdpic_set_step_fusion(self.ctx, enable)

    def step_fusion(self) -> int:
        return mhdpic_step_fusion(self.ctx)

    def set_field_tma(self, enable: bool) -> None:
        """Stage the pushes' field tiles by tensor copies (default where possible) or by the threads."""
        mhdpic_set_field_tma(self.ctx, enable)

    def field_tma(self) -> int:
        return mhdpic_field_tma(self.ctx)

    # -- read-back ----------------------------------------------------------
    def deposits(self, which: int):
        out = self.torch.empty((4, self.nc), dtype=self.torch.float64, device=self.device)
        mhdpic_get_deposits(self.ctx, which, out.data_ptr())
        return out

    def set_subcycle_sort(self, every: int) -> None:
        mhdpic_set_subcycle_sort(self.ctx, every)

    def set_sort_lookahead(self, t: float) -> None:
        """Sort by the cell each particle reaches in time t (dt/2: the half-step cell)."""
        mhdpic_set_sort_lookahead(self.ctx, t)

    def spectrum(self, kind: int, edges, region=None, n_moment: int = 6):
        """Per-box counts (nbox, nbins) and sums (nbox, 2) of q^(n+1), q^n."""
        edges = np.ascontiguousarray(edges, dtype=np.float64)
        reg = None
        if region is not None:
            reg = np.zeros(6, dtype=np.float64)
            r = np.asarray(region, dtype=np.float64).ravel()
            reg[:r.shape[0]] = r
        nb = edges.shape[0] - 1
        counts = np.zeros(len(self.boxes) * nb, dtype=np.int64)
        sums = np.zeros(2 * len(self.boxes), dtype=np.float64)
        mhdpic_spectrum(self.ctx, kind, edges, reg, n_moment, counts, sums)
        return counts.reshape(len(self.boxes), nb), sums.reshape(len(self.boxes), 2)

    def lambda_map(self):
        out = self.torch.empty((3, self.nc), dtype=self.torch.float64, device=self.device)
        mhdpic_lambda_map(self.ctx, out.data_ptr())
        return out

    def fields(self):
        out = self.torch.empty((6, self.nc), dtype=self.torch.float64, device=self.device)
        mhdpic_get_fields(self.ctx, out.data_ptr())
        return out

    def num_keys(self) -> int:
        return mhdpic_num_keys(self.ctx)

    def status(self) -> int:
        return mhdpic_get_status(self.ctx)

    def clear_status(self) -> None:
        mhdpic_clear_status(self.ctx)

    def launches(self) -> int:
        return mhdpic_launch_count(self.ctx)

    def synchronize(self) -> None:
        self.stream.synchronize()

    def close(self) -> None:
        """Bring the particle state into the caller's buffers and free the context."""
        if getattr(self, "ctx", None):
            try:
                mhdpic_sync_particles(self.ctx)
            finally:
                mhdpic_destroy(self.ctx)
                self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
