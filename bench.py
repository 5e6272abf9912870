"""Benchmark of the cosmic-ray particle update (particle-steps per second).

Default workload: 3-D periodic 128^3 box, 32 CRs per cell (67,108,864 CRs),
uniform gas with a random-phase Alfvenic perturbation dB/B0 = 0.1 (64 modes),
CR beam |p| = 100 boosted to 10 v_A along B, C = 300.  One step is the whole
hot path: staged-field push with both deposits (interp_push), feedback to the
gas with field restaging (apply_feedback), and the cell sort every
``--sort-every`` steps.

Prints ONE JSON line.  Under torchrun each rank advances its own independent
box (seed = rank), the time is the maximum over ranks and the value is the
particle-steps of all ranks per second (weak scaling, no collective on the
data path).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload instead (rank 0 only), one process and box per host core.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CR particle-steps/s (push+deposit), % HBM roofline; mixed vs FP64 at stated err"
UNIT = "particle-steps/s"

# bytes the method must move per particle-step in the push kernel: particle
# state read + write (mixed: int32 cell, D f32 offsets, the two-word
# four-velocity as 3 f32 leading words and one packed residual word; FP64:
# D + 3 doubles)
PARTICLE_BYTES = {(3, "mixed"): 32, (2, "mixed"): 28, (3, "fp64"): 48, (2, "fp64"): 40}
# bytes a mixed-precision particle occupies (two 16-byte records; in 2-D the
# third offset slot is padding), what host copies move
RECORD_BYTES = {(3, "mixed"): 32, (2, "mixed"): 32, (3, "fp64"): 48, (2, "fp64"): 40}
# per cell and launch: staged E, B read once (6 words) + 8 deposit channels
# read-modify-written once (8 B each, twice)
CELL_FIELD_BYTES = {"mixed": 24, "fp64": 48}
CELL_DEPOSIT_BYTES = 8 * 8 * 2
# per cell, algorithmic bytes of the coupled step's gas kernels (FP64 gas):
# predictor reads rho, mom(3), egas, B(3) and the moments n, J (4 x int64),
# writes the half state (8 doubles), the staged mixed fields (32 B) and clears
# the next moments (4 x int64); corrector reads the corrector deposit
# (4 x int64), the half state rho, mom(3), B(3) and the gas mom(3), egas, B(3),
# writes mom, egas, B and clears the deposit (4 x int64)
GAS_PREDICT_BYTES = 64 + 32 + 64 + 32 + 32
GAS_CORRECT_BYTES = 32 + 56 + 56 + 56 + 32
# DRAM bytes (read + write) per particle of one k_push_mixed<D, full> launch,
# measured with ncu (dram__bytes_read.sum + dram__bytes_write.sum) on a small
# case of the current kernel version, a push that applies a sort (reads its
# particles through the permutation, as every push does at a sort cadence of
# one); traffic scales with the particle count (cells scale alike at fixed
# particles per cell).  Remove an entry whenever its kernel changes, until it
# is measured again.  Both from 'ncu --set full' of one launch: the 3-D beam at
# 64^3 x 32 (590.9 MB for 8,388,608 particles), Bell at 512^2 x 64 (1183.5 MB
# for 16,777,216 particles); commands in profiles/.
PUSH_TRAFFIC_BYTES_PER_PARTICLE = {"alfvenic_beam_3d": 590.871296e6 / 8388608,
                                   "bell_2d": 1183.462144e6 / 16777216}
# int32 shared-memory atomic adds per particle of the push's two TSC deposits:
# 8 channels on 3^D cells, one word per contribution for the charge density
# and two (hi, lo) for the other seven channels, and one contribution count
# per deposit
SMEM_ATOMICS_PER_PARTICLE = {3: 27 * (1 + 7 * 2) + 2, 2: 9 * (1 + 7 * 2) + 2}
# SM-cycles per warp-wide 32-bit shared atomic add with its 32 lanes on 32
# banks, each adding its own value (standalone probe on a GB300)
SMEM_ATOMIC_CYCLES = 1.1
# Shared-memory wavefronts per particle of the push (its shared loads,
# stores and atomics, bank conflicts included), from the same captures as
# the traffic above (l1tex__data_pipe_lsu_wavefronts_mem_shared.sum:
# 307,599,692 for the 3-D beam at 64^3 x 32, 186,552,819 for Bell at
# 512^2 x 64); remove an entry whenever its kernel changes.
PUSH_SHARED_WAVEFRONTS_PER_PARTICLE = {"alfvenic_beam_3d": 307599692 / 8388608,
                                       "bell_2d": 186552819 / 16777216}
# wavefronts per SM-cycle that a standalone probe of warp-wide shared atomic
# adds reaches on this GPU with the deposit tile's own address pattern (the
# highest rate measured for the pipe)
SHARED_PIPE_WAVEFRONTS_PER_CYCLE = 0.93


def _rank_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


WORKLOADS = {
    "alfvenic_beam_3d": "3-D periodic {n}^3 grid, {ppc} CR/cell, uniform gas + random-phase Alfvenic dB/B0=0.1 "
                        "(64 modes), beam |p|=100 boosted 10 v_A along B, C=300, TSC, no Hall term",
    "bell_2d": "2-D periodic {n2d}^2 grid, 64 CR/cell, B along x, dN/dp ~ p^-2 on [10, 1e4] drifting 0.5 v_A, "
               "C=300, CR-Hall term on",
    "shock_2d": "2-D 16384x128 grid, reflecting x walls, 40 CR/cell average with 80% in the 5% of cells "
                "nearest the wall, upstream v=-20 v_A, dN/dp ~ p^-2 on [1, 1e5], C=200",
    "shock_front_2d": "2-D 16384x128 grid, conducting wall at x=0 and open inflow face, shocked gas (front at "
                      "x=4096: rho 4, v 0, P1=(4/3) rho0 v0^2 behind it; rho0 1, v=-20 v_A ahead), 40 CR/cell "
                      "average with 80% in the 5% of cells nearest the wall, 25% free slots, dN/dp ~ p^-2 on "
                      "[1, 1e5], C=200; CR injection at the tracked front (eta 2e-3, 10 E_sh) timed apart",
    "ensemble_2d": "96 independent 2-D periodic boxes, sides log-uniform in [32, 512], 4-64 CR/cell, "
                   "dB/B0 in [0, 0.3], |p|=10, C=100, advanced together",
    "periodic_thermal_2d": "2-D periodic 64^2 grid, 16 CR/cell, uniform gas, B along x, |p|=10, C=100",
}


def _workload(args, seed):
    """The boxes of the selected workload and their common time step."""
    from paper_1412_1087_gb300 import workloads as wl
    if args.workload == "alfvenic_beam_3d":
        boxes = [wl.alfvenic_beam_3d(seed=seed, n=args.n, ppc=args.ppc)]
    elif args.workload == "bell_2d":
        boxes = [wl.bell_2d(seed=seed, n=args.n2d)]
    elif args.workload == "shock_2d":
        boxes = [wl.shock_2d(seed=seed)]
    elif args.workload == "shock_front_2d":
        boxes = [wl.shock_front_2d(seed=seed, nx=16384, ny=128, ppc=40.0, front=0.25)]
    elif args.workload == "ensemble_2d":
        boxes = wl.ensemble_2d(nbox=96, seed0=seed * 1000)
    else:
        boxes = [wl.periodic_thermal_2d(seed=seed)]
    return boxes, min(b.dt for b in boxes)


def _workload_desc(args):
    d = WORKLOADS[args.workload].format(n=args.n, ppc=args.ppc, n2d=args.n2d)
    return args.workload + ": " + d


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def aggregate_ranks(total_ms: float, particle_steps: float, dist=None, device=None):
    """Whole-job figures over ranks: the slowest rank's time and the sum of the
    particle-steps all ranks advanced (weak scaling, no data-path collective)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return total_ms, particle_steps
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    n = torch.tensor([particle_steps], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def smem_atomic_roofline(ndim, npart, push_avg_s, sm_mhz, nsm):
    """The push against the conflict-free rate of the shared-memory atomic
    pipe: the deposits' warp-wide atomic instructions per second over one
    per SMEM_ATOMIC_CYCLES SM-cycles on every SM at the sampled clock.  Bank
    conflicts (lanes whose particles share a cell) raise the cycles an
    instruction takes above that rate, so frac < 1 counts them too."""
    per = SMEM_ATOMICS_PER_PARTICLE[ndim]
    achieved = per / 32.0 * npart / push_avg_s / 1e9
    peak = nsm * sm_mhz * 1e6 / SMEM_ATOMIC_CYCLES / 1e9
    return {"bound": "shared-memory atomics", "achieved": achieved, "peak": peak,
            "unit": "G warp atomic instructions/s", "frac": achieved / peak,
            "atomics_per_particle": per, "cycles_per_instruction": SMEM_ATOMIC_CYCLES,
            "sm_mhz": sm_mhz, "sms": nsm}


def shared_pipe_roofline(wavefronts_per_particle, npart, push_avg_s, sm_mhz, nsm):
    """The push against the shared-memory pipe it is bound by: its measured
    wavefronts per particle (conflicts included) per second over the probe's
    rate on every SM at the given clock."""
    achieved = wavefronts_per_particle * npart / push_avg_s / 1e9
    peak = nsm * sm_mhz * 1e6 * SHARED_PIPE_WAVEFRONTS_PER_CYCLE / 1e9
    return {"bound": "shared-memory pipe", "achieved": achieved, "peak": peak,
            "unit": "G wavefronts/s", "frac": achieved / peak,
            "wavefronts_per_particle": wavefronts_per_particle,
            "wavefronts_per_cycle_peak": SHARED_PIPE_WAVEFRONTS_PER_CYCLE, "sm_mhz": sm_mhz, "sms": nsm}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _time_engine(eng, dt, steps, warmup, sort_every, torch, per_push=True, lookahead=None):
    """Run warmup + timed steps; returns (total_ms, push_ms_sum, launches).
    With a look-ahead (in steps) the sorts here look sort_every times as far
    ahead, as mhdpic_run's sorts at that cadence do; it is restored after."""
    st = eng.stream
    if lookahead is not None:
        eng.set_sort_lookahead(lookahead * dt * max(sort_every, 1))
    for k in range(warmup):
        eng.interp_push(dt, 1)
        eng.apply_feedback(False)
        if sort_every and (k + 1) % sort_every == 0:
            eng.sort()
    torch.cuda.synchronize()
    l0 = eng.launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(st)
    for k in range(steps):
        if per_push:
            ev[k][0].record(st)
        eng.interp_push(dt, 1)
        if per_push:
            ev[k][1].record(st)
        eng.apply_feedback(False)
        if sort_every and (k + 1) % sort_every == 0:
            eng.sort()
    end.record(st)
    torch.cuda.synchronize()
    total = start.elapsed_time(end)
    push = sum(a.elapsed_time(b) for a, b in ev) if per_push else float("nan")
    if lookahead is not None:
        eng.set_sort_lookahead(lookahead * dt)
    return total, push, eng.launches() - l0


def _time_run(eng, dt, steps, warmup, sort_every, torch):
    """Time `steps` steps of mhdpic_run at the given cadence after `warmup`
    untimed ones; returns the total ms (events on the library's stream)."""
    st = eng.stream
    if warmup:
        eng.run(dt, warmup, sort_every)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(st)
    eng.run(dt, steps, sort_every)
    end.record(st)
    torch.cuda.synchronize()
    return start.elapsed_time(end)


def _whole_cycles(steps, k):
    """(warm-up, timed) step counts for a side measurement at sort cadence k:
    one whole cycle of warm-up, so that its last step sorts and the timed
    steps start where every cycle starts, and whole cycles timed."""
    k = max(int(k), 1)
    return k, k * max(1, -(-int(steps) // k))


def _sample_box(args, seed, size):
    """A bounded sample of the selected workload's recipe ('cpu' or 'err' size)."""
    from paper_1412_1087_gb300 import workloads as wl
    big = size == "cpu"
    if args.workload == "alfvenic_beam_3d":
        n = args.sample_n if big else args.err_n
        return wl.alfvenic_beam_3d(seed=seed, n=n, ppc=args.ppc), "%d^3 x %d CR/cell" % (n, args.ppc)
    if args.workload == "bell_2d":
        n = 176 if big else 64
        return wl.bell_2d(seed=seed, n=n), "%d^2 x 64 CR/cell" % n
    if args.workload == "shock_2d":
        nx, ny = (2048, 32) if big else (512, 16)
        return wl.shock_2d(seed=seed, nx=nx, ny=ny), "%d x %d, 40 CR/cell average" % (nx, ny)
    if args.workload == "shock_front_2d":
        nx, ny = (2048, 32) if big else (512, 16)
        return (wl.shock_front_2d(seed=seed, nx=nx, ny=ny, ppc=40.0, front=0.25),
                "%d x %d, 40 CR/cell average" % (nx, ny))
    if args.workload == "ensemble_2d":
        side = 256 if big else 64
        b = wl.ensemble_2d(nbox=1, seed0=seed * 1000, max_side=side)[0]
        return b, "one ensemble box, side %d" % b.n[0]
    return wl.periodic_thermal_2d(seed=seed), "64^2 x 16 CR/cell"


def _cpu_baseline(args, seed, nsteps):
    import oracle as orc
    from paper_1412_1087_gb300 import workloads as wl
    box, what = _sample_box(args, seed, "cpu")
    st = orc.State(box, wl.absolute_positions(box), box.p.astype(np.float64))
    t0 = time.perf_counter()
    for _ in range(nsteps):
        st.step(box.dt)
    dt = time.perf_counter() - t0
    live = int((box.cell >= 0).sum())
    return {"value": live * nsteps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%s recipe at %s (%d CRs), %d full steps, single thread"
                      % (args.workload, what, live, nsteps), "seconds": dt}


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _cpu_replica(workload, sample_n, ppc, seed, nsteps, warmup, barrier, queue, wait_s):
    """One host process of the all-core oracle figure: its own sample box,
    built (and advanced warmup untimed steps) before the common start, then
    nsteps full oracle steps."""
    try:
        import oracle as orc
        from paper_1412_1087_gb300 import workloads as wl
        args = argparse.Namespace(workload=workload, sample_n=sample_n, ppc=ppc, err_n=0)
        box, what = _sample_box(args, seed, "cpu")
        st = orc.State(box, wl.absolute_positions(box), box.p.astype(np.float64))
        for _ in range(warmup):
            st.step(box.dt)
        barrier.wait(timeout=wait_s)
        t0 = time.time()
        for _ in range(nsteps):
            st.step(box.dt)
        queue.put((seed, int((box.cell >= 0).sum()), t0, time.time(), what, None))
    except Exception as e:  # reported to the parent, which then gives up
        barrier.abort()
        queue.put((seed, 0, 0.0, 0.0, "", "%s: %s" % (type(e).__name__, e)))


def _cpu_all_cores(args, nsteps, nproc=None, limit_s=300.0, warmup=0):
    """The oracle as it stands on every host core: one process per core, each
    advancing its own box of the sample recipe (seeds 1000, 1001, ...); all
    start together after building their boxes, and the figure is the
    particle-steps of all processes over the wall time from the common start
    to the last finish.  Processes are spawned, never forked, so that none
    inherits a CUDA context.  A process that fails, or no result within
    limit_s, ends the figure with the reason."""
    import multiprocessing as mp
    import queue as queue_mod
    if nproc is None:
        nproc = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(nproc)
    q = ctx.Queue()
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    os.environ.update({k: "1" for k in _THREAD_VARS})
    procs = [ctx.Process(target=_cpu_replica, daemon=True,
                         args=(args.workload, args.sample_n, args.ppc, 1000 + i, nsteps, warmup, barrier, q, limit_s))
             for i in range(nproc)]
    try:
        for p in procs:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    res, err = [], None
    deadline = time.time() + limit_s
    try:
        for _ in procs:
            r = q.get(timeout=max(1.0, deadline - time.time()))
            if r[5] is not None:
                err = r[5]
                break
            res.append(r)
    except queue_mod.Empty:
        err = "no result within %.0f s" % limit_s
    for p in procs:
        p.join(timeout=5 if err is None else 0.1)
        if p.is_alive():
            p.terminate()
            p.join()
    if err is not None:
        return {"unavailable": err}
    t0 = min(r[2] for r in res)
    wall = max(r[3] for r in res) - t0
    live = sum(r[1] for r in res)
    return {"value": live * nsteps / wall, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": "%d processes, each the %s recipe at %s (%d CRs in all), %d full steps, "
                      "one thread each" % (nproc, args.workload, res[0][4], live, nsteps),
            "seconds": wall}


def _error_vs_oracle(args, seed, torch, nsteps=10):
    """Both GPU paths against the oracle on a sample of the workload: one step
    (relative L2 of each deposited channel, per box), then nsteps steps with
    feedback and no sort (so the particles keep their order) for the largest
    position and momentum deviations."""
    import oracle as orc
    from paper_1412_1087_gb300 import mhdpic as m
    from paper_1412_1087_gb300 import workloads as wl
    if args.workload == "ensemble_2d":
        boxes = wl.ensemble_2d(nbox=8, seed0=seed * 1000, max_side=64)
        what = "8 ensemble boxes of side <= 64"
    else:
        box, what = _sample_box(args, seed, "err")
        boxes = [box]
    dt = min(b.dt for b in boxes)

    def rl(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    states = []
    for b in boxes:
        g = orc.grid_of(b)
        perm, _ = orc.sort_cells(g, (4, 4, 4) if b.ndim == 3 else (8, 8, 1), b.cell)
        x = np.ascontiguousarray(wl.absolute_positions(b)[:, perm])
        v = np.ascontiguousarray(b.p.astype(np.float64)[:, perm])
        states.append((x, v))
    one = [orc.State(b, x, v).push_only(dt) for b, (x, v) in zip(boxes, states)]
    multi = []
    for b, (x, v) in zip(boxes, states):
        st = orc.State(b, x, v)
        for _ in range(nsteps):
            st.step(dt)
        multi.append((st.x, st.v))
    out = {}
    for name, prec in (("mixed", m.MHDPIC_PREC_MIXED), ("fp64", m.MHDPIC_PREC_FP64)):
        eng = m.Engine(boxes, precision=prec)
        eng.interp_push(dt, 1)
        gc = eng.deposits(0).cpu().numpy()
        gm = eng.deposits(1).cpu().numpy()
        eng.close()
        per_box = []
        c0 = 0
        for b, (corr, md) in zip(boxes, one):
            sl = slice(c0, c0 + b.ncell)
            per_box.append({"corrector_rel_l2_max": max(rl(gc[q, sl], corr[q]) for q in range(4)),
                            "moments_rel_l2_max": max(rl(gm[q, sl], md[q]) for q in range(4))})
            c0 += b.ncell
        # nsteps with feedback, no sort
        eng = m.Engine(boxes, precision=prec)
        for _ in range(nsteps):
            eng.interp_push(dt, 1)
            eng.apply_feedback(False)
        if prec == m.MHDPIC_PREC_FP64:
            xg_all = eng.x.cpu().numpy()
        else:
            cell, off = eng.cell.cpu().numpy(), eng.off.cpu().numpy()
        pg_all = eng.velocities().cpu().numpy()
        starts = eng.box_start.copy()
        eng.close()
        dxmax = dpmax = 0.0
        for bi, (b, (xo, vo)) in enumerate(zip(boxes, multi)):
            s, e = starts[bi], starts[bi + 1]
            if prec == m.MHDPIC_PREC_FP64:
                xg = xg_all[:, s:e]
            else:
                c = cell[s:e].astype(np.int64)
                co = [c % b.n[0], (c // b.n[0]) % b.n[1], c // (b.n[0] * b.n[1])]
                xg = np.stack([b.x0[d] + (co[d] + off[d, s:e].astype(np.float64)) * b.dx[d]
                               for d in range(b.ndim)])
                xg[:, c < 0] = np.nan
            live = ~np.isnan(xg[0]) & ~np.isnan(xo[0])
            for d in range(b.ndim):
                L = b.n[d] * b.dx[d]
                dd = xg[d, live] - xo[d, live]
                if b.bc[d] == 0:
                    dd = dd - L * np.round(dd / L)
                if dd.size:
                    dxmax = max(dxmax, float(np.abs(dd).max() / b.dx[d]))
            pg = pg_all[:, s:e][:, live]
            po = vo[:, live]
            if po.size:
                dpmax = max(dpmax, float((np.abs(pg - po).max(axis=0) / np.maximum(
                    np.sqrt((po ** 2).sum(axis=0)), 1e-300)).max()))
        out[name] = {"corrector_rel_l2_max": max(r["corrector_rel_l2_max"] for r in per_box),
                     "moments_rel_l2_max": max(r["moments_rel_l2_max"] for r in per_box),
                     "max_position_deviation_cells_after_%d_steps" % nsteps: dxmax,
                     "max_momentum_deviation_rel_after_%d_steps" % nsteps: dpmax}
        if len(boxes) > 1:
            out[name]["per_box"] = per_box
    out["sample"] = "one step, then %d steps with feedback and no sort, at %s" % (nsteps, what)
    return out


def _build_boxes(name, seed):
    """The full-size boxes of a named workload (for the extra workloads)."""
    ns = argparse.Namespace(workload=name, n=128, ppc=32, n2d=1024)
    return _workload(ns, seed)


def _measure_workload(name, boxes, dt, args, torch, m, dev, stream, peak, peak_kind):
    """One more full-size workload, measured as the headline one is: the
    library's tuner picks the sort cadence on real steps, then args.steps
    eager steps (every push bracketed by events: the push kernel's roofline)
    and args.steps graph-replayed steps (the rate); the worst per-box errors
    against the oracle come from _error_vs_oracle on a sample of the recipe."""
    npart = sum(int((b.cell >= 0).sum()) for b in boxes)
    ncell = sum(b.ncell for b in boxes)
    ndim = boxes[0].ndim
    eng = m.Engine(boxes, precision=m.MHDPIC_PREC_MIXED, device=dev, stream=stream)
    eng.set_sort_lookahead(args.sort_lookahead * dt)
    eng.set_field_tma(bool(args.field_tma))
    eng.run(dt, 20, 0)
    k = eng.sort_cadence()
    torch.cuda.synchronize()
    _, push_ms, _ = _time_engine(eng, dt, args.steps, _whole_cycles(args.warmup, k)[1], k, torch,
                                 lookahead=args.sort_lookahead)
    for _ in range(args.warmup):
        eng.run(dt, max(k, 1), k)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = eng.launches()
    ev0.record(stream)
    eng.run(dt, args.steps, k)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = eng.launches() - l0
    flags = eng.status()
    eng.close()
    del eng
    torch.cuda.empty_cache()
    push_avg_s = push_ms / args.steps / 1e3
    bytes_push = npart * 2 * PARTICLE_BYTES[(ndim, "mixed")] + ncell * (CELL_FIELD_BYTES["mixed"] + CELL_DEPOSIT_BYTES)
    achieved = bytes_push / push_avg_s / 1e9
    out = {"workload": _workload_desc(argparse.Namespace(workload=name, n=128, ppc=32, n2d=1024)),
           "boxes": len(boxes), "particles": npart, "cells": ncell, "dt": dt, "sort_every": k,
           "value": float(npart) * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
           "steps": args.steps, "gpu_launches_per_step": launches / args.steps,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "kernel": "k_push_mixed<%d,full>" % ndim, "peak_kind": peak_kind,
                        "bytes_per_launch": bytes_push, "avg_launch_ms": push_avg_s * 1e3},
           "status_flags": m.status_names(flags)}
    if args.err_n > 0:
        err = _error_vs_oracle(argparse.Namespace(workload=name, err_n=args.err_n, sample_n=args.sample_n,
                                                  ppc=args.ppc), 0, torch)
        worst = {}
        for prec in ("mixed", "fp64"):
            e = err[prec]
            worst[prec] = {kk: e[kk] for kk in e if kk != "per_box"}
        out["error_vs_oracle"] = dict(worst, sample=err["sample"])
    return out


def run_native(args):
    import torch
    from paper_1412_1087_gb300 import build as libbuild
    from paper_1412_1087_gb300 import mhdpic as m

    rank, world, lrank = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(lrank)
    if rank == 0:
        libbuild.build()
    if world > 1:
        dist.barrier()
    m.load()
    dev = "cuda:%d" % lrank
    boxes, dt = _workload(args, seed=rank)
    # the other full-size workloads the default run also measures, built on a
    # host thread while the GPU times the headline box (numpy releases the
    # GIL in its array operations)
    extra_names = [w for w in (args.extra_workloads.split(",") if args.extra_workloads else [])
                   if w and w != args.workload]
    extra_boxes = {}

    def _build_extra():
        for w in extra_names:
            try:
                extra_boxes[w] = _build_boxes(w, seed=rank)
            except Exception as e:  # reported in the line, never fatal
                extra_boxes[w] = e

    import threading
    extra_thread = threading.Thread(target=_build_extra, daemon=True)
    if extra_names:
        extra_thread.start()
    npart = sum(int((b.cell >= 0).sum()) for b in boxes)   # particles, not free slots
    ncell = sum(b.ncell for b in boxes)
    ndim = boxes[0].ndim
    # the layout (brick shape, hence particles per block) picked by the
    # project's tuner on copies of the boxes, unless given
    brick = (0, 0, 0)
    layout = None
    if args.tune_layout:
        from paper_1412_1087_gb300 import tune
        layout = tune.tune_layout(boxes, steps=8, device=dev, lookahead=args.sort_lookahead)
        brick = tuple(layout["brick"])
        torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    eng = m.Engine(boxes, precision=m.MHDPIC_PREC_MIXED, brick=brick, device=dev, stream=stream)
    # sorts key the particles by the cell they reach in this much time (half
    # a step: the cell where the next push gathers and deposits the corrector)
    eng.set_sort_lookahead(args.sort_lookahead * dt)
    eng.set_field_tma(bool(args.field_tma))

    # sort cadence: given, or picked by the library's tuner (mhdpic_run with
    # sort_every = 0 times one cycle of each candidate cadence on real steps)
    # totals of gas + CR momentum and energy before any step (no corrector
    # is pending here, so this feedback call changes nothing)
    tot0 = eng.apply_feedback(totals=True).sum(axis=0)
    steps_done = 0
    tuned = args.sort_every == 0
    if tuned:
        eng.run(dt, 20, 0)
        torch.cuda.synchronize()
        args.sort_every = eng.sort_cadence()
        steps_done += 20

    # eager steps, one call each, so that every push kernel is bracketed by
    # events on the library's stream: the push kernel's roofline
    # warm-up rounded up to whole sort cycles: the timed pushes keep the
    # steady-state distances from their sorts
    eager_warm = _whole_cycles(args.warmup, args.sort_every)[1]
    eager_ms, push_ms, _ = _time_engine(eng, dt, args.steps, eager_warm, args.sort_every, torch,
                                        lookahead=args.sort_lookahead)
    steps_done += args.steps + eager_warm
    # the sort alone (keys, scan, scatter, segment sort, work list), a few calls
    sev0, sev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eng.sort()
    torch.cuda.synchronize()
    sev0.record(stream)
    for _ in range(3):
        eng.sort()
    sev1.record(stream)
    torch.cuda.synchronize()
    sort_ms = sev0.elapsed_time(sev1) / 3

    # timed region (device time, max over ranks): the production step, the
    # cycle of push + feedback + sort at the tuned cadence captured once in a
    # CUDA graph and replayed by mhdpic_run
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        eng.run(dt, max(args.sort_every, 1), args.sort_every)   # capture, then replays
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(lrank) as clk:
        l0 = eng.launches()
        ev0.record(stream)
        eng.run(dt, args.steps, args.sort_every)
        ev1.record(stream)
        torch.cuda.synchronize()
        launches = eng.launches() - l0
    clocks = clk.summary()
    steps_done += args.warmup * max(args.sort_every, 1) + args.steps
    # the same graph-replayed steps with the step split into its separate
    # launches (scales, push, feedback + staging) in turn on one stream
    # against the form the timed region used: the one-launch step, or at a
    # sort every step the feedback on a second stream beside the sort; on
    # this box in this run
    fused_form = "feedback_beside_sort" if args.sort_every == 1 else "one_launch"
    fusion = {"one_launch_steps": bool(eng.step_fusion()) and args.sort_every != 1,
              "form": fused_form if eng.step_fusion() else "separate_launches"}
    if eng.step_fusion() and args.fusion_ab:
        ab = {}
        for fuse in (False, True):
            eng.set_step_fusion(fuse)
            eng.run(dt, max(args.sort_every, 1) * 2, args.sort_every)   # capture and warm up
            torch.cuda.synchronize()
            ev0.record(stream)
            eng.run(dt, args.steps, args.sort_every)
            ev1.record(stream)
            torch.cuda.synchronize()
            ab[fused_form if fuse else "separate_launches"] = ev0.elapsed_time(ev1) / args.steps
            steps_done += max(args.sort_every, 1) * 2 + args.steps
        fusion["ms_per_step"] = ab
    # the drift is taken over at least args.conservation_steps steps in all:
    # the rest run here, graph-replayed at the same cadence
    if steps_done < args.conservation_steps:
        eng.run(dt, args.conservation_steps - steps_done, args.sort_every)
        steps_done = args.conservation_steps
    tot1 = eng.apply_feedback(totals=True).sum(axis=0)
    # momentum scale: gross gas momentum plus gross CR momentum
    scaleP = 0.0
    pcr = eng.velocities()
    c0 = 0
    for bi, b in enumerate(boxes):
        dV = b.dx[0] * b.dx[1] * b.dx[2]
        scaleP += float(eng.mom[:, c0:c0 + b.ncell].abs().sum().item()) * dV
        s0, s1 = int(eng.box_start[bi]), int(eng.box_start[bi + 1])
        scaleP += b.m_cr * float(pcr[:, s0:s1].abs().sum().item())
        c0 += b.ncell
    scaleP = max(scaleP, 1e-300)
    # only what the boxes conserve: momentum along periodic (and unresolved)
    # axes, a reflecting wall taking up the rest; nothing once particles can
    # leave through an open face
    open_face = any(bc == 2 for b in boxes for bc in b.bc[:b.ndim])
    axes = [] if open_face else [d for d in range(3) if all(d >= b.ndim or b.bc[d] == 0 for b in boxes)]
    dPv = np.abs((tot1[0:3] + tot1[4:7]) - (tot0[0:3] + tot0[4:7]))
    conservation = {"steps": steps_done, "momentum_axes": axes,
                    "momentum_drift": float(dPv[axes].max()) / scaleP if axes else None,
                    "energy_drift": None if open_face else float(abs((tot1[3] + tot1[7]) - (tot0[3] + tot0[7])))
                    / max(abs(float(tot0[3] + tot0[7])), 1e-300)}
    total_ms = ev0.elapsed_time(ev1)
    graph_ms = total_ms / args.steps
    total_ms, job_steps = aggregate_ranks(total_ms, float(npart) * args.steps,
                                          dist if world > 1 else None, dev)
    value = job_steps / (total_ms / 1e3)

    # sub-cycled mode (the paper's production mode, App. A.4): nsub particle
    # sub-steps of dt with the staged fields held fixed per feedback, the
    # corrector summed over the sub-steps, a sort every sort_every sub-steps
    # and after every call
    subcycled = None
    if args.nsub > 1:
        calls = max(2, args.steps // args.nsub)
        eng.set_subcycle_sort(args.sort_every)
        for _ in range(2):
            eng.interp_push(dt, args.nsub)
            eng.apply_feedback(False)
            eng.sort()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(calls):
            eng.interp_push(dt, args.nsub)
            eng.apply_feedback(False)
            eng.sort()
        ev1.record(stream)
        torch.cuda.synchronize()
        sub_ms = ev0.elapsed_time(ev1)
        subcycled = {"nsub": args.nsub, "calls": calls,
                     "value": float(npart) * args.nsub * calls / (sub_ms / 1e3), "unit": UNIT,
                     "ms_per_call": sub_ms / calls}
    # diagnostics (Section 4.3, eq:lambda): a 64-bin log energy spectrum with
    # the E_max sums of eq:emax, and the Lambda map, timed once each after warm-up
    diagnostics = None
    if args.diagnostics:
        edges = np.concatenate([[0.0], np.geomspace(1e-3, 1e6, 64)])
        lam = None
        for _ in range(2):
            eng.spectrum(m.MHDPIC_SPEC_ENERGY, edges, None, 6)
            lam = eng.lambda_map()
        torch.cuda.synchronize()
        ev0.record(stream)
        counts, sums = eng.spectrum(m.MHDPIC_SPEC_ENERGY, edges, None, 6)
        ev1.record(stream)
        torch.cuda.synchronize()
        spec_ms = ev0.elapsed_time(ev1)
        ev0.record(stream)
        lam = eng.lambda_map()
        ev1.record(stream)
        torch.cuda.synchronize()
        diagnostics = {"spectrum_ms": spec_ms, "lambda_map_ms": ev0.elapsed_time(ev1),
                       "spectrum_particles": int(counts.sum()),
                       "E_max_n6": [float(a / b) if b > 0 else None for a, b in sums],
                       "lambda_abs_max": float(lam.abs().max().item())}
        del lam
    # standalone charge/current deposit (mhdpic_deposit), twice: the first
    # call sorts when no sort is pending, the second always reuses one
    standalone = None
    if args.diagnostics:
        torch.cuda.synchronize()
        ms_dep = []
        for _ in range(2):
            ev0.record(stream)
            eng.deposit()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms_dep.append(ev0.elapsed_time(ev1))
        standalone = {"deposit_ms_first_call": ms_dep[0], "deposit_ms": ms_dep[1]}
    # coupled MHD-PIC step (App. A.3, eq:scheme): gas predictor with the
    # half-step field staging, push, gas corrector, sort at the cadence above;
    # the plane-parallel linear MHD gas model where every box is x-periodic,
    # else the CR sources alone
    coupled = None
    if args.coupled_steps > 0:
        lin = all(b.bc[0] == 0 for b in boxes)
        model = m.MHDPIC_GAS_LINEAR_X if lin else m.MHDPIC_GAS_SOURCES
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        t_pred = t_corr = t_all = 0.0
        for k in range(2 + args.coupled_steps):
            timed = k >= 2
            if timed:
                evs[0].record(stream)
            eng.gas_predict(dt, model)
            if timed:
                evs[1].record(stream)
            eng.interp_push(dt, 1)
            if timed:
                evs[2].record(stream)
            eng.gas_correct(dt, model)
            if timed:
                evs[3].record(stream)
            if args.sort_every and (k + 1) % args.sort_every == 0:
                eng.sort()
            if timed:
                torch.cuda.synchronize()
                t_pred += evs[0].elapsed_time(evs[1])
                t_corr += evs[2].elapsed_time(evs[3])
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(args.coupled_steps):
            eng.gas_predict(dt, model)
            eng.interp_push(dt, 1)
            eng.gas_correct(dt, model)
            if args.sort_every and (k + 1) % args.sort_every == 0:
                eng.sort()
        ev1.record(stream)
        torch.cuda.synchronize()
        t_all = ev0.elapsed_time(ev1)
        K = args.coupled_steps
        coupled = {"model": "linear MHD along x" if lin else "CR sources only", "steps": K,
                   "value": float(npart) * K / (t_all / 1e3), "unit": UNIT, "ms_per_step": t_all / K,
                   "predict_ms": t_pred / K, "correct_ms": t_corr / K,
                   "predict_gbs": ncell * GAS_PREDICT_BYTES / (t_pred / K / 1e3) / 1e9,
                   "correct_gbs": ncell * GAS_CORRECT_BYTES / (t_corr / K / 1e3) / 1e9}
    # shock boxes (open inflow face): front tracking and CR injection each
    # step (Section 5), timed apart; every call sorts before and after
    injection = None
    if args.inject_steps > 0 and all(b.bc[0] == 2 for b in boxes) and len(boxes) == 1:
        eta = 2e-3
        for _ in range(2):
            eng.interp_push(dt, 1)
            eng.apply_feedback(False)
            eng.inject(dt, eta, 10.0, 5.0 / 3.0, 11)
        torch.cuda.synchronize()
        ev2 = torch.cuda.Event(enable_timing=True)

        def inject_steps():
            t_step = t_inj = 0.0
            n_inj = 0
            front = None
            for _ in range(args.inject_steps):
                ev2.record(stream)
                eng.interp_push(dt, 1)
                eng.apply_feedback(False)
                ev0.record(stream)
                n, xs, xt = eng.inject(dt, eta, 10.0, 5.0 / 3.0, 11)
                ev1.record(stream)
                torch.cuda.synchronize()
                t_step += ev2.elapsed_time(ev0)
                t_inj += ev0.elapsed_time(ev1)
                n_inj += n
                front = (xs, xt)
            return t_step / args.inject_steps, t_inj / args.inject_steps, n_inj, front

        step_ms, inj_ms, n_inj, front = inject_steps()
        # early-particle removal (Section 5): every particle injected from
        # here on is early (t_early far ahead) and goes at twice its
        # injection time; the step then also carries the injection times
        # through the sort and checks them in the push
        eng.set_injection_times(None, 0.0, 1e30)
        live0 = eng.live_particles()
        step_tr_ms, inj_tr_ms, n_tr, _ = inject_steps()
        injection = {"calls": args.inject_steps, "ms_per_call": inj_ms,
                     "particles_per_call": n_inj / args.inject_steps, "eta": eta, "energy_factor": 10.0,
                     "front_x": front[0], "tail_x": front[1], "live_particles": eng.live_particles(),
                     "step_ms": step_ms,
                     "removal": {"step_ms": step_tr_ms, "inject_ms_per_call": inj_tr_ms,
                                 "injected": n_tr, "live_before": live0,
                                 "live_after": eng.live_particles()}}
    flags = eng.status()
    field_tma = bool(eng.field_tma())

    # roofline of the push kernel (the dominant kernel)
    peak, peak_kind = _peaks()
    prec = "mixed"
    bytes_push = npart * 2 * PARTICLE_BYTES[(ndim, prec)] + ncell * (CELL_FIELD_BYTES[prec] + CELL_DEPOSIT_BYTES)
    push_avg_s = push_ms / args.steps / 1e3
    achieved = bytes_push / push_avg_s / 1e9
    try:
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz, mhz_kind = clocks.get("sm_mhz"), "median sampled under load"
        if not mhz:
            mhz, mhz_kind = 2070.0, "nominal maximum"
        smem = dict(smem_atomic_roofline(ndim, npart, push_avg_s, float(mhz), nsm), sm_mhz_kind=mhz_kind)
        pipe = None
        if args.workload in PUSH_SHARED_WAVEFRONTS_PER_PARTICLE:
            pipe = dict(shared_pipe_roofline(PUSH_SHARED_WAVEFRONTS_PER_PARTICLE[args.workload], npart, push_avg_s,
                                             float(mhz), nsm), sm_mhz_kind=mhz_kind)
    except Exception as e:  # a secondary figure never costs the line
        smem = {"unavailable": "%s: %s" % (type(e).__name__, e)}
        pipe = None
    traffic = None
    if args.workload in PUSH_TRAFFIC_BYTES_PER_PARTICLE:
        traffic = PUSH_TRAFFIC_BYTES_PER_PARTICLE[args.workload] * npart
    eng_stats = {"field_tma": field_tma, "sort_ms": sort_ms,
                 "push_ms_per_step": push_ms / args.steps, "graph_run_ms_per_step": graph_ms,
                 "eager_ms_per_step": eager_ms / args.steps,
                 "subcycled": subcycled, "diagnostics": diagnostics, "coupled": coupled,
                 "injection": injection, "layout_tuning": layout, "conservation": conservation,
                 "standalone_deposit": standalone, "step_fusion": fusion,
                 "particles": npart, "cells": ncell,
                 "dt": dt}

    # plain FP64 GPU path on the same boxes
    fp64 = None
    eng.close()
    del eng
    torch.cuda.empty_cache()
    if args.fp64_steps > 0:
        e64 = m.Engine(boxes, precision=m.MHDPIC_PREC_FP64, device=dev, stream=stream)
        e64.set_sort_lookahead(args.sort_lookahead * dt)
        w64, n64 = _whole_cycles(args.fp64_steps, args.sort_every)
        t64, _, _ = _time_engine(e64, dt, n64, w64, args.sort_every, torch, lookahead=args.sort_lookahead)
        v64 = npart * n64 / (t64 / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": t64 / n64,
                "steps": n64, "speedup_mixed_over_fp64": value / world / v64}
        e64.close()
        del e64
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers (copies inside the timed
    # region).  Headline: the particles stay resident on the device and every
    # step uploads the gas state a host MHD solver owns (rho, mom, egas, B) and
    # reads back the fed-back mom, egas.  Detail: every buffer on the host, so
    # each call also moves the particles both ways.
    e2e = None
    e2e_all_host = None
    if args.e2e_steps > 0:
        gas_h2d = ncell * 8 * 8                 # feedback reads rho, mom(3), egas, B(3)
        gas_d2h = ncell * 4 * 8                 # and writes mom(3), egas
        pbytes = npart * RECORD_BYTES[(ndim, prec)]
        runs = [(m.MHDPIC_MEM_HOST_GAS, gas_h2d, gas_d2h)]
        if args.e2e_all_host:
            # push moves the particles both ways, and so does every sort
            sort_extra = pbytes / args.sort_every if args.sort_every else 0
            runs.append((m.MHDPIC_MEM_HOST, gas_h2d + pbytes + sort_extra, gas_d2h + pbytes + sort_extra))
        res = []
        for mem, h2d, d2h in runs:
            eh = m.Engine(boxes, precision=m.MHDPIC_PREC_MIXED, memory=mem, brick=brick, device=dev, stream=stream)
            eh.set_sort_lookahead(args.sort_lookahead * dt)
            we, ne = _whole_cycles(args.e2e_steps, args.sort_every)
            # the production call, mhdpic_run at the cadence of the timed
            # region (with host buffers its steps run eagerly), and the same
            # steps as one call per stage (interp_push, apply_feedback, sort)
            te = _time_run(eh, dt, ne, we, args.sort_every, torch)
            tc, _, _ = _time_engine(eh, dt, ne, we, args.sort_every, torch, per_push=False,
                                    lookahead=args.sort_lookahead)
            eh.close()
            del eh
            torch.cuda.empty_cache()
            te, e2e_steps = aggregate_ranks(te, float(npart) * ne, dist if world > 1 else None, dev)
            tc, _ = aggregate_ranks(tc, float(npart) * ne, dist if world > 1 else None, dev)
            res.append({"value": e2e_steps / (te / 1e3), "unit": UNIT,
                        "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                        "steps": ne, "ms_per_step": te / ne, "call": "mhdpic_run",
                        "per_stage_calls": {"value": e2e_steps / (tc / 1e3), "ms_per_step": tc / ne}})
        e2e = dict(res[0], mode="particles resident on the GPU, gas state in pinned host memory")
        if len(res) > 1:
            e2e_all_host = dict(res[1], mode="particles and gas in pinned host memory")

    extra = None
    if extra_names:
        extra_thread.join()
        extra = {}
        for w in extra_names:
            b = extra_boxes.get(w)
            if isinstance(b, Exception) or b is None:
                extra[w] = {"unavailable": "%s: %s" % (type(b).__name__, b)}
                continue
            try:
                extra[w] = _measure_workload(w, b[0], b[1], args, torch, m, dev, stream, peak, peak_kind)
            except Exception as e:  # a secondary figure never costs the line
                extra[w] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
            extra_boxes.pop(w, None)
            torch.cuda.empty_cache()

    out = None
    if rank == 0:
        # the oracle's host-core figures are taken at one GPU only
        cpu = _cpu_baseline(args, seed=0, nsteps=args.cpu_steps) if args.cpu_steps > 0 and world == 1 else None
        if cpu is not None and args.cpu_all_cores:
            try:
                # box building plus the steps, a few times the single thread's time
                cpu["all_cores"] = _cpu_all_cores(args, args.cpu_steps, limit_s=120.0 + 10.0 * cpu["seconds"])
            except Exception as e:  # the host figure never costs the GPU line
                cpu["all_cores"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
        err = _error_vs_oracle(args, 0, torch) if args.err_n > 0 else None
        if err is not None:
            err["conservation_drift_this_run"] = eng_stats["conservation"]
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "dtype_detail": "f32 push, int64 fixed-point deposits, f64 gas and totals",
            "data": "synthetic",
            "config": {"workload": _workload_desc(args), "precision": "mixed", "sort_every": args.sort_every, "sort_every_tuned": tuned,
                       "sort_lookahead_steps": args.sort_lookahead,
                       "field_tiles": "tensor copies" if eng_stats.get("field_tma") else "thread copies",
                       "brick": list(brick) if any(brick) else "default", "brick_tuned": bool(args.tune_layout),
                       "l2": "inputs larger than L2 (%.2f GB particle state)"
                             % (npart * RECORD_BYTES[(ndim, prec)] / 1e9),
                       "parallelism": "independent box per GPU" if world > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_push_mixed<%d,full>" % ndim, "peak_kind": peak_kind,
                         "bytes_per_launch": bytes_push, "avg_launch_ms": push_avg_s * 1e3},
            "smem_atomics": smem,
            "shared_pipe": pipe,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64_gpu": fp64,
            "error_vs_oracle": err,
            "status_flags": m.status_names(flags),
            "detail": dict(eng_stats, e2e_all_host=e2e_all_host, workloads=extra),
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def run_reference(args):
    """The oracle as it stands on the host cores, on the selected workload's
    sample recipe: one process and box per core (``--ref-procs``, 0 for every
    core), else, with one process or if the processes fail, a single thread
    in this process."""
    rank, world, _ = _rank_env()
    if rank != 0:
        return None
    import oracle
    oracle.build()
    r = None
    if args.ref_procs != 1:
        r = _cpu_all_cores(args, args.steps, nproc=args.ref_procs or None,
                           limit_s=300.0 + 30.0 * (args.steps + args.warmup), warmup=args.warmup)
    if r is not None and "unavailable" not in r:
        value, cores, sample, dt = r["value"], r["cores"], "FP64 CPU oracle, " + r["sample"], r["seconds"]
    else:
        import oracle as orc
        from paper_1412_1087_gb300 import workloads as wl
        box, what = _sample_box(args, 0, "cpu")
        st = orc.State(box, wl.absolute_positions(box), box.p.astype(np.float64))
        for _ in range(args.warmup):
            st.step(box.dt)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st.step(box.dt)
        dt = time.perf_counter() - t0
        live = int((box.cell >= 0).sum())
        value, cores = live * args.steps / dt, 1
        sample = "FP64 CPU oracle, %s recipe at %s (%d CRs) per step, single thread" % (args.workload, what, live)
        if r is not None:
            sample += " (the processes failed: %s)" % r["unavailable"]
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": _workload_desc(args), "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="alfvenic_beam_3d")
    ap.add_argument("--n", type=int, default=128, help="cells per side of the 3-D box")
    ap.add_argument("--ppc", type=int, default=32)
    ap.add_argument("--n2d", type=int, default=1024, help="cells per side of the 2-D Bell box")
    ap.add_argument("--sort-every", type=int, default=0,
                    help="sort cadence in steps (0: picked by the library's tuner)")
    ap.add_argument("--sort-lookahead", type=float, default=0.5,
                    help="sorts key particles by their cell this many steps ahead (0: the current cell)")
    ap.add_argument("--field-tma", type=int, default=1,
                    help="stage the push's field tiles by tensor copies where possible (0: by the threads)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--diagnostics", type=int, default=1, help="time the spectrum and Lambda map once")
    ap.add_argument("--nsub", type=int, default=5, help="particle sub-steps per call of the sub-cycled figure (<2: off)")
    ap.add_argument("--e2e-all-host", type=int, default=1, help="also time the all-host-buffer mode")
    ap.add_argument("--tune-layout", type=int, default=1,
                    help="pick the brick shape with the layout tuner before the run (0: the default brick)")
    ap.add_argument("--inject-steps", type=int, default=4,
                    help="time front tracking + injection this many calls on shock boxes (0: off)")
    ap.add_argument("--coupled-steps", type=int, default=4,
                    help="time the coupled predictor-corrector step this many steps (0: off)")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="also time the oracle on every host core, one process and box per core (0: off)")
    ap.add_argument("--sample-n", type=int, default=40, help="side of the oracle's sample box")
    ap.add_argument("--ref-procs", type=int, default=0,
                    help="--impl reference: oracle processes, one box each (0: one per host core)")
    ap.add_argument("--err-n", type=int, default=24, help="side of the error-check box (0: skip)")
    ap.add_argument("--fusion-ab", type=int, default=1,
                    help="also time the step as separate launches against the one-launch step (0: off)")
    ap.add_argument("--conservation-steps", type=int, default=1000,
                    help="steps the gas + CR conservation drift is taken over (at least)")
    ap.add_argument("--extra-workloads", default="ensemble_2d,bell_2d",
                    help="other full-size workloads measured in detail.workloads (comma list, '' for none)")
    return ap


def main(argv=None):
    ap = build_parser()
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "native":
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
