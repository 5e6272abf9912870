"""Layout autotuner: the brick (field-tile) shape, and with it the particles a
block works on per item, picked by timing real steps.

Each candidate brick gets its own context over copies of the boxes; the
library's own tuner (``mhdpic_run`` with sort_every = 0) picks that layout's
sort cadence, and the candidate is timed over whole graph-replayed cycles of
push + feedback + sort with CUDA events on the context's stream.  The fastest
wins.  The deposits do not depend on the brick (all sums are of the same
per-contribution fixed-point integers), so the choice changes speed only.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

from . import mhdpic as m

# Candidates per dimensionality.  The default bricks (4x4x4, 8x8) have the
# padded, bank-spread tile layout; the others use plain strides.
CANDIDATES = {
    3: [(4, 4, 4), (4, 4, 2), (8, 4, 4), (4, 4, 8)],
    2: [(8, 8, 1), (16, 8, 1), (8, 4, 1), (16, 16, 1)],
}


def tune_layout(boxes: Sequence, precision: int = m.MHDPIC_PREC_MIXED, candidates: Optional[List] = None,
                steps: int = 8, device: str = "cuda:0", lookahead: float = 0.0) -> Dict:
    """Time each candidate brick on copies of ``boxes``, sorting with a
    look-ahead of ``lookahead`` steps (mhdpic_set_sort_lookahead); returns
    {"brick", "sort_every", "ms_per_step", "table": [...]} for the fastest."""
    import torch

    dt = min(b.dt for b in boxes)
    ndim = boxes[0].ndim
    cands = candidates or CANDIDATES[ndim]
    table = []
    best = None
    for brick in cands:
        copies = [b.copy() for b in boxes]
        stream = torch.cuda.Stream(device=device)
        try:
            eng = m.Engine(copies, precision=precision, brick=brick, device=device, stream=stream)
        except m.MhdpicError as e:   # e.g. a tile too large for shared memory
            table.append({"brick": list(brick), "error": str(e)})
            continue
        try:
            eng.set_sort_lookahead(lookahead * dt)
            eng.run(dt, 3 * 4, 0)                  # the library tunes the sort cadence
            k = eng.sort_cadence()
            cycles = max(1, steps // k)
            eng.run(dt, 2 * k, k)                  # capture and warm up the cycle
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            eng.run(dt, cycles * k, k)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / (cycles * k)
            row = {"brick": list(brick), "sort_every": k, "ms_per_step": ms}
            table.append(row)
            if best is None or ms < best["ms_per_step"]:
                best = row
        finally:
            eng.close()
            del eng
            torch.cuda.empty_cache()
    if best is None:
        raise m.MhdpicError("no candidate brick could be set up")
    return {"brick": best["brick"], "sort_every": best["sort_every"], "ms_per_step": best["ms_per_step"],
            "table": table}
