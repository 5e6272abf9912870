"""Field tiles staged by tensor copies (mhdpic_set_field_tma).

The staged mixed-precision fields live in padded planes with ghost cells
(periodic copies, mirror images at walls, the last cell beyond an open face),
so every push tile is one box of the planes, copied by two
cp.async.bulk.tensor operations.  The results must be the same bit for bit
as with the tile copied by the threads, across box shapes, boundaries,
ragged bricks and the one-launch step; bricks with an odd x extent (the copy
alignment rule) and FP64 contexts stage by the threads.
"""
import numpy as np
import pytest

from paper_1412_1087_gb300 import workloads as wl
from tests._parity import mixed_rows, tilt_B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402

MIXED = m.MHDPIC_PREC_MIXED


def _case(name):
    if name == "beam3d_ragged":
        return [tilt_B(wl.alfvenic_beam_3d(n=14, ppc=6, nmodes=8, seed=71), 71)], (0, 0, 0)
    if name == "beam3d_brick844":
        return [tilt_B(wl.alfvenic_beam_3d(n=14, ppc=6, nmodes=8, seed=72), 72)], (8, 4, 4)
    if name == "thermal2d_hall":
        b = tilt_B(wl.periodic_thermal_2d(nx=29, ny=21, ppc=9, dv_amp=0.4, seed=73), 73)
        b.hall = 1
        return [b], (0, 0, 0)
    if name == "shock2d_walls":
        return [tilt_B(wl.shock_2d(nx=96, ny=10, ppc=8.0, seed=74), 74, amp=0.1)], (0, 0, 0)
    if name == "shock_front_open":
        return [tilt_B(wl.shock_front_2d(nx=96, ny=10, ppc=8.0, front=0.25, seed=75), 75, amp=0.1)], (0, 0, 0)
    boxes = wl.ensemble_2d(nbox=5, seed0=76, max_side=40)
    boxes[2].cell = boxes[2].cell[:0]
    boxes[2].off = np.ascontiguousarray(boxes[2].off[:, :0])
    boxes[2].p = np.ascontiguousarray(boxes[2].p[:, :0])
    return [tilt_B(b, 77, amp=0.05) for b in boxes], (16, 8, 1)


def _state(eng):
    rows = mixed_rows(eng)
    rows = rows[:, np.lexsort(rows[::-1])]
    return (rows, eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy(), eng.mom.cpu().numpy(),
            eng.egas.cpu().numpy(), eng.fields().cpu().numpy())


@pytest.mark.parametrize("name", ["beam3d_ragged", "beam3d_brick844", "thermal2d_hall", "shock2d_walls",
                                  "shock_front_open", "five_boxes"])
def test_tensor_copies_give_the_same_bits_as_thread_copies(name):
    boxes, brick = _case(name)
    dt = min(b.dt for b in boxes)
    stream = torch.cuda.Stream()
    outs = []
    for tma in (False, True):
        eng = m.Engine(boxes, precision=MIXED, brick=brick, stream=stream)
        assert eng.field_tma() == 1          # the default where the layout allows it
        eng.set_field_tma(tma)
        assert eng.field_tma() == (1 if tma else 0)
        eng.set_sort_lookahead(0.5 * dt)
        for _ in range(3):                   # eager pushes (applying a sort, then not)
            eng.interp_push(dt, 1)
            eng.apply_feedback()
        eng.sort()
        eng.run(dt, 6, 2)                    # one-launch steps from the graph
        stream.synchronize()
        outs.append(_state(eng) + (eng.status(),))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert outs[1][-1] == 0


def test_thread_copies_where_the_layout_rules_out_tensor_copies():
    box = tilt_B(wl.periodic_thermal_2d(nx=17, ny=13, ppc=4, seed=78), 78)
    eng = m.Engine([box], precision=MIXED, brick=(3, 5, 1))   # odd x extent: copy alignment
    assert eng.field_tma() == 0
    eng.set_field_tma(True)
    assert eng.field_tma() == 0
    eng.close()
    eng = m.Engine([box], precision=m.MHDPIC_PREC_FP64)
    assert eng.field_tma() == 0
    eng.close()


def test_copy_wait_limit_raises_a_flag_instead_of_waiting():
    """With a 1 ns limit, a wait that finds its tensor copy still in flight
    (the push's field tile, the key pass's particle records) gives up: the
    launch is flagged MHDPIC_ST_COPY_TIMEOUT and its blocks end after their
    copies have landed.  With the status cleared and the limit restored the
    same context steps normally, its particles in range and finite."""
    box = tilt_B(wl.alfvenic_beam_3d(n=32, ppc=16, nmodes=8, seed=78), 78)
    stream = torch.cuda.Stream()
    eng = m.Engine([box], precision=MIXED, stream=stream)
    assert eng.field_tma() == 1
    m.mhdpic_debug_set_copy_limit(eng.ctx, 1)
    flags = 0
    for _ in range(5):   # each launch has thousands of waits; one that finds a copy in flight suffices
        eng.sort()
        stream.synchronize()
        flags |= eng.status()
        if flags & 128:
            break
        eng.interp_push(box.dt, 1)
        stream.synchronize()
        flags |= eng.status()
        if flags & 128:
            break
    assert flags & 128, m.status_names(flags)
    m.mhdpic_debug_set_copy_limit(eng.ctx, 0)
    eng.clear_status()
    assert eng.status() == 0
    eng.run(box.dt, 4, 2)
    eng.sync_particles()
    stream.synchronize()
    assert eng.status() == 0, m.status_names(eng.status())
    cell = eng.cell.cpu().numpy()
    assert cell.min() >= 0 and cell.max() < box.ncell
    assert np.isfinite(eng.vel.cpu().numpy()).all()
    eng.close()
