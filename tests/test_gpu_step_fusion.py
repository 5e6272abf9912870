"""The one-launch step of mhdpic_run (mhdpic_set_step_fusion): the corrector
scales, the push with both deposits and the feedback with the field staging
in one cooperative kernel whose phases are separated by grid-wide barriers.

It must give the same bits as the separate launches (push, then feedback),
take one launch per step where no sort falls, match the oracle on a batch of
boxes with an empty one, and give up on a barrier after its limit with a
status flag rather than wait (tested with a short limit set from the host; no
kernel is made to stall).
"""
import numpy as np
import pytest

import oracle as orc
from paper_1412_1087_gb300 import workloads as wl
from tests._parity import mixed_rows, rel_l2, sorted_oracle_state, tilt_B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402

MIXED = m.MHDPIC_PREC_MIXED


def _five_boxes():
    boxes = wl.ensemble_2d(nbox=5, seed0=61, max_side=40)
    boxes[2].cell = boxes[2].cell[:0]
    boxes[2].off = np.ascontiguousarray(boxes[2].off[:, :0])
    boxes[2].p = np.ascontiguousarray(boxes[2].p[:, :0])
    for b in boxes:
        tilt_B(b, 62, amp=0.05)
    return boxes


def _case(name):
    if name == "beam3d":
        return [tilt_B(wl.alfvenic_beam_3d(n=12, ppc=6, nmodes=8, seed=63), 63)]
    if name == "thermal2d_hall":
        b = tilt_B(wl.periodic_thermal_2d(nx=29, ny=21, ppc=9, dv_amp=0.4, seed=64), 64)
        b.hall = 1
        b.m_cr = 0.02
        return [b]
    return _five_boxes()


@pytest.mark.parametrize("name", ["beam3d", "thermal2d_hall", "five_boxes"])
@pytest.mark.parametrize("k", [1, 3])
def test_one_launch_steps_equal_separate_launches(name, k):
    boxes = _case(name)
    dt = min(b.dt for b in boxes)
    stream = torch.cuda.Stream()
    nsteps = 4 * k + 1
    outs, launches = [], []
    for fuse in (False, True):
        eng = m.Engine(boxes, precision=MIXED, stream=stream)
        eng.set_sort_lookahead(0.5 * dt)
        eng.set_step_fusion(fuse)
        assert eng.step_fusion() == (1 if fuse else 0)
        l0 = eng.launches()
        eng.run(dt, nsteps, k)
        stream.synchronize()
        launches.append(eng.launches() - l0)
        tot = eng.apply_feedback(totals=True)
        outs.append((mixed_rows(eng), eng.deposits(1).cpu().numpy(), eng.mom.cpu().numpy(),
                     eng.egas.cpu().numpy(), eng.fields().cpu().numpy(), tot, eng.status()))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert outs[1][-1] == 0
    # the corrector-scale and feedback kernels of every step are folded into
    # the push; at a sort every step both run the push, then the feedback
    # beside the sort
    assert launches[0] - launches[1] == (0 if k == 1 else 2 * nsteps), launches


def _particle_rows(eng):
    if eng.x is None:
        return mixed_rows(eng)
    return np.vstack([eng.x.cpu().numpy(), eng.velocities().cpu().numpy()])


@pytest.mark.parametrize("prec,mem", [(MIXED, m.MHDPIC_MEM_DEVICE), (m.MHDPIC_PREC_FP64, m.MHDPIC_MEM_DEVICE),
                                      (MIXED, m.MHDPIC_MEM_HOST_GAS)])
@pytest.mark.parametrize("name", ["beam3d", "thermal2d_hall", "five_boxes"])
def test_feedback_beside_the_sort_equals_the_calls_in_turn(name, prec, mem):
    """At a sort every step, mhdpic_run puts each step's feedback on a second
    stream beside the sort that follows the push (captured in the step graph;
    with the gas in host memory also the gas copies, eagerly); the result is
    the same bits as push, feedback and sort called in turn, in either
    precision."""
    boxes = _case(name)
    dt = min(b.dt for b in boxes)
    stream = torch.cuda.Stream()
    outs = []
    for graph in (True, False):
        eng = m.Engine(boxes, precision=prec, memory=mem, stream=stream)
        eng.set_sort_lookahead(0.5 * dt)
        if graph:
            eng.run(dt, 7, 1)   # one eager cycle, the capture, replays
        else:
            for _ in range(7):
                eng.interp_push(dt, 1)
                eng.apply_feedback()
                eng.sort()
        stream.synchronize()
        tot = eng.apply_feedback(totals=True)
        outs.append((_particle_rows(eng), eng.deposits(1).cpu().numpy(), eng.mom.cpu().numpy(),
                     eng.egas.cpu().numpy(), eng.fields().cpu().numpy(), tot, eng.status()))
        eng.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert outs[0][-1] == 0


def test_one_launch_step_is_one_launch_between_sorts():
    boxes = _case("beam3d")
    dt = boxes[0].dt
    stream = torch.cuda.Stream()
    eng = m.Engine(boxes, precision=MIXED, stream=stream)
    eng.run(dt, 8, 4)                          # aligned, captured and replayed
    l0 = eng.launches()
    eng.run(dt, 8, 4)                          # one replay of the 8-step cycle
    stream.synchronize()
    per_cycle = eng.launches() - l0
    eng.sort()
    l1 = eng.launches()
    eng.sort()
    sort_launches = eng.launches() - l1
    assert per_cycle == 8 + 2 * sort_launches, (per_cycle, sort_launches)
    assert eng.status() == 0
    eng.close()


def test_one_launch_steps_match_the_oracle_on_five_boxes_with_an_empty_one():
    boxes = _five_boxes()
    dt = min(b.dt for b in boxes)
    stream = torch.cuda.Stream()
    eng = m.Engine(boxes, precision=MIXED, stream=stream)
    eng.set_sort_lookahead(0.5 * dt)
    assert eng.step_fusion() == 1
    eng.run(dt, 6, 2)
    tg = eng.apply_feedback(totals=True)
    gm = eng.mom.cpu().numpy()
    assert eng.status() == 0
    starts = eng.box_start.copy()
    eng.close()
    c0 = 0
    for bi, b in enumerate(boxes):
        sl = slice(c0, c0 + b.ncell)
        c0 += b.ncell
        if b.np == 0:
            assert np.array_equal(gm[:, sl], b.mom)   # nothing to feed back
            assert np.all(tg[bi, 4:] == 0)
            continue
        _, _, x, v = sorted_oracle_state(b)
        st = orc.State(b, x, v)
        for _ in range(6):
            st.step(dt)
        to = st.totals()
        mom_scale = np.abs(st.mom).sum() + b.m_cr * np.abs(st.v).sum()
        e_scale = abs(to[3]) + abs(to[7])
        assert np.abs(tg[bi, 4:7] - to[4:7]).max() < 2e-5 * mom_scale
        assert abs(tg[bi, 7] - to[7]) < 2e-5 * e_scale
        assert rel_l2(gm[:, sl], st.mom) < 1e-6
    assert starts[-1] == sum(b.np for b in boxes)


def test_barrier_limit_raises_a_flag_instead_of_waiting():
    """With a 1 ns wait limit every block that is not the last to arrive
    gives up at once: the step is flagged (MHDPIC_ST_BARRIER) and the kernel
    ends.  Clearing the status resets the barrier, and a fresh context on the
    same GPU steps normally."""
    boxes = _case("beam3d")
    dt = boxes[0].dt
    stream = torch.cuda.Stream()
    eng = m.Engine(boxes, precision=MIXED, stream=stream)
    assert eng.step_fusion() == 1
    m.mhdpic_debug_set_barrier_limit(eng.ctx, 1)
    eng.run(dt, 1, 2)   # a cycle of two steps: the first is the one-launch step
    stream.synchronize()
    flags = eng.status()
    assert flags & 64, m.status_names(flags)
    eng.clear_status()
    m.mhdpic_debug_set_barrier_limit(eng.ctx, 0)
    assert eng.status() == 0
    eng.close()
    ref = m.Engine(boxes, precision=MIXED, stream=stream)
    ref.run(dt, 4, 2)
    stream.synchronize()
    assert ref.status() == 0
    ref.close()
