"""Layout autotuner and the independence of the results from the layout
(needs a GPU).  All deposits are sums of the same per-contribution
fixed-point integers whatever brick holds a particle, so the brick shape
changes speed only: deposits and gas bit for bit, particles as a set."""
import numpy as np
import pytest

from paper_1412_1087_gb300 import workloads as wl
from tests._parity import mixed_rows, tilt_B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1412_1087_gb300 import mhdpic as m  # noqa: E402
from paper_1412_1087_gb300 import tune  # noqa: E402


def _state(eng):
    rows = mixed_rows(eng)
    rows = rows[:, np.lexsort(rows[::-1])]
    return (eng.deposits(0).cpu().numpy(), eng.deposits(1).cpu().numpy(), eng.mom.cpu().numpy(),
            eng.egas.cpu().numpy(), rows)


@pytest.mark.parametrize("ndim", [3, 2])
def test_results_do_not_depend_on_the_brick(ndim):
    if ndim == 3:
        box = tilt_B(wl.alfvenic_beam_3d(n=16, ppc=6, nmodes=8, seed=31), 31)
    else:
        box = tilt_B(wl.bell_2d(n=48, ppc=10, seed=32), 32, amp=0.05)
    outs = []
    for brick in tune.CANDIDATES[ndim][:3]:
        eng = m.Engine([box.copy()], precision=m.MHDPIC_PREC_MIXED, brick=brick)
        for s in range(3):
            eng.interp_push(box.dt, 1)
            eng.apply_feedback()
            eng.sort()
        eng.interp_push(box.dt, 1)
        outs.append(_state(eng))
        assert eng.status() == 0
        eng.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)


def test_tune_layout_picks_the_fastest_candidate():
    box = wl.alfvenic_beam_3d(n=24, ppc=8, nmodes=8, seed=33)
    res = tune.tune_layout([box], steps=4)
    timed = [r for r in res["table"] if "ms_per_step" in r]
    assert timed and list(res["brick"]) in [list(b) for b in tune.CANDIDATES[3]]
    assert res["ms_per_step"] == min(r["ms_per_step"] for r in timed)
    assert res["sort_every"] >= 1
