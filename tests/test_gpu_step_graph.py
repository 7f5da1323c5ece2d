"""The Arnoldi step issued as one CUDA graph replay against the same step
issued kernel by kernel (sim_ls_step_graph).

Both modes run the same kernels on the same data, so a whole run must give
bit-identical states and the same Newton and FGMRES iteration counts, in
every preconditioner precision and with kernel timers on (the graph's timer
brackets are event nodes read after each replay; both modes must report the
same number of timed launches per family).
"""
import numpy as np
import pytest

import paper_1701_06254_gb300 as R
from paper_1701_06254_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(case, steps, graph, timers=(), **opts):
    g = R.Sim(case, **opts)
    g.ls.step_graph(graph)
    if timers:
        g.ls.kernel_timer(timers)
    g.init_hydrostatic()
    g.advance(steps)
    return g


@pytest.mark.parametrize("prec", [R.PREC_FP64, R.PREC_MIXED, R.PREC_MIXED_BF16], ids=["fp64", "mixed", "bf16"])
def test_graph_replay_is_bit_identical(prec):
    """The channelised 1M-cell physics on a 42x38x8 grid (several RAS tiles,
    a ragged edge, 13 wells): three 10-day steps."""
    c = I.case2(nx=42, ny=38, nz=8)
    a = _run(c, 3, True, precision=prec)
    b = _run(c, 3, False, precision=prec)
    for x, y in zip(a.get_state(), b.get_state()):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))
    sa, sb = a.stats(), b.stats()
    for k in ("newton", "linear_its", "linear_solves"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])


def test_graph_replay_keeps_kernel_timers():
    c = I.case0()
    fams = [R.T_RAS, R.T_ORTHO, R.T_VCYCLE, R.T_SPMV64, R.T_SPMV_PREC]
    a = _run(c, 2, True, timers=fams, precision=R.PREC_MIXED)
    b = _run(c, 2, False, timers=fams, precision=R.PREC_MIXED)
    for x, y in zip(a.get_state(), b.get_state()):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))
    for f in fams:
        na, ma = a.ls.kernel_time(f)
        nb, mb = b.ls.kernel_time(f)
        assert na == nb > 0, (f, na, nb)
        assert ma > 0 and mb > 0, (f, ma, mb)


def test_switching_modes_between_solves():
    """Turning the graph off and on again between steps (the recording is
    dropped and made again) changes nothing."""
    c = I.case0()
    ref = _run(c, 3, True, precision=R.PREC_MIXED)
    g = R.Sim(c, precision=R.PREC_MIXED)
    g.init_hydrostatic()
    for k, on in enumerate((True, False, True)):
        g.ls.step_graph(on)
        g.advance(1)
    for x, y in zip(g.get_state(), ref.get_state()):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))
