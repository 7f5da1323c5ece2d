"""The three launch modes of the FGMRES Arnoldi step (sim_ls_step_graph):
a whole restart cycle from one graph launch with a device-side WHILE node
(2), one graph replay per step (1), and kernel-by-kernel launches (0).

All modes run the same kernels on the same data, so a whole run must give
bit-identical states and the same Newton and FGMRES iteration counts, in
every preconditioner precision and with kernel timers on (the graph's timer
brackets are event nodes read after each replay; both graph-free and
per-step modes must report the same number of timed launches per family).
"""
import numpy as np
import pytest

import paper_1701_06254_gb300 as R
from paper_1701_06254_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(case, steps, mode, timers=(), **opts):
    g = R.Sim(case, **opts)
    g.ls.step_graph(mode)
    if timers:
        g.ls.kernel_timer(timers)
    g.init_hydrostatic()
    g.advance(steps)
    return g


def _same(a, b):
    for x, y in zip(a.get_state(), b.get_state()):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))
    sa, sb = a.stats(), b.stats()
    for k in ("newton", "linear_its", "linear_solves"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])


@pytest.mark.parametrize("prec", [R.PREC_FP64, R.PREC_MIXED, R.PREC_MIXED_BF16], ids=["fp64", "mixed", "bf16"])
def test_launch_modes_are_bit_identical(prec):
    """The channelised 1M-cell physics on a 42x38x8 grid (several RAS tiles,
    a ragged edge, 13 wells): three 10-day steps in each mode."""
    c = I.case2(nx=42, ny=38, nz=8)
    runs = {m: _run(c, 3, m, precision=prec) for m in (2, 1, 0)}
    for m, g in runs.items():
        assert g.ls.graph_mode() == m, (m, g.ls.graph_mode())
    _same(runs[2], runs[0])
    _same(runs[1], runs[0])


@pytest.mark.parametrize("restart,max_lin", [(50, 7), (5, 13)])
def test_device_loop_stops_at_the_iteration_cap(restart, max_lin):
    """Solves cut by max_lin, within one cycle or in the third of three
    restart cycles, end on the device at the same step as the host-driven
    loop, with the same relative residual."""
    c = I.case2(nx=42, ny=38, nz=8)
    out = {}
    for mode in (2, 0):
        g = R.Sim(c, precision=R.PREC_MIXED, restart=restart, max_lin=max_lin)
        g.ls.step_graph(mode)
        g.init_hydrostatic()
        g.begin_step(c.dt)
        g.assemble()
        out[mode] = g.linear_solve(1e-14)
        assert g.ls.graph_mode() == mode
        out[mode] += (g.ls.export(R.X_SOLUTION),)
    assert out[2][0] == out[0][0] == max_lin
    assert out[2][1] == out[0][1]
    np.testing.assert_array_equal(out[2][2], out[0][2])


def test_graph_replay_keeps_kernel_timers():
    """With timers on, the device loop gives way to one replay per step."""
    c = I.case0()
    fams = [R.T_RAS, R.T_ORTHO, R.T_VCYCLE, R.T_SPMV64, R.T_SPMV_PREC]
    a = _run(c, 2, 2, timers=fams, precision=R.PREC_MIXED)
    b = _run(c, 2, 0, timers=fams, precision=R.PREC_MIXED)
    assert a.ls.graph_mode() == 1
    _same(a, b)
    for f in fams:
        na, ma = a.ls.kernel_time(f)
        nb, mb = b.ls.kernel_time(f)
        assert na == nb > 0, (f, na, nb)
        assert ma > 0 and mb > 0, (f, ma, mb)


def test_switching_modes_between_solves():
    """Changing the mode between steps (the recordings are dropped and made
    again) changes nothing."""
    c = I.case0()
    ref = _run(c, 4, 0, precision=R.PREC_MIXED)
    g = R.Sim(c, precision=R.PREC_MIXED)
    g.init_hydrostatic()
    for mode in (2, 0, 1, 2):
        g.ls.step_graph(mode)
        g.advance(1)
        assert g.ls.graph_mode() == mode
    _same(g, ref)
