"""The Python binding's buffer checks, on the CPU with a stub in place of
the CUDA library (no GPU, no device memory).

Every call that hands the library a raw pointer must first make sure the
buffer holds as many values of the right type as the library will read or
write; a short or mistyped buffer raises ValueError before the C call.
Valid calls (numpy arrays, and contiguous tensors as the benchmark passes
them) must reach the library unchanged.
"""
import ctypes

import numpy as np
import pytest

import paper_1701_06254_gb300 as R

torch = pytest.importorskip("torch")


class _Stub:
    """Records the entry points called; every call succeeds."""

    def __init__(self, nb=0):
        self.calls = []
        self.nb = nb

    def __getattr__(self, name):
        def f(*args):
            self.calls.append(name)
            if name == "sim_ls_export" and args[-1] is not None:
                args[-1]._obj.value = 2 * self.nb * 8 if args[1] == R.X_RHS else 0
            return 0
        return f


def _sim(n=12, nw=2):
    s = R.Sim.__new__(R.Sim)
    s._L, s.h, s.n, s.nw = _Stub(), None, n, nw
    return s


def _ls(n=12, nw=2, nnzb=40):
    ls = R.LinearSystem.__new__(R.LinearSystem)
    ls._L, ls.h, ls._own = _Stub(n + nw), None, False
    ls.n, ls.nw, ls.nb, ls.nnzb = n, nw, n + nw, nnzb
    return ls


def test_set_state_checks_counts_and_types():
    s = _sim()
    s.set_state(np.zeros(12), np.zeros(12), np.zeros(2))
    s.set_state([0.0] * 12, np.zeros(12, np.float32), np.zeros(3))          # converted; pb may be longer
    s.set_state(torch.zeros(12, dtype=torch.float64), torch.zeros(12, dtype=torch.float64),
                torch.zeros(2, dtype=torch.float64))
    assert s._L.calls.count("sim_set_state") == 3
    bad = [
        (np.zeros(11), np.zeros(12), np.zeros(2)),                            # short p
        (np.zeros(12), np.zeros(13), np.zeros(2)),                            # long sw
        (np.zeros(12), np.zeros(12), np.zeros(1)),                            # short pb
        (torch.zeros(12, dtype=torch.float32), np.zeros(12), np.zeros(2)),    # FP32 tensor
        (torch.zeros(12, dtype=torch.int64), np.zeros(12), np.zeros(2)),      # integer tensor
        (torch.zeros(24, dtype=torch.float64)[::2], np.zeros(12), np.zeros(2)),   # strided tensor
    ]
    for p, sw, pb in bad:
        with pytest.raises(ValueError):
            s.set_state(p, sw, pb)
    assert s._L.calls.count("sim_set_state") == 3


def test_set_state_without_wells():
    s = _sim(nw=0)
    s.set_state(np.zeros(12), np.zeros(12), np.zeros(0))
    s.set_state(np.zeros(12), np.zeros(12), None)
    assert s._L.calls.count("sim_set_state") == 2


def test_get_state_into_caller_buffers():
    s = _sim()
    pinned = (torch.empty(12, dtype=torch.float64), torch.empty(12, dtype=torch.float64),
              torch.empty(2, dtype=torch.float64))                           # as bench.py passes them
    s.get_state(pinned)
    s.get_state((np.zeros(12), np.zeros(12), np.zeros(5)))
    s.get_state()
    assert s._L.calls.count("sim_get_state") == 3
    ro = np.zeros(12)
    ro.flags.writeable = False
    bad = [
        (np.zeros(12, np.float32), np.zeros(12), np.zeros(2)),                # would be reinterpreted
        (np.zeros(10), np.zeros(12), np.zeros(2)),                            # short
        (ro, np.zeros(12), np.zeros(2)),                                      # read-only
        (np.zeros(12), np.zeros(12), np.zeros(1)),                            # short pb
        ([0.0] * 12, np.zeros(12), np.zeros(2)),                              # a list cannot receive
    ]
    for out in bad:
        with pytest.raises(ValueError):
            s.get_state(out)
    assert s._L.calls.count("sim_get_state") == 3


def test_linear_system_buffers():
    ls = _ls()
    ls.set(np.zeros(160), np.zeros(28), np.zeros(12))
    for val, b, key in ((np.zeros(159), np.zeros(28), np.zeros(12)), (np.zeros(160), np.zeros(26), np.zeros(12)),
                        (np.zeros(160), np.zeros(28), np.zeros(14))):
        with pytest.raises(ValueError):
            ls.set(val, b, key)
    assert ls._L.calls.count("sim_ls_set") == 1
    # operators: 2 per block row, the V-cycle one per cell
    for op, n in ((R.OP_SPMV, 28), (R.OP_RAS, 28), (R.OP_CPR, 28), (R.OP_VCYCLE, 12)):
        assert ls.apply(op, np.zeros(n)).shape == (n,)
        with pytest.raises(ValueError):
            ls.apply(op, np.zeros(n + 1))
    ls.apply(99, np.zeros(28))                      # an unknown operator is the library's to reject
    assert ls._L.calls.count("sim_ls_apply") == 5
    ls.residual_norm(np.zeros(28))
    with pytest.raises(ValueError):
        ls.residual_norm(np.zeros(12))
    y, _, _ = ls.solve(1e-8)
    assert y.shape == (28,)
    ls.solve(1e-8, y=np.zeros(28))
    for y in (np.zeros(27), np.zeros(28, np.float32)):
        with pytest.raises(ValueError):
            ls.solve(1e-8, y=y)
    assert ls._L.calls.count("sim_ls_solve") == 2


def test_linear_system_of_a_simulator_skips_the_unknown_block_count():
    """The handle a Sim lends out knows n and nb but not the block count:
    values are converted but not counted."""
    ls = _ls()
    del ls.nnzb
    ls.set(np.zeros(7), np.zeros(28), np.zeros(12))
    assert ls._L.calls == ["sim_ls_set"]


def test_warm_start_grids():
    ws = R.WarmStart.__new__(R.WarmStart)
    ws._L, ws.h = _Stub(), None
    assert ws.forward(np.zeros((2, 3, 4, 8))).shape == (2, 3, 4, 8)
    ws.backward(np.zeros((2, 3, 4, 8)), np.zeros((2, 3, 4, 2)))
    for feat in (np.zeros((2, 3, 4, 2)), np.zeros((3, 4, 8)), np.zeros((0, 3, 4, 8))):
        with pytest.raises(ValueError):
            ws.forward(feat)
    for target in (np.zeros((2, 3, 4, 8)), np.zeros((2, 3, 5, 2))):
        with pytest.raises(ValueError):
            ws.backward(np.zeros((2, 3, 4, 8)), target)
    assert ws._L.calls == ["sim_ws_forward", "sim_ws_backward"]
