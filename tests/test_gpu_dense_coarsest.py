"""The dense coarsest-level inverse (LU with partial pivoting, then the
columns of the inverse) on matrices that need row swaps.

The simulator's coarse pressure matrices are diagonally dominant, so their
LU never swaps rows.  Here the cells' diagonal blocks are scaled down until
an off-diagonal entry is the largest in its column; with amg_coarse_max at
least the cell count, the hierarchy is level 0 alone and the V-cycle is the
dense solve x = A_pp^{-1} f, compared with numpy's solve of the exported
level-0 operator.  The sizes 32, 60, 90 and 128 cover one to four rows per
lane in the column kernel.
"""
import numpy as np
import pytest

import oracle
import paper_1701_06254_gb300 as R
from paper_1701_06254_gb300 import inputs as I


def _assembled(case, seed):
    """The oracle's assembled Jacobian on seeded (old, new) states."""
    p0, s0, pb0 = I.random_state(case, seed)
    p1, s1, pb1 = I.random_state(case, seed + 1)
    o = oracle.Sim(case)
    o.set_state(p0, s0, pb0); o.store_old(); o.set_dt(1.5)
    o.set_state(p1, s1, pb1); o.assemble()
    return o.system()


def _dense(L):
    n = L["n"]
    a = np.zeros((n, n))
    for i in range(n):
        for q in range(L["rp"][i], L["rp"][i + 1]):
            a[i, L["ci"][q]] = L["v"][q]
    return a


@pytest.mark.gpu
@pytest.mark.parametrize("dims", [(4, 4, 2), (5, 4, 3), (6, 5, 3), (8, 4, 4)])
def test_coarsest_inverse_with_row_swaps(dims):
    sl = pytest.importorskip("scipy.linalg")
    c = I.small_case(*dims, seed=41)
    rp, ci, val, b, key = _assembled(c, 700)
    val = np.array(val, dtype=np.float64)
    for i in range(c.n):                       # cells' diagonal blocks scaled down
        for q in range(rp[i], rp[i + 1]):
            if ci[q] == i:
                val[4 * q:4 * q + 4] *= 0.05
    wc0 = [w.perf_cells[0] for w in c.wells]
    gl = R.LinearSystem(c.nx, c.ny, c.nz, len(c.wells), rp, ci, wc0, precision=R.PREC_FP64,
                        decoupling=R.DEC_NONE, amg_coarse_max=256)
    gl.set(val, b, key)
    gl.setup()
    assert gl.amg_nlev() == 1
    L0 = gl.amg_level(0)
    assert L0["n"] == c.n and L0["coarse_dense"] == 1
    a = _dense(L0)
    _, piv = sl.lu_factor(a)
    assert (piv != np.arange(c.n)).sum() >= c.n // 4    # the factorisation does swap rows
    rng = np.random.default_rng(3)
    for _ in range(3):
        f = rng.standard_normal(c.n)
        x = gl.apply(R.OP_VCYCLE, f)
        xr = np.linalg.solve(a, f)
        assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max()
