"""GPU vs oracle for the well controls of eqs. (11)-(14) with BHP limits,
control switching and schedule changes, and for capillary pressure (eq. 9).

Assembly is compared element by element to 1e-12 (relative to each block
row's largest entry) with the reordering key bit for bit; whole runs per
step with |dp|/p <= 1e-6, |ds_w| <= 1e-6, Newton counts within one, and the
same well controls (and switch counts) as the oracle after every step.
"""
import copy

import numpy as np
import pytest

import oracle
import paper_1701_06254_gb300 as R
from paper_1701_06254_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PC_SW = (0.2, 0.3, 0.5, 0.7, 0.8)
PC_VAL = (2.0, 1.0, 0.6, 0.3, 0.0)


def _with_capillary(c):
    c.fluid = copy.deepcopy(c.fluid)
    c.fluid.pc_sw, c.fluid.pc = PC_SW, PC_VAL
    return c


def _controls_case(seed, nx=7, ny=6, nz=3, water_rate_producer=True):
    c = _with_capillary(I.small_case(nx, ny, nz, seed=seed))
    c.wells = [I.Well(I.INJ, I.WRATE, 120.0, c.column(0, 0), bhp_limit=260.0),
               I.Well(I.PROD, I.ORATE, 40.0, c.column(nx - 1, ny - 1), bhp_limit=150.0),
               I.Well(I.PROD, I.LRATE, 50.0, c.column(nx - 1, 0), bhp_limit=150.0),
               I.Well(I.PROD, I.WRATE, 10.0, c.column(0, ny - 1)) if water_rate_producer else
               I.Well(I.PROD, I.BHP, 170.0, c.column(0, ny - 1))]
    return c


@pytest.mark.parametrize("seed", [71, 72])
def test_assembly_with_capillary_pressure_and_rate_controls(seed):
    c = _controls_case(seed)
    rng = np.random.default_rng(seed)
    p0, p1 = rng.uniform(185.0, 215.0, c.n), rng.uniform(185.0, 215.0, c.n)
    s0, s1 = rng.uniform(0.22, 0.78, c.n), rng.uniform(0.22, 0.78, c.n)
    pb = np.array([240.0, 160.0, 170.0, 175.0])
    o = oracle.Sim(c)
    o.set_state(p0, s0, pb); o.store_old(); o.set_dt(2.0)
    o.set_state(p1, s1, pb); o.assemble()
    g = R.Sim(c)
    g.set_state(p0, s0, pb); g.begin_step(2.0)
    g.set_state(p1, s1, pb)
    nrm = g.assemble()
    rp, ci, val, b, key = o.system()
    gval, gb = g.ls.export(R.X_VALS), g.ls.export(R.X_RHS)
    a = np.abs(val.reshape(-1, 4)).max(axis=1)
    sc = np.repeat(np.maximum.reduceat(a, rp[:-1]), np.diff(rp))
    err = np.abs(gval - val).reshape(-1, 4).max(axis=1) / sc
    assert err.max() < 1e-12, err.max()
    assert np.abs(gb - b).max() <= 1e-12 * np.abs(b).max()
    np.testing.assert_array_equal(g.ls.export(R.X_KEY), key)
    np.testing.assert_allclose(nrm, o.residual_norm(), rtol=1e-12)


def _compare_step(o, g, k, n0o, n0g):
    po, so, pbo, to = o.get_state()
    pg, sg, pbg, tg = g.get_state()
    assert tg == to, k
    assert np.max(np.abs(pg - po) / np.abs(po)) <= 1e-6, k
    assert np.max(np.abs(sg - so)) <= 1e-6, k
    assert np.max(np.abs(pbg - pbo) / np.abs(pbo)) <= 1e-6, k
    assert abs((g.stats()["newton"] - n0g) - (o.stats()["newton"] - n0o)) <= 1, k
    co, _ = o.well_controls()
    cg, _ = g.well_controls()
    np.testing.assert_array_equal(cg, co)
    assert g.stats()["switches"] == o.stats()["switches"], k


@pytest.mark.parametrize("prec", [R.PREC_FP64, R.PREC_MIXED_BF16], ids=["fp64", "bf16"])
def test_whole_run_with_limits_schedule_and_capillary_pressure(prec):
    """Four steps of 2 days with capillary pressure, an injector held at its
    maximum BHP and an oil-rate producer at its minimum BHP, then a schedule
    change (a BHP producer shut, the injector's rate lowered: it returns to
    its rate) and three more steps in which the liquid-rate producer reaches
    its limit too: states, Newton counts, controls and switch counts follow
    the oracle.  (A water-rate producer is left out: at the connate start no
    water moves, and its rate equation would have no solution.)"""
    c = _controls_case(73, water_rate_producer=False)
    c.dt = 2.0
    c.wells[0].target = 600.0                  # beyond its BHP limit: switched at the first step
    c.wells[1].target = 500.0                  # beyond reach at 150 bar: switched
    o = oracle.Sim(c, newton_tol=1e-9, lin_tol=1e-9, max_lin=200)
    g = R.Sim(c, newton_tol=1e-9, lin_tol=1e-9, max_lin=200, precision=prec)
    o.init_hydrostatic(); g.init_hydrostatic()
    for k in range(7):
        if k == 4:
            for sim in (o, g):
                sim.set_well(3, I.SHUT, 0.0)
                sim.set_well(0, I.WRATE, 60.0, bhp_limit=260.0)
        n0o, n0g = o.stats()["newton"], g.stats()["newton"]
        assert o.advance(1) == 0
        g.advance(1)
        _compare_step(o, g, k, n0o, n0g)
    assert o.stats()["switches"] == 3
    ctrl, _ = g.well_controls()
    np.testing.assert_array_equal(ctrl, [I.WRATE, I.BHP, I.BHP, I.SHUT])


def test_whole_run_held_producer_returns_to_rate():
    """The oracle pin's scenario on the GPU: an oil-rate producer held at its
    minimum BHP returns to its rate once an injector opened by a schedule
    change has raised the pressure, at the same step as in the oracle."""
    c = _with_capillary(I.small_case(6, 5, 3, seed=61))
    c.wells[1] = I.Well(I.PROD, I.ORATE, 150.0, c.column(5, 4), bhp_limit=150.0)
    o = oracle.Sim(c, newton_tol=1e-10, lin_tol=1e-10, max_lin=200)
    g = R.Sim(c, newton_tol=1e-10, lin_tol=1e-10, max_lin=200)
    for sim in (o, g):
        sim.init_hydrostatic(p_datum=160.0)
        sim.set_well(0, I.SHUT, 0.0)
    ctrl_seen = []
    for k in range(7):
        if k == 1:
            for sim in (o, g):
                sim.set_well(0, I.WRATE, 300.0)
        n0o, n0g = o.stats()["newton"], g.stats()["newton"]
        assert o.advance(1) == 0
        g.advance(1)
        _compare_step(o, g, k, n0o, n0g)
        ctrl_seen.append(int(g.well_controls()[0][1]))
    assert ctrl_seen[0] == I.BHP and ctrl_seen[-1] == I.ORATE
