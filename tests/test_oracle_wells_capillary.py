"""Pins of the oracle's well controls (eqs. 11-14, BHP limits with control
switching, schedule changes) and capillary pressure (eq. 9), against
invariants and closed forms (no GPU needed).

Readings taken where the paper is silent:
* rate targets are surface volumes (sm3/day): the mass rates of eq. (10)
  divided by each phase's reference density; a producer's target counts
  production as positive; the liquid rate of eq. (14) is oil plus water;
* a rate-controlled well may carry a BHP limit (an injector's maximum, a
  producer's minimum); passing it during a Newton iteration puts the well
  on BHP control at the limit, and at the start of a later time step it
  returns to its rate when at the limit it would deliver more than that
  rate;
* p_c is a table of (s_w, p_c) points joined by straight lines, constant
  beyond its ends; p_w = p_o - p_c(s_w) sets the water density, viscosity,
  potential and perforation drawdown.
"""
import copy
import math

import numpy as np
import pytest

from paper_1701_06254_gb300 import inputs as I

G = 9.80665


def incompressible(g=0.0, pc_sw=(), pc=()):
    return I.Fluid(c_f=(0.0, 0.0), c_r=0.0, c_mu=(0.0, 0.0), g=g, pc_sw=tuple(pc_sw), pc=tuple(pc))


# ---------------------------------------------------------------- p_c ----
PC_SW = (0.2, 0.3, 0.5, 0.7, 0.8)
PC_VAL = (2.0, 1.0, 0.6, 0.3, 0.0)


def _pc_inverse(pc):
    """s_w with p_c(s_w) = pc on the decreasing piecewise-linear table."""
    for k in range(len(PC_SW) - 1):
        if PC_VAL[k + 1] <= pc <= PC_VAL[k]:
            return PC_SW[k] + (PC_VAL[k] - pc) * (PC_SW[k + 1] - PC_SW[k]) / (PC_VAL[k] - PC_VAL[k + 1])
    raise ValueError(pc)


def _column_at_capillary_gravity_equilibrium(nz=10, dz=2.0, top=1000.0):
    """A vertical column of incompressible oil and water in which both phase
    potentials (eq. 5) are uniform: p_o = P0 + rho_o g (z - top), and s_w in
    each cell such that p_c(s_w) = p_o - p_w with p_w = W0 + rho_w g (z - top)."""
    fl = incompressible(g=G, pc_sw=PC_SW, pc=PC_VAL)
    n = nz
    k = np.full(n, 100.0)
    c = I.Case("column", 1, 1, nz, 10.0, 10.0, dz, top, k, k.copy(), k.copy(), np.full(n, 0.2), fl, [],
               dt=5.0, n_steps=1)
    z = top + (np.arange(nz) + 0.5) * dz
    P0, W0 = 200.0, 199.05
    po = P0 + fl.rho_ref[1] * G * (z - top) * 1e-5
    pw = W0 + fl.rho_ref[0] * G * (z - top) * 1e-5
    sw = np.array([_pc_inverse(x) for x in po - pw])
    return c, po, sw


def test_capillary_gravity_equilibrium_is_at_rest(oracle_lib):
    """Capillary-gravity equilibrium: with p_w = p_o - p_c(s_w) (eq. 9) and
    both potentials uniform, no face carries any flux, so the residual of
    eq. (17) vanishes and two time steps change nothing.  The saturations
    span two segments of the p_c table and both phases are mobile."""
    c, po, sw = _column_at_capillary_gravity_equilibrium()
    assert sw.min() > 0.3 and sw.max() > 0.5 and sw.min() < 0.5      # two table segments
    s = oracle_lib.Sim(c, newton_tol=1e-12, lin_tol=1e-12)
    s.set_state(po, sw, np.zeros(0)); s.store_old(); s.set_dt(5.0)
    s.assemble()
    b = s.system()[3]
    # flux that a 1e-3 bar potential difference would drive across one face
    T = 9.869233e-16 * 1e5 / 1e-3 * 86400.0 * 100.0 * 100.0 / 2.0
    scale = T * 1000.0 * 0.1 / 0.5 * 1e-3
    assert np.abs(b).max() < 1e-9 * scale, np.abs(b).max() / scale
    assert s.advance(2) == 0
    p1, s1, _, _ = s.get_state()
    np.testing.assert_allclose(p1, po, rtol=1e-12)
    np.testing.assert_allclose(s1, sw, atol=1e-10)


def test_capillary_pressure_drives_imbibition(oracle_lib):
    """Without gravity or wells, a wetter cell beside a drier one at the same
    oil pressure: p_c is lower in the wetter cell, so its water pressure is
    higher and water flows into the drier cell (eq. 9 into eq. 5); oil
    flows the other way only through the pressure it builds.  Total water
    and oil masses stay put (no wells)."""
    fl = incompressible(pc_sw=PC_SW, pc=PC_VAL)
    fl.c_f = (4.5e-5, 1e-4)
    k = np.full(2, 100.0)
    c = I.Case("pair", 2, 1, 1, 10.0, 10.0, 10.0, 1000.0, k, k.copy(), k.copy(), np.full(2, 0.2), fl, [],
               dt=1.0, n_steps=1)
    s = oracle_lib.Sim(c, newton_tol=1e-12, lin_tol=1e-12)
    s.set_state(np.array([200.0, 200.0]), np.array([0.6, 0.35]), np.zeros(0), 0.0)
    m0 = s.mass()
    assert s.advance(1) == 0
    p1, s1, _, _ = s.get_state()
    assert s1[0] < 0.6 and s1[1] > 0.35                 # water moved from the wetter to the drier cell
    m1 = s.mass()
    np.testing.assert_allclose(m1, m0, rtol=1e-10)


@pytest.mark.parametrize("seed", [41, 42])
def test_jacobian_with_capillary_pressure_and_rate_controls(oracle_lib, seed):
    """Analytic Jacobian against central differences with p_c (its slope
    enters the water density, viscosity, potential and drawdown through
    d/ds_w) and with oil-rate, liquid-rate and water-rate producers."""
    c = I.small_case(3, 3, 2, seed=seed)
    c.fluid = copy.deepcopy(c.fluid)
    c.fluid.pc_sw, c.fluid.pc = PC_SW, PC_VAL
    c.fluid.c_mu = (3e-4, 1e-3)
    c.wells = [I.Well(I.INJ, I.WRATE, 100.0, c.column(0, 0)),
               I.Well(I.PROD, I.ORATE, 30.0, c.column(2, 2)),
               I.Well(I.PROD, I.LRATE, 40.0, c.column(2, 0)),
               I.Well(I.PROD, I.WRATE, 20.0, c.column(0, 2))]
    s = oracle_lib.Sim(c)
    rng = np.random.default_rng(seed)
    # saturations away from the table's breakpoints and the Corey clamps
    def draw(n):
        v = rng.uniform(0.31, 0.69, n)
        return np.where(np.abs(v - 0.5) < 0.02, v + 0.05, v)
    p0, p1 = rng.uniform(190.0, 210.0, c.n), rng.uniform(190.0, 210.0, c.n)
    s0, s1 = draw(c.n), draw(c.n)
    pb1 = np.array([260.0, 120.0, 130.0, 140.0])
    s.set_state(p0, s0, pb1); s.store_old(); s.set_dt(1.5)
    s.set_state(p1, s1, pb1); s.assemble()
    rp, ci, val, b, key = s.system()
    nb = c.n + len(c.wells)
    J = np.zeros((2 * nb, 2 * nb))
    for i in range(nb):
        for q in range(rp[i], rp[i + 1]):
            J[2 * i:2 * i + 2, 2 * ci[q]:2 * ci[q] + 2] = val[4 * q:4 * q + 4].reshape(2, 2)
    x0 = np.concatenate([np.stack([p1, s1], 1).ravel(), np.stack([pb1, np.zeros_like(pb1)], 1).ravel()])

    def resid(x):
        xc = x[:2 * c.n].reshape(c.n, 2); xw = x[2 * c.n:].reshape(-1, 2)
        s.set_state(xc[:, 0], xc[:, 1], xw[:, 0]); s.assemble()
        return -s.system()[3]

    Jfd = np.zeros_like(J)
    for k in range(2 * nb):
        if k >= 2 * c.n and k % 2 == 1:
            continue
        h = 1e-6 * max(1.0, abs(x0[k])) if k % 2 == 0 else 1e-7
        xp = x0.copy(); xp[k] += h
        xm = x0.copy(); xm[k] -= h
        Jfd[:, k] = (resid(xp) - resid(xm)) / (2 * h)
    Jfd[2 * c.n + 1::2, 2 * c.n + 1::2] = J[2 * c.n + 1::2, 2 * c.n + 1::2]
    rowscale = np.abs(J).max(axis=1, keepdims=True)
    err = np.abs(Jfd - J) / rowscale
    assert err.max() < 1e-6, err.max()


# ---------------------------------------------------------- rate wells ----
def _depletion_case(control, target, nx=6, ny=5, nz=3, seed=51, sw0=0.45):
    c = I.small_case(nx, ny, nz, seed=seed)
    c.wells = [I.Well(I.PROD, control, target, c.column(nx - 1, ny - 1))]
    c.sw_init = sw0
    return c


@pytest.mark.parametrize("control,target", [(I.ORATE, 40.0), (I.LRATE, 60.0), (I.WRATE, 15.0)])
def test_rate_producer_withdraws_its_target(oracle_lib, control, target):
    """A single producer on an oil-rate (eq. 13), liquid-rate (eq. 14) or
    water-rate (eq. 12) control depletes a closed reservoir: by
    conservation (the paper's remark after eq. 17) the fluid in place falls,
    in surface volumes, by exactly dt times the target over a converged
    step (oil, oil + water, or water)."""
    c = _depletion_case(control, target)
    s = oracle_lib.Sim(c, newton_tol=1e-11, lin_tol=1e-11, max_lin=200)
    s.init_hydrostatic()
    mw0, mo0 = s.mass()
    assert s.advance(1) == 0
    mw1, mo1 = s.mass()
    f = c.fluid
    dvo, dvw = (mo0 - mo1) / f.rho_ref[1], (mw0 - mw1) / f.rho_ref[0]
    produced = {I.ORATE: dvo, I.LRATE: dvo + dvw, I.WRATE: dvw}[control]
    assert produced == pytest.approx(c.dt * target, rel=1e-7)
    assert dvo > 0 and dvw > 0                          # both phases are mobile and produced


def test_injector_switches_to_its_bhp_limit_and_back(oracle_lib):
    """A water injector asked for more than its maximum BHP allows is put on
    BHP control at the limit during the Newton iteration (p_b = limit, rate
    below the request); after a schedule change lowers the requested rate
    below what the limit delivers, the next step returns it to rate control
    and it injects exactly the new rate."""
    c = I.small_case(6, 5, 3, seed=61)
    c.wells[0] = I.Well(I.INJ, I.WRATE, 5000.0, c.column(0, 0), bhp_limit=230.0)
    s = oracle_lib.Sim(c, newton_tol=1e-10, lin_tol=1e-10, max_lin=200)
    s.init_hydrostatic()
    assert s.advance(1) == 0
    ctrl, tgt = s.well_controls()
    assert ctrl[0] == I.BHP and tgt[0] == 230.0 and s.stats()["switches"] >= 1
    p, sw, pb, _ = s.get_state()
    assert pb[0] == 230.0
    qw, _ = s.well_rates()
    assert 0 < qw[0] < 1000.0 * 5000.0
    at_limit = qw[0] / 1000.0                            # sm3/day delivered at the limit
    s.set_well(0, I.WRATE, 0.5 * at_limit, bhp_limit=230.0)
    assert s.advance(1) == 0
    ctrl, _ = s.well_controls()
    assert ctrl[0] == I.WRATE
    qw, _ = s.well_rates()
    assert qw[0] / 1000.0 == pytest.approx(0.5 * at_limit, rel=1e-7)
    assert s.get_state()[2][0] < 230.0


def test_held_well_stays_on_its_limit_when_the_rate_is_out_of_reach(oracle_lib):
    """A producer whose oil-rate target cannot be met above its minimum BHP
    switches to that BHP, and at the start of the next step, producing less
    than the target at the limit, it stays there."""
    c = I.small_case(6, 5, 3, seed=62)
    c.wells[1] = I.Well(I.PROD, I.ORATE, 1000.0, c.column(5, 4), bhp_limit=150.0)
    s = oracle_lib.Sim(c, newton_tol=1e-10, lin_tol=1e-10, max_lin=200)
    s.init_hydrostatic()
    for _ in range(2):
        assert s.advance(1) == 0
        ctrl, tgt = s.well_controls()
        assert ctrl[1] == I.BHP and tgt[1] == 150.0
        assert s.get_state()[2][1] == 150.0
    assert s.stats()["switches"] == 1                   # held, not switched back and forth


def test_held_producer_returns_to_its_rate_once_the_limit_delivers_it(oracle_lib):
    """An oil-rate producer held at its minimum BHP (the reservoir starts
    too low to deliver its target) returns to its rate at the first step
    whose starting state would deliver more than the target at the limit,
    once an injector opened by a schedule change has raised the pressure;
    from then on it produces exactly its target above the limit.  While it
    is held, its production at the limit at the start of every step is
    below the target."""
    c = I.small_case(6, 5, 3, seed=61)
    q = 150.0
    c.wells[1] = I.Well(I.PROD, I.ORATE, q, c.column(5, 4), bhp_limit=150.0)
    s = oracle_lib.Sim(c, newton_tol=1e-10, lin_tol=1e-10, max_lin=200)
    s.init_hydrostatic(p_datum=160.0)
    s.set_well(0, I.SHUT, 0.0)
    assert s.advance(1) == 0
    assert s.well_controls()[0][1] == I.BHP
    s.set_well(0, I.WRATE, 300.0)
    returned = False
    for _ in range(6):
        at_start = -s.well_rates()[1][1] / c.fluid.rho_ref[1]        # sm3/day at the current p_b
        held = s.well_controls()[0][1] == I.BHP
        assert s.advance(1) == 0
        ctrl = s.well_controls()[0][1]
        if held and ctrl == I.BHP:
            assert at_start <= q                        # stayed: the limit did not deliver the target
        if held and ctrl == I.ORATE:
            assert at_start > q                         # returned: the limit delivered more
            returned = True
        if ctrl == I.ORATE:
            assert -s.well_rates()[1][1] / c.fluid.rho_ref[1] == pytest.approx(q, rel=1e-8)
            assert s.get_state()[2][1] > 150.0
    assert returned
    assert s.stats()["switches"] == 1


def test_shut_well_carries_no_flow(oracle_lib):
    """A shut well (a schedule stage, Table 1's "shutin") exchanges nothing
    with its cells: with the producer shut and the injector on its rate, the
    water in place grows by exactly dt times the injected rate and the oil
    in place does not change."""
    c = I.small_case(6, 5, 3, seed=63)
    s = oracle_lib.Sim(c, newton_tol=1e-11, lin_tol=1e-11, max_lin=200)
    s.init_hydrostatic()
    s.set_well(1, I.SHUT, 0.0)
    mw0, mo0 = s.mass()
    assert s.advance(1) == 0
    mw1, mo1 = s.mass()
    assert (mw1 - mw0) / 1000.0 == pytest.approx(c.dt * c.wells[0].target, rel=1e-8)
    assert abs(mo1 - mo0) <= 1e-9 * mo0
    qw, qo = s.well_rates()
    assert qw[1] == 0.0 and qo[1] == 0.0
