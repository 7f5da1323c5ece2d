"""Pins of the CPU oracle's model, discretisation and Newton loop against
closed forms, invariants and finite differences (no GPU needed).

Passages: eqs. (3)-(18) (model and discretisation), eq. (10) (wells),
Algorithm 1 (Newton), eq. (26) (forcing term) of arXiv 1701.06254.
"""
import copy
import math

import numpy as np
import pytest

from paper_1701_06254_gb300 import inputs as I

CDARCY = 9.869233e-16 * 1e5 / 1e-3 * 86400.0   # m3 cP / (day bar mD m)


def incompressible_fluid(g=0.0):
    return I.Fluid(c_f=(0.0, 0.0), c_r=0.0, c_mu=(0.0, 0.0), g=g)


def line_case(nx, dx, k, q_inj, p_bhp, sw0, inj_at_start=True, dt=1.0, phi=0.2, fluid=None, p0=None):
    n = nx
    kk = np.full(n, float(k))
    c = I.Case(f"line{nx}", nx, 1, 1, dx, 1.0, 1.0, 1000.0, kk, kk.copy(), kk.copy(),
               np.full(n, phi), fluid or incompressible_fluid(), [], dt=dt, n_steps=1,
               p_init=p_bhp + 10.0 if p0 is None else p0, sw_init=sw0)
    a, b = (0, nx - 1) if inj_at_start else (nx - 1, 0)
    c.wells = [I.Well(I.INJ, I.WRATE, q_inj, [a]), I.Well(I.PROD, I.BHP, p_bhp, [b])]
    return c


def test_linear_pressure_profile(oracle_lib):
    """Homogeneous, incompressible, single-phase water (s_w = 1 - S_or, so
    k_ro = 0) between a rate injector and a BHP producer: Darcy's law,
    eq. (1), gives a linear pressure with drop q mu_w dx / (C_D k A) per
    cell, exact for two-point fluxes; the well drops follow eq. (10)."""
    q, mu_w, k, dx, A = 10.0, 0.5, 100.0, 10.0, 100.0
    c = line_case(50, dx, k, q, 100.0, 0.8)
    c.dy = c.dz = 10.0
    s = oracle_lib.Sim(c, newton_tol=1e-13, lin_tol=1e-13, max_lin=200)
    s.init_hydrostatic()
    assert s.advance(1) == 0
    p, sw, pb, t = s.get_state()
    T = CDARCY * k * A / dx
    dp_expect = q * mu_w / T
    np.testing.assert_allclose(np.diff(p), -dp_expect, rtol=1e-10)
    np.testing.assert_allclose(sw, 0.8, atol=1e-12)
    wi = s.well_index()
    # producer: rho q = WI rho (k_rw / mu_w) (p - p_b), k_rw = 1
    np.testing.assert_allclose(p[-1] - pb[1], q * mu_w / wi[1], rtol=1e-10)
    # injector uses the total mobility k_rw/mu_w + k_ro/mu_o = 1/mu_w here
    np.testing.assert_allclose(pb[0] - p[0], q * mu_w / wi[0], rtol=1e-10)
    qw, qo = s.well_rates()
    np.testing.assert_allclose(qw, [1000.0 * q, -1000.0 * q], rtol=1e-10)


def test_pressure_dependent_viscosity(oracle_lib):
    """Eq. (7) with c_mu != 0, steady incompressible single-phase water: the
    same rate crosses every face, each face's mobility is taken from its
    upstream cell (eq. 18), so the drop across the face between cells i and
    i+1 is q mu_w(p_i) / T with mu_w(p) = mu_ref + c_mu (p - p_ref)."""
    q, dx, A, k, n = 10.0, 10.0, 100.0, 100.0, 40
    fl = incompressible_fluid()
    fl.c_mu = (5e-4, 0.0)
    c = line_case(n, dx, k, q, 100.0, 0.8, fluid=fl)
    c.dy = c.dz = 10.0
    s = oracle_lib.Sim(c, newton_tol=1e-13, lin_tol=1e-13, max_lin=200)
    s.init_hydrostatic()
    assert s.advance(1) == 0
    p = s.get_state()[0]
    mu = 0.5 + 5e-4 * (p[:-1] - fl.p_ref)
    T = CDARCY * k * A / dx
    np.testing.assert_allclose(-np.diff(p), q * mu / T, rtol=1e-9)
    assert np.ptp(mu) > 0.005                                     # the viscosity does vary


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_series_flow_through_heterogeneous_cells(oracle_lib, axis):
    """Steady incompressible single-phase water through cells of different
    permeability in series, along each grid axis: the same rate q crosses
    every face, and the pressure drop between neighbouring cell centres is
    the sum of the two half-cell resistances, q mu_w (L / (2 k_i) +
    L / (2 k_i+1)) / (C_D A), with k the permeability along the axis (the
    other two components differ, and must not enter); Darcy's law, eq. (1),
    on each half cell."""
    q, mu_w, L, A, n = 10.0, 0.5, 10.0, 100.0, 30
    rng = np.random.default_rng(8)
    k = np.exp(rng.normal(math.log(100.0), 1.0, n))
    other = np.exp(rng.normal(math.log(100.0), 1.0, n))
    dims = {"x": (n, 1, 1), "y": (1, n, 1), "z": (1, 1, n)}[axis]
    perm = {a: (k if a == axis else other.copy()) for a in "xyz"}
    c = I.Case(f"line_{axis}", *dims, L, L, L, 1000.0, perm["x"], perm["y"], perm["z"], np.full(n, 0.2),
               incompressible_fluid(), [], dt=1.0, n_steps=1, p_init=110.0, sw_init=0.8)
    c.wells = [I.Well(I.INJ, I.WRATE, q, [0]), I.Well(I.PROD, I.BHP, 100.0, [n - 1])]
    s = oracle_lib.Sim(c, newton_tol=1e-13, lin_tol=1e-13, max_lin=200)
    s.init_hydrostatic()
    assert s.advance(1) == 0
    p = s.get_state()[0]
    drop = q * mu_w * (L / (2.0 * k[:-1]) + L / (2.0 * k[1:])) / (CDARCY * A)
    np.testing.assert_allclose(-np.diff(p), drop, rtol=1e-9)


def test_peaceman_isotropic_square(oracle_lib):
    """Peaceman's equivalent radius for an isotropic square cell is
    0.14 sqrt(dx^2 + dy^2) = 0.198 dx (the classical result)."""
    c = I.small_case(3, 3, 2, seed=1)
    k = 50.0
    c.kx[:] = k; c.ky[:] = k; c.kz[:] = 0.1 * k
    s = oracle_lib.Sim(c)
    wi = s.well_index()
    ro = 0.14 * math.sqrt(2.0) * c.dx
    expect = 2 * math.pi * CDARCY * k * c.dz / math.log(ro / 0.1)
    np.testing.assert_allclose(wi, expect, rtol=1e-13)


def test_peaceman_anisotropic_invariances(oracle_lib):
    """Peaceman's anisotropic well index does not depend on how the grid is
    turned: exchanging kx with ky together with dx with dy leaves it
    unchanged; and for kx = ky it reduces to the isotropic formula with
    0.14 sqrt(dx^2 + dy^2) on a rectangular cell."""
    def wi(kx, ky, dx, dy):
        c = I.small_case(3, 3, 2, seed=1)
        c.kx[:] = kx; c.ky[:] = ky; c.kz[:] = 0.1 * min(kx, ky)
        c.dx, c.dy = dx, dy
        return oracle_lib.Sim(c).well_index()
    np.testing.assert_allclose(wi(100.0, 900.0, 10.0, 25.0), wi(900.0, 100.0, 25.0, 10.0), rtol=1e-13)
    assert not np.allclose(wi(100.0, 900.0, 10.0, 25.0), wi(900.0, 100.0, 10.0, 25.0), rtol=1e-3)
    k, dx, dy = 70.0, 10.0, 25.0
    ro = 0.14 * math.sqrt(dx * dx + dy * dy)
    c = I.small_case(3, 3, 2, seed=1)
    np.testing.assert_allclose(wi(k, k, dx, dy), 2 * math.pi * CDARCY * k * c.dz / math.log(ro / 0.1), rtol=1e-13)


def _closed_form_accumulation(case, p, sw):
    """phi rho_a s_a from eqs. (4), (6), (8) (oil, water), per cell."""
    f = case.fluid
    phi = case.phi * (1.0 + f.c_r * (p - f.p_ref))
    rw = f.rho_ref[0] * (1.0 + f.c_f[0] * (p - f.p_ref))
    ro = f.rho_ref[1] * (1.0 + f.c_f[1] * (p - f.p_ref))
    return phi * ro * (1.0 - sw), phi * rw * sw


@pytest.mark.parametrize("seed", [3, 4])
def test_mass_balance_identity(oracle_lib, seed):
    """Face fluxes cancel pairwise (the paper's conservation remark after
    eq. 17), so for ANY state the sum of the residuals of eq. (17) over all
    cells equals the total accumulation change minus the well rates."""
    c = I.small_case(5, 4, 3, seed=seed)
    s = oracle_lib.Sim(c)
    p0, s0, pb0 = I.random_state(c, seed + 100)
    p1, s1, pb1 = I.random_state(c, seed + 200)
    s.set_state(p0, s0, pb0); s.store_old()
    s.set_state(p1, s1, pb1); s.set_dt(2.0)
    s.assemble()
    rp, ci, val, b, key = s.system()
    R = -b[:2 * c.n].reshape(c.n, 2)
    ao0, aw0 = _closed_form_accumulation(c, p0, s0)
    ao1, aw1 = _closed_form_accumulation(c, p1, s1)
    V = c.dx * c.dy * c.dz
    qw, qo = s.well_rates()
    exp_o = (V / 2.0) * (ao1 - ao0).sum() - qo.sum()
    exp_w = (V / 2.0) * (aw1 - aw0).sum() - qw.sum()
    scale_o = (V / 2.0) * np.abs(ao1 - ao0).sum()
    scale_w = (V / 2.0) * np.abs(aw1 - aw0).sum()
    assert abs(R[:, 0].sum() - exp_o) <= 1e-9 * scale_o
    assert abs(R[:, 1].sum() - exp_w) <= 1e-9 * scale_w
    # and the residual is not trivially balanced: individual rows are large
    assert np.abs(R[:, 0]).max() > 1e-3 * scale_o / c.n


def _dense_J(rp, ci, val, nb):
    J = np.zeros((2 * nb, 2 * nb))
    for i in range(nb):
        for q in range(rp[i], rp[i + 1]):
            j = ci[q]
            J[2 * i:2 * i + 2, 2 * j:2 * j + 2] = val[4 * q:4 * q + 4].reshape(2, 2)
    return J


@pytest.mark.parametrize("seed,crossflow", [(5, False), (6, False), (7, True)])
def test_jacobian_matches_finite_differences(oracle_lib, seed, crossflow):
    """Analytic 2x2-block Jacobian vs central differences of the residual
    (eq. 17 with upstreaming eq. 18 and wells eq. 10) at a random state
    away from relative-permeability and upstream kinks; with crossflow the
    injector's wellbore pressure is below every cell's, so its perforations
    produce from the cells (upstream = cell)."""
    c = I.small_case(3, 3, 2, seed=seed)
    s = oracle_lib.Sim(c)
    p0, s0, pb0 = I.random_state(c, seed + 10)
    p1, s1, pb1 = I.random_state(c, seed + 20)
    if crossflow:
        pb1 = np.array([100.0 if w.kind == I.INJ else pb for w, pb in zip(c.wells, pb1)])
    s.set_state(p0, s0, pb0); s.store_old()
    s.set_dt(1.5)
    s.set_state(p1, s1, pb1); s.assemble()
    rp, ci, val, b, key = s.system()
    nb = c.n + len(c.wells)
    J = _dense_J(rp, ci, val, nb)
    x0 = np.concatenate([np.stack([p1, s1], 1).ravel(), np.stack([pb1, np.zeros_like(pb1)], 1).ravel()])

    def resid(x):
        xc = x[:2 * c.n].reshape(c.n, 2); xw = x[2 * c.n:].reshape(-1, 2)
        s.set_state(xc[:, 0], xc[:, 1], xw[:, 0]); s.assemble()
        return -s.system()[3]

    Jfd = np.zeros_like(J)
    for k in range(2 * nb):
        if k >= 2 * c.n and k % 2 == 1:
            continue                      # padded dummy unknown of a well row
        h = 1e-6 * max(1.0, abs(x0[k])) if k % 2 == 0 else 1e-7
        xp = x0.copy(); xp[k] += h
        xm = x0.copy(); xm[k] -= h
        Jfd[:, k] = (resid(xp) - resid(xm)) / (2 * h)
    Jfd[2 * c.n + 1::2, 2 * c.n + 1::2] = J[2 * c.n + 1::2, 2 * c.n + 1::2]
    rowscale = np.abs(J).max(axis=1, keepdims=True)
    err = np.abs(Jfd - J) / rowscale
    assert err.max() < 1e-6, err.max()


def _cell_residuals(oracle_lib, case, p, sw, pb):
    s = oracle_lib.Sim(case)
    s.set_state(p, sw, pb); s.store_old(); s.set_dt(1.0)
    s.set_state(p, sw, pb); s.assemble()
    return -s.system()[3][:2 * case.n].reshape(case.n, 2)     # rows: (oil, water) per cell


def test_well_flow_directions(oracle_lib):
    """Eq. (10) with the flow directions of reading R7: a producer whose
    wellbore pressure is above its cells' takes nothing from them and puts
    nothing in; an injector whose wellbore pressure is below its cells'
    (crossflow) draws from them with each phase's own mobility, so a cell at
    connate water saturation gives up oil but no water."""
    c = I.small_case(4, 3, 3, seed=31)
    bare = copy.deepcopy(c)
    bare.wells = []
    rng = np.random.default_rng(32)
    p = 200.0 + rng.uniform(0.0, 5.0, c.n)
    inj, prod = c.wells
    sw = np.full(c.n, 0.5)
    R = _cell_residuals(oracle_lib, c, p, sw, np.array([p.max() + 50.0, p.max() + 50.0]))
    R0 = _cell_residuals(oracle_lib, bare, p, sw, np.zeros(0))
    cells = np.array(prod.perf_cells)
    np.testing.assert_array_equal(R[cells], R0[cells])           # the producer does nothing
    assert np.all(R[np.array(inj.perf_cells), 1] != R0[np.array(inj.perf_cells), 1])   # the injector does inject
    sw = np.full(c.n, c.fluid.swc)
    R = _cell_residuals(oracle_lib, c, p, sw, np.array([p.min() - 50.0, p.min() - 50.0]))
    R0 = _cell_residuals(oracle_lib, bare, p, sw, np.zeros(0))
    cells = np.array(inj.perf_cells)
    np.testing.assert_array_equal(R[cells, 1], R0[cells, 1])     # no water leaves at connate saturation
    assert np.all(R[cells, 0] != R0[cells, 0])                   # oil does


def test_hydrostatic_initial_state_is_at_rest(oracle_lib):
    """The initial state gives every cell the datum oil potential (eq. 5)
    with s_w = S_wc (no water mobility): without wells nothing moves."""
    c = I.small_case(4, 4, 5, seed=9)
    c.wells = []
    s = oracle_lib.Sim(c, newton_tol=1e-12, lin_tol=1e-12)
    s.init_hydrostatic()
    p0, s0, _, _ = s.get_state()
    assert np.all(np.diff(p0.reshape(5, 16)[:, 0]) > 0)       # pressure rises with depth
    # eq. (5) with eq. (6): p_k - rho_o(p_k) g z_k = p_datum - rho_o(p_datum) g z_top at every
    # cell centre z_k = top + (k + 1/2) dz (depth positive downwards, bar)
    f = c.fluid
    rho = lambda p: f.rho_ref[1] * (1.0 + f.c_f[1] * (p - f.p_ref))
    z = c.top + (np.arange(5) + 0.5) * c.dz
    pk = p0.reshape(5, 16)[:, 0]
    np.testing.assert_allclose(pk - rho(pk) * f.g * z * 1e-5,
                               c.p_init - rho(c.p_init) * f.g * c.top * 1e-5, rtol=1e-13)
    assert s.advance(2) == 0
    p1, s1, _, _ = s.get_state()
    np.testing.assert_allclose(p1, p0, rtol=1e-12)
    np.testing.assert_allclose(s1, s0, atol=1e-14)


def test_saturation_chop_bounds_each_update(oracle_lib):
    """With sat_chop > 0 each Newton iteration changes every cell's s_w by
    at most sat_chop (the chop acts on the update before it is applied),
    and on a first iteration far from equilibrium it does bind."""
    c = I.small_case(6, 5, 3, seed=21, dt=30.0)
    for chop in (0.02, 0.05):
        s = oracle_lib.Sim(c, max_newton=1, sat_chop=chop)
        s.init_hydrostatic(sw0=0.2)
        s.store_old()
        s.set_dt(30.0)
        p0, s0, _, _ = s.get_state()
        rc, its = s.newton()
        p1, s1, _, _ = s.get_state()
        assert rc == 1 and its == 1                      # one update applied, not yet converged
        ds = np.abs(s1 - s0)
        assert ds.max() <= chop * (1 + 1e-12)
        assert np.isclose(ds.max(), chop, rtol=1e-12)    # the chop was active
        assert np.abs(p1 - p0).max() > 0


def test_time_step_cuts_cover_the_interval(oracle_lib):
    """A step whose Newton iteration fails is retried with half the step
    length until it converges, and the rest of the interval is covered with
    the cut length: the clock advances by exactly dt, in more than one
    sub-step, and the state is a converged one."""
    c = I.small_case(6, 5, 3, seed=21, dt=30.0)
    s = oracle_lib.Sim(c, max_newton=3)
    s.init_hydrostatic(sw0=0.2)
    assert s.advance(1) == 0
    st = s.stats()
    assert st["cuts"] >= 1 and st["steps"] >= 2, st
    assert st["t"] == 30.0
    assert st["norm"] <= c.newton_tol


def test_inexact_newton_solves_loosely(oracle_lib):
    """Algorithm 1 with the forcing terms of eq. (26): each linear solve
    stops at eta_l >= 0.01 instead of the fixed 1e-8 of standard Newton, so
    over the same steps the inexact method needs far fewer FGMRES
    iterations, while both converge."""
    c = I.case0()
    counts = {}
    for newton in (0, 1):
        s = oracle_lib.Sim(c, newton=newton, lin_tol=1e-8)
        s.init_hydrostatic()
        assert s.advance(3) == 0
        counts[newton] = s.stats()["lin"]
    assert counts[1] < 0.6 * counts[0], counts


def test_forcing_term_choice_two(oracle_lib):
    """Eq. (26), second choice, with the clamp to [0.01, 0.1]; eta_0 = 0.1."""
    f = oracle_lib.forcing
    assert f(0, 5.0, 1.0, 2.0) == 0.1
    assert f(3, 1.0, 0.95, 2.0) == pytest.approx(0.025, rel=1e-15)     # inside the band
    assert f(3, 1.0, 0.99999, 10.0) == 0.01                              # clamped low
    assert f(3, 5.0, 0.0, 2.0) == 0.1                                    # clamped high
    assert f(3, 1.0, 2.0, 3.0) == 0.01                                   # negative -> 0.01


# ---------------------------------------------------------------------------
# Buckley-Leverett: 1D, incompressible, no gravity, no capillary pressure.
# Corey n = 2, S_wc = S_or = 0.2, M = mu_o / mu_w = 4.  The Welge tangent
# gives s_hat_f = 1/sqrt(5): S_f = 0.2 + 0.6/sqrt(5) = 0.468328, and the
# front travels at q/(phi A) * df_w/dS_w(S_f) = q/(phi A) * 2.696723.
# ---------------------------------------------------------------------------
def _fw(s, muw=0.5, muo=2.0, nw=2.0, no=2.0):
    """Fractional flow of water, Corey relative permeabilities, S_wc = S_or = 0.2."""
    sh = np.clip((s - 0.2) / 0.6, 0, 1)
    lw, lo = sh ** nw / muw, (1 - sh) ** no / muo
    return lw / (lw + lo)


def _dfw(s, muw=0.5, muo=2.0, nw=2.0, no=2.0):
    sh = np.clip((s - 0.2) / 0.6, 0, 1)
    lw, lo = sh ** nw / muw, (1 - sh) ** no / muo
    dlw, dlo = nw * sh ** (nw - 1) / muw / 0.6, -no * (1 - sh) ** (no - 1) / muo / 0.6
    return (dlw * (lw + lo) - lw * (dlw + dlo)) / (lw + lo) ** 2


def _welge_front(nw, no):
    """Front saturation of the Buckley-Leverett solution: the tangent from
    (S_wc, 0) to f_w, f_w'(S_f) (S_f - S_wc) = f_w(S_f), found by bisection
    (the left side exceeds the right below S_f)."""
    lo, hi = 0.2 + 1e-9, 0.8 - 1e-9
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _dfw(mid, nw=nw, no=no) * (mid - 0.2) > _fw(mid, nw=nw, no=no):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_welge_constants():
    sf = 0.2 + 0.6 / math.sqrt(5.0)
    assert sf == pytest.approx(0.468328, abs=1e-6)
    assert _fw(sf) == pytest.approx(0.723607, abs=1e-6)
    # tangent from (S_wc, 0): f_w(S_f) / (S_f - S_wc) = f_w'(S_f)
    assert _dfw(sf) == pytest.approx(_fw(sf) / (sf - 0.2), rel=1e-12)
    assert _dfw(sf) == pytest.approx(2.696723, abs=1e-6)


def _bl_analytic(x, t, q, phi, A):
    sf = 0.2 + 0.6 / math.sqrt(5.0)
    v = x * phi * A / (q * t)
    out = np.full_like(x, 0.2)
    for i, vi in enumerate(v):
        if vi < _dfw(sf):
            lo, hi = sf, 0.8 - 1e-12
            if vi <= _dfw(hi):
                out[i] = hi
                continue
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if _dfw(mid) > vi:
                    lo = mid
                else:
                    hi = mid
            out[i] = 0.5 * (lo + hi)
    return out


def _bl_run(oracle_lib, nx, nsteps, t_end):
    L, q, phi = 100.0, 0.02, 0.2
    fl = incompressible_fluid()
    c = line_case(nx, L / nx, 100.0, q, 100.0, 0.2, dt=t_end / nsteps, phi=phi, fluid=fl)
    s = oracle_lib.Sim(c, newton_tol=1e-9, lin_tol=1e-10, max_lin=200)
    s.init_hydrostatic()
    assert s.advance(nsteps) == 0
    p, sw, pb, t = s.get_state()
    x = (np.arange(nx) + 0.5) * (L / nx)
    return x, sw, _bl_analytic(x, t, q, phi, 1.0)


def test_buckley_leverett_front(oracle_lib):
    """The saturation front sits at x_f = q t / (phi A) * 2.696723; the
    first-order implicit upwind scheme smears it ahead of x_f by a distance
    that shrinks under refinement (3.0 m at dx = 1 m, 1.8 m at 0.5 m)."""
    t_end = 150.0
    xf = 0.02 * t_end / 0.2 * 2.696723                        # 40.45 m
    mid = 0.5 * (0.2 + 0.2 + 0.6 / math.sqrt(5.0))
    gaps = []
    for nx in (100, 200):
        x, sw, ex = _bl_run(oracle_lib, nx, nx * 3 // 2, t_end)
        gaps.append(x[np.nonzero(sw < mid)[0][0]] - xf)
        # saturation never exceeds 1 - S_or and the injected water is all in place
        assert sw.max() <= 0.8 + 1e-9
        np.testing.assert_allclose(((sw - 0.2) * 0.2 * (100.0 / nx)).sum(), 0.02 * t_end, rtol=1e-6)
    assert 0.0 < gaps[1] < gaps[0] <= 3.5, gaps
    assert gaps[1] <= 2.5, gaps


def test_buckley_leverett_front_unequal_exponents(oracle_lib):
    """Corey exponents n_w = 3, n_o = 2: the front travels at
    f_w'(S_f) = 2.345 pore volumes per unit q t / (phi A) (Welge tangent),
    so at t = 150 d it sits at 35.2 m; upwinding smears the computed front
    ahead of it by at most a few cells, and the water injected is all in
    place."""
    sf = _welge_front(3.0, 2.0)
    speed = _fw(sf, nw=3.0, no=2.0) / (sf - 0.2)
    assert speed == pytest.approx(2.345018, abs=1e-5)
    nx, t_end, L, q, phi = 200, 150.0, 100.0, 0.02, 0.2
    fl = incompressible_fluid()
    fl.nw = 3.0
    c = line_case(nx, L / nx, 100.0, q, 100.0, 0.2, dt=t_end / 300, phi=phi, fluid=fl)
    s = oracle_lib.Sim(c, newton_tol=1e-9, lin_tol=1e-10, max_lin=200)
    s.init_hydrostatic()
    assert s.advance(300) == 0
    sw = s.get_state()[1]
    x = (np.arange(nx) + 0.5) * (L / nx)
    xf = q * t_end / phi * speed
    gap = x[np.nonzero(sw < 0.5 * (0.2 + sf))[0][0]] - xf
    assert 0.0 < gap <= 2.5, gap
    np.testing.assert_allclose(((sw - 0.2) * phi * (L / nx)).sum(), q * t_end, rtol=1e-6)


def test_buckley_leverett_converges_under_refinement(oracle_lib):
    errs = []
    for nx in (50, 100, 200):
        x, sw, ex = _bl_run(oracle_lib, nx, nx, 150.0)
        errs.append(np.abs(sw - ex).mean())
    assert errs[0] > errs[1] > errs[2], errs


# ---------------------------------------------------------------------------
# The Newton convergence measure (Algorithm 1 tests ||b|| >= epsilon before
# each solve; reading R13 fixes the norm): the largest |R| dt / (rho_ref V
# phi) over the cells' two equations -- the change in saturation that the
# residual mass stands for -- and the largest dimensionless well residual.

def _one_cell_case(dx=30.0, dy=40.0, dz=7.0, phi=0.23, k=50.0, fluid=None, wells=()):
    kk = np.full(1, k)
    c = I.Case("one_cell", 1, 1, 1, dx, dy, dz, 1000.0, kk, kk.copy(), kk.copy(), np.full(1, phi),
               fluid or incompressible_fluid(), list(wells), dt=1.0, n_steps=1, p_init=200.0, sw_init=0.3)
    return c


@pytest.mark.parametrize("c_w,c_o,expect", [(0.0, 0.0, 0.05), (1e-3, 0.0, 0.05 * 1.1), (0.0, 2e-3, 0.05 * 1.2)])
def test_newton_measure_closed_cell(oracle_lib, c_w, c_o, expect):
    """One closed cell without wells, rigid rock: s_w moves from 0.30 to
    0.35 over a step of 2.5 days.  Each equation's residual is then only
    its accumulation term, V/dt phi rho_a (s_a^{n+1} - s_a^n) (eq. 17), so
    the measure is |Delta s_w| rho_a / rho_a,ref = 0.05 for an
    incompressible phase and 0.05 (1 + c_a (p - p_ref)) for a compressible
    one at p = p_ref + 100 bar (eq. 6): the larger of the two rows."""
    fl = incompressible_fluid()
    fl.c_f = (c_w, c_o)
    fl.rho_ref = (1000.0, 800.0)
    c = _one_cell_case(fluid=fl)
    s = oracle_lib.Sim(c)
    p = np.array([fl.p_ref + 100.0])
    s.set_state(p, np.array([0.30]), np.zeros(0)); s.store_old()
    s.set_state(p, np.array([0.35]), np.zeros(0)); s.set_dt(2.5)
    s.assemble()
    assert s.residual_norm() == pytest.approx(expect, rel=1e-12)


def test_newton_measure_bhp_well_row(oracle_lib):
    """A BHP producer whose wellbore pressure (210 bar) is above its cell's
    (200 bar) takes nothing from it (reading R7), and the state equals the
    old time level, so the cell rows vanish and the measure is the well row
    of eq. (11) scaled by its target: |p_b - target| / target = 60/150."""
    c = _one_cell_case(wells=[I.Well(I.PROD, I.BHP, 150.0, [0])])
    s = oracle_lib.Sim(c)
    p, sw = np.array([200.0]), np.array([0.3])
    s.set_state(p, sw, np.array([210.0])); s.store_old(); s.set_dt(1.0)
    s.assemble()
    assert s.residual_norm() == pytest.approx(0.4, rel=1e-12)


def test_newton_measure_water_rate_row(oracle_lib):
    """A water-rate injector (eq. 12) 1 bar above its cell at connate
    saturation (k_rw = 0, k_ro = 1): water enters with the total mobility
    1/mu_o (reading R7), q_w = WI rho_w (p_b - p) / mu_o with Peaceman's
    index for a square isotropic cell, 2 pi C_D k dz / ln(0.14 sqrt(2) dx /
    r_w).  The cell is large, so its own scaled residual is negligible, and
    the measure is the well row |q_w - rho_w q| / (rho_w q)."""
    k, dx, dz, q = 1.0, 1000.0, 100.0, 0.1
    c = _one_cell_case(dx=dx, dy=dx, dz=dz, k=k, wells=[I.Well(I.INJ, I.WRATE, q, [0])])
    s = oracle_lib.Sim(c)
    fl = c.fluid
    p, sw = np.array([200.0]), np.array([fl.swc])
    s.set_state(p, sw, np.array([201.0])); s.store_old(); s.set_dt(1.0)
    s.assemble()
    wi = 2 * math.pi * CDARCY * k * dz / math.log(0.14 * math.sqrt(2.0) * dx / 0.1)
    qw = wi * fl.rho_ref[0] * 1.0 / fl.mu_ref[1]
    expect = abs(qw - fl.rho_ref[0] * q) / (fl.rho_ref[0] * q)
    assert expect > 1.0                                 # the well row dominates ...
    cell = qw * 1.0 / (fl.rho_ref[0] * dx * dx * dz * 0.23)
    assert cell < 1e-6                                  # ... the cell row does not
    assert s.residual_norm() == pytest.approx(expect, rel=1e-12)


def test_openmp_build_gives_identical_results(oracle_lib):
    """The OpenMP build of the oracle (used only to time it on all host
    cores) parallelises loops that write disjoint outputs and sum nothing
    across iterations, so two time steps give bit-identical states."""
    c = I.small_case(9, 8, 3, seed=17)
    out = []
    for omp in (False, True):
        s = oracle_lib.Sim(c, omp=omp)
        s.init_hydrostatic()
        assert s.advance(2) == 0
        out.append(s.get_state())
    for a, b in zip(out[0][:3], out[1][:3]):
        np.testing.assert_array_equal(a, b)
