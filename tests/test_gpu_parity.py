"""GPU (sm_103a) path vs the CPU oracle, through the C ABI.

Integer work (sparsity patterns, reordering permutations, C/F splits, AMG
patterns, level sets) must match bit for bit when both sides get the same
FP64 input; the ABF-decoupled matrix and the FP64 AMG setup also match bit
for bit (both evaluate the same formulas with round-to-nearest operations in
the same order).  Floating-point results are compared with the tolerances
stated in each test: 1e-12 relative for assembly (different summation
order), 1e-10 for FP64 operator applications, and per-cell |dp|/p <= 1e-6,
|ds| <= 1e-6 with Newton counts within +-1 for whole runs.
"""
import numpy as np
import pytest

import oracle
import paper_1701_06254_gb300 as R
from paper_1701_06254_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _states(case, seed):
    p0, s0, pb0 = I.random_state(case, seed)
    p1, s1, pb1 = I.random_state(case, seed + 1)
    return (p0, s0, pb0), (p1, s1, pb1)


def _pair(case, seed, dt=1.5, **opts):
    """Oracle and GPU simulators on the same random (old, new) states, assembled."""
    (p0, s0, pb0), (p1, s1, pb1) = _states(case, seed)
    o = oracle.Sim(case, **opts)
    o.set_state(p0, s0, pb0); o.store_old(); o.set_dt(dt)
    o.set_state(p1, s1, pb1); o.assemble()
    g = R.Sim(case, **opts)
    g.set_state(p0, s0, pb0); g.begin_step(dt)
    g.set_state(p1, s1, pb1)
    nrm = g.assemble()
    return o, g, nrm


def _rowscale(val, rp, nb):
    a = np.abs(val.reshape(-1, 4)).max(axis=1)
    return np.maximum.reduceat(a, rp[:-1])


CASES = [
    lambda: I.small_case(6, 5, 3, seed=21),
    lambda: I.small_case(11, 7, 4, seed=22),            # ragged 8x8 tiles
    lambda: I.small_case(13, 1, 1, seed=23),            # 1D
    lambda: I.small_case(3, 3, 9, seed=24, gravity=True),
]


@pytest.mark.parametrize("mk", CASES)
def test_assembly_matches_oracle(mk):
    c = mk()
    o, g, nrm = _pair(c, 100)
    rp, ci, val, b, key = o.system()
    grp = g.ls.export(R.X_ROWPTR, 0, np.int32)
    gci = g.ls.export(R.X_COLS, 0, np.int32)
    np.testing.assert_array_equal(grp, rp)
    np.testing.assert_array_equal(gci, ci)
    gval = g.ls.export(R.X_VALS)
    gb = g.ls.export(R.X_RHS)
    nb = len(rp) - 1
    sc = np.repeat(_rowscale(val, rp, nb), np.diff(rp))
    err = np.abs(gval - val).reshape(-1, 4).max(axis=1) / sc
    assert err.max() < 1e-12, err.max()
    bs = np.abs(b).reshape(-1, 2).max(axis=1).max()
    assert np.abs(gb - b).max() <= 1e-12 * bs
    np.testing.assert_array_equal(g.ls.export(R.X_KEY), key)          # eq. (5), same IEEE order
    np.testing.assert_allclose(nrm, o.residual_norm(), rtol=1e-12)


def _shared_system(case, seed, **opts):
    """The oracle's assembled Jacobian handed to both linear solvers."""
    o, _, _ = _pair(case, seed, **opts)
    rp, ci, val, b, key = o.system()
    wc0 = [w.perf_cells[0] for w in case.wells]
    gl = R.LinearSystem(case.nx, case.ny, case.nz, len(case.wells), rp, ci, wc0, **opts)
    gl.set(val, b, key)
    return o, gl, (rp, ci, val, b, key)


SYS = [
    (lambda: I.small_case(6, 5, 3, seed=31), dict(tile_x=2, tile_y=2, amg_coarse_max=8)),
    (lambda: I.small_case(11, 7, 4, seed=32), dict(tile_x=3, tile_y=4, amg_coarse_max=16)),
    (lambda: I.case0(), dict()),
    (lambda: I.case0(), dict(amg_coarse_max=40, tile_x=5, tile_y=3)),
]


@pytest.mark.parametrize("mk,opts", SYS)
def test_setup_integer_work_is_bit_exact(mk, opts):
    c = mk()
    o, gl, (rp, ci, val, b, key) = _shared_system(c, 200, **opts)
    o.ls.setup()
    gl.setup()
    _, _, dval, db, _ = o.ls.get()
    # ABF decoupling: same bits
    np.testing.assert_array_equal(gl.export(R.X_VALS), dval)
    np.testing.assert_array_equal(gl.export(R.X_RHS), db)
    # local potential reordering per subdomain (eqs. 30-32)
    assert gl.ras_count() == o.ls.nsub
    for s in range(o.ls.nsub):
        np.testing.assert_array_equal(gl.ras_ext(s), o.ls.sub(s)["ext"])
    # AMG hierarchy: every level, bit for bit
    oa = o.ls.amg()
    assert gl.amg_nlev() == oa.nlev
    for l in range(oa.nlev):
        Lo, Lg = oa.level(l), gl.amg_level(l)
        np.testing.assert_array_equal(Lg["rp"], Lo["rp"])
        np.testing.assert_array_equal(Lg["ci"], Lo["ci"])
        np.testing.assert_array_equal(Lg["v"], Lo["v"])
        if l < oa.nlev - 1:
            np.testing.assert_array_equal(Lg["cf"], Lo["cf"])
            assert Lg["rounds"] == Lo["rounds"]
            np.testing.assert_array_equal(Lg["prp"], Lo["prp"])
            np.testing.assert_array_equal(Lg["pci"], Lo["pci"])
            np.testing.assert_array_equal(Lg["pv"], Lo["pv"])


@pytest.mark.parametrize("prec", [R.PREC_FP64, R.PREC_MIXED, R.PREC_MIXED_BF16], ids=["fp64", "mixed", "bf16"])
def test_qi_decoupling_is_bit_exact(prec):
    """Quasi-IMPES decoupling (eq. 29): the decoupled matrix and right-hand
    side equal the oracle's bit for bit in every precision (the mixed ones
    decouple in the same pass that writes the FP32 planes)."""
    c = I.small_case(11, 7, 4, seed=32)
    o, _, _ = _pair(c, 200, decoupling=R.DEC_QI)
    rp, ci, val, b, key = o.system()
    wc0 = [w.perf_cells[0] for w in c.wells]
    gl = R.LinearSystem(c.nx, c.ny, c.nz, len(c.wells), rp, ci, wc0, decoupling=R.DEC_QI, precision=prec,
                        tile_x=3, tile_y=4)
    gl.set(val, b, key)
    o.ls.setup()
    gl.setup()
    _, _, dval, db, _ = o.ls.get()
    np.testing.assert_array_equal(gl.export(R.X_VALS), dval)
    np.testing.assert_array_equal(gl.export(R.X_RHS), db)


def _levels_brute(rp, ci):
    m = len(rp) - 1
    L = np.zeros(m, int); U = np.zeros(m, int)
    for i in range(m):
        cols = ci[rp[i]:rp[i + 1]]
        lo = [L[c] for c in cols if c < i]
        L[i] = 1 + max(lo) if lo else 0
    for i in range(m - 1, -1, -1):
        cols = ci[rp[i]:rp[i + 1]]
        hi = [U[c] for c in cols if c > i]
        U[i] = 1 + max(hi) if hi else 0
    return L, U


def test_ilu_level_sets_match_topological_levels():
    c = I.small_case(9, 6, 5, seed=41)
    o, gl, _ = _shared_system(c, 300, tile_x=4, tile_y=3)
    o.ls.setup(); gl.setup()
    for s in range(o.ls.nsub):
        d = o.ls.sub(s)
        L, U = _levels_brute(d["rp"], d["ci"])
        nL, nU, gL, gU = gl.ras_levels(s)
        np.testing.assert_array_equal(gL, L)
        np.testing.assert_array_equal(gU, U)
        assert nL == L.max() + 1 and nU == U.max() + 1


@pytest.mark.parametrize("mk,opts", SYS[:3])
def test_operators_match_oracle_fp64(mk, opts):
    c = mk()
    o, gl, _ = _shared_system(c, 400, **opts)
    o.ls.setup(); gl.setup()
    rng = np.random.default_rng(5)
    nb = c.n + len(c.wells)
    x = rng.standard_normal(2 * nb)
    for op, fo in ((R.OP_SPMV, o.ls.mv), (R.OP_RAS, o.ls.ras), (R.OP_CPR, o.ls.cpr)):
        yg, yo = gl.apply(op, x), fo(x)
        assert np.abs(yg - yo).max() <= 1e-10 * np.abs(yo).max(), op
    xp = rng.standard_normal(c.n)
    yg, yo = gl.apply(R.OP_VCYCLE, xp), o.ls.amg().apply(xp)
    assert np.abs(yg - yo).max() <= 1e-10 * np.abs(yo).max()


@pytest.mark.parametrize("mk,opts", SYS)
def test_fgmres_matches_oracle(mk, opts):
    c = mk()
    o, gl, _ = _shared_system(c, 500, **opts)
    o.ls.setup(); gl.setup()
    rco, yo, itso, relo = o.ls.solve(1e-10)
    yg, itsg, relg = gl.solve(1e-10)
    assert rco == 0 and relg <= 1e-10
    assert abs(itsg - itso) <= 1
    assert np.abs(yg - yo).max() <= 1e-7 * np.abs(yo).max()


@pytest.mark.parametrize("mk,opts", SYS)
def test_mixed_fgmres_reaches_tight_tolerance(mk, opts):
    """The mixed-precision solver keeps its Krylov basis in double-float
    (hi + lo FP32, about 48 significant bits): far below the benchmark's
    relres 1e-6 it still converges, to a true residual of 1e-10, to the FP64
    oracle's solution, in at most 25% more iterations than the oracle's FP64
    solver (the FP32 preconditioner is weaker)."""
    c = mk()
    o, gl, _ = _shared_system(c, 500, precision=R.PREC_MIXED_BF16, **opts)
    o.ls.setup(); gl.setup()
    rco, yo, itso, relo = o.ls.solve(1e-10)
    yg, itsg, relg = gl.solve(1e-10)
    assert rco == 0 and relg <= 1e-10, relg
    assert itsg <= 1.25 * itso + 2, (itsg, itso)
    assert np.abs(yg - yo).max() <= 1e-7 * np.abs(yo).max()


def test_mixed_precision_operators_track_fp64():
    """FP32 RAS / AMG / CPR stay within single-precision distance of the
    FP64 oracle; the integer setup work is unchanged (done in FP64)."""
    c = I.case0()
    o, gl, _ = _shared_system(c, 600, precision=R.PREC_MIXED)
    o.ls.setup(); gl.setup()
    oa = o.ls.amg()
    for l in range(oa.nlev - 1):
        np.testing.assert_array_equal(gl.amg_level(l)["cf"], oa.level(l)["cf"])
    x = np.random.default_rng(6).standard_normal(2 * (c.n + 2))
    for op, fo in ((R.OP_RAS, o.ls.ras), (R.OP_CPR, o.ls.cpr)):
        yg, yo = gl.apply(op, x), fo(x)
        assert np.abs(yg - yo).max() <= 1e-3 * np.abs(yo).max(), op
    yg, itsg, relg = gl.solve(1e-8)
    assert relg <= 1e-8
    gb = R.LinearSystem(c.nx, c.ny, c.nz, 2, *_shared_system(c, 600)[2][:2], [w.perf_cells[0] for w in c.wells],
                        precision=R.PREC_MIXED_BF16)
    gb.set(*_shared_system(c, 600)[2][2:])
    gb.setup()
    yb = gb.apply(R.OP_RAS, x)
    yo = o.ls.ras(x)
    assert np.abs(yb - yo).max() <= 3e-2 * np.abs(yo).max()
    yb, itsb, relb = gb.solve(1e-8)
    assert relb <= 1e-8


def _run_compare(case, nsteps, **opts):
    o = oracle.Sim(case, **opts)
    o.init_hydrostatic()
    g = R.Sim(case, **opts)
    g.init_hydrostatic()
    po, so, pbo, _ = o.get_state()
    pg, sg, pbg, _ = g.get_state()
    np.testing.assert_allclose(pg, po, rtol=1e-13)
    np.testing.assert_array_equal(sg, so)
    for k in range(nsteps):
        n0o, n0g = o.stats()["newton"], g.stats()["newton"]
        assert o.advance(1) == 0
        g.advance(1)
        po, so, pbo, to = o.get_state()
        pg, sg, pbg, tg = g.get_state()
        assert tg == to
        assert np.max(np.abs(pg - po) / np.abs(po)) <= 1e-6, k
        assert np.max(np.abs(sg - so)) <= 1e-6, k
        assert abs((g.stats()["newton"] - n0g) - (o.stats()["newton"] - n0o)) <= 1, k
    return o, g


def test_whole_run_lognormal_case_fp64():
    """The plain method on the 20x20x5 case: 10 steps of 1 day, standard
    Newton to 1e-8, CPR-FGMRES to 1e-8."""
    _run_compare(I.case0(), 10)


def test_whole_run_lognormal_case_mixed_precision():
    """Same run with the FP32 preconditioner: the converged Newton states do
    not depend on the preconditioner precision, so the same tolerances hold."""
    _run_compare(I.case0(), 10, precision=R.PREC_MIXED)


def test_whole_run_channelised_case_mixed_with_chop():
    """The 1M-cell case's physics (channelised facies, 13 wells, 10-day
    steps, saturation chop 0.1) on a 42x38x8 grid: several RAS tiles with a
    ragged edge, mixed precision, 3 steps."""
    c = I.case2(nx=42, ny=38, nz=8)
    _run_compare(c, 3, precision=R.PREC_MIXED)


def test_whole_run_lognormal_case_bf16_ras():
    """RAS factor values stored in BF16 (FP32 arithmetic): the converged
    Newton states still match the FP64 oracle."""
    _run_compare(I.case0(), 5, precision=R.PREC_MIXED_BF16)


def test_whole_run_inexact_newton():
    c = I.small_case(10, 8, 4, seed=51, dt=5.0)
    c.newton, c.newton_tol = "inexact", 1e-7
    _run_compare(c, 4, newton=1, newton_tol=1e-7)


@pytest.mark.parametrize("mk", [
    lambda: I.Case("one", 1, 1, 1, 10.0, 10.0, 10.0, 1000.0, np.array([50.0]), np.array([50.0]),
                   np.array([5.0]), np.array([0.2]), I.Fluid(), [], dt=1.0, n_steps=1),
    lambda: I.small_case(2, 1, 1, seed=61),
    lambda: I.small_case(17, 9, 2, seed=62),
])
@pytest.mark.parametrize("prec", [R.PREC_FP64, R.PREC_MIXED_BF16], ids=["fp64", "bf16"])
def test_edge_grids_run(mk, prec):
    """Degenerate and ragged grids: a single cell without wells, two cells,
    tiles that do not divide the grid; in FP64 and in mixed precision (the
    double-float Krylov basis and SpMV with a single ragged block)."""
    c = mk()
    _run_compare(c, 2, precision=prec)


def test_residual_norm_entry_point():
    """sim_ls_residual_norm equals the oracle's ||b - A x|| on the decoupled system."""
    c = I.small_case(7, 6, 3, seed=81)
    o, gl, _ = _shared_system(c, 800)
    o.ls.setup(); gl.setup()
    _, _, _, db, _ = o.ls.get()
    x = np.random.default_rng(8).standard_normal(2 * (c.n + 2))
    ref = np.linalg.norm(db - o.ls.mv(x))
    assert abs(gl.residual_norm(x) - ref) <= 1e-12 * ref


def test_zero_rhs_and_errors():
    c = I.small_case(4, 4, 2, seed=71)
    o, gl, (rp, ci, val, b, key) = _shared_system(c, 700)
    gl.set(val, np.zeros_like(b), key)
    gl.setup()
    y, its, rel = gl.solve(1e-8)
    assert its == 0 and rel == 0.0 and not y.any()
    with pytest.raises(R.SimError):
        gl.apply(99, np.zeros(2 * (c.n + 2)))
    bad = b.copy(); bad[3] = np.nan
    gl.set(val, bad, key)
    gl.setup()
    with pytest.raises(R.SimError) as e:
        gl.solve(1e-8)
    assert e.value.code == 5          # SIM_ERR_NAN


# the benchmark's configuration of the 1M-cell case (bench.py defaults)
BENCH_OPTS = dict(precision=R.PREC_MIXED_BF16, decoupling=R.DEC_QI, reorder=1, tile_x=4, tile_y=4, max_lin=200)


def test_full_size_channelised_parity():
    """The 1M-cell channelised case in exactly the benchmark's configuration
    (Quasi-IMPES, local potential reordering, mixed precision with BF16 RAS
    values, 4x4 tiles, saturation chop 0.1, relres 1e-6, FGMRES(50) with at
    most 200 iterations): assembly over all cells to 1e-12, the QI-decoupled
    system, every subdomain's order checked on a sample and the level-0 C/F
    split bit for bit on shared input, then one whole 10-day time step on
    both sides from the equilibrium start: per cell |dp|/p <= 1e-6,
    |ds_w| <= 1e-6, Newton iterations within one."""
    c = I.case2()
    o = oracle.Sim(c, **BENCH_OPTS)
    o.init_hydrostatic(); o.store_old(); o.set_dt(c.dt); o.assemble()
    g = R.Sim(c, **BENCH_OPTS)
    g.init_hydrostatic(); g.begin_step(c.dt)
    nrm = g.assemble()
    rp, ci, val, b, key = o.system()
    gval, gb = g.ls.export(R.X_VALS), g.ls.export(R.X_RHS)
    sc = np.repeat(_rowscale(val, rp, len(rp) - 1), np.diff(rp))
    assert (np.abs(gval - val).reshape(-1, 4).max(axis=1) / sc).max() < 1e-12
    assert np.abs(gb - b).max() <= 1e-12 * np.abs(b).max()
    np.testing.assert_allclose(nrm, o.residual_norm(), rtol=1e-12)
    # shared-input setup: QI decoupling, reordering, C/F at level 0
    gl = R.LinearSystem(c.nx, c.ny, c.nz, len(c.wells), rp, ci, [w.perf_cells[0] for w in c.wells], **BENCH_OPTS)
    gl.set(val, b, key)
    gl.setup()
    o.ls.setup()
    _, _, dval, db, _ = o.ls.get()
    np.testing.assert_array_equal(gl.export(R.X_VALS), dval)
    np.testing.assert_array_equal(gl.export(R.X_RHS), db)
    for s in (0, 1, 137, 1249, o.ls.nsub - 1):
        np.testing.assert_array_equal(gl.ras_ext(s), o.ls.sub(s)["ext"])
    np.testing.assert_array_equal(gl.amg_level(0)["cf"], o.ls.amg().level(0)["cf"])
    np.testing.assert_array_equal(gl.amg_level(1)["ci"], o.ls.amg().level(1)["ci"])
    del gl
    # one whole time step, from the equilibrium start, on both sides
    o2 = oracle.Sim(c, **BENCH_OPTS)
    o2.init_hydrostatic()
    g.init_hydrostatic()
    assert o2.advance(1) == 0
    g.advance(1)
    po, so, pbo, to = o2.get_state()
    pg, sg, pbg, tg = g.get_state()
    assert tg == to == c.dt
    assert np.max(np.abs(pg - po) / np.abs(po)) <= 1e-6
    assert np.max(np.abs(sg - so)) <= 1e-6
    assert np.max(np.abs(pbg - pbo) / np.abs(pbo)) <= 1e-6
    assert abs(g.stats()["newton"] - o2.stats()["newton"]) <= 1
    assert np.max(np.abs(so - c.sw_init)) > 0.05          # the step did move water


@pytest.mark.parametrize("precision,newton", [(R.PREC_FP64, "inexact"), (R.PREC_MIXED, "standard")],
                         ids=["fp64_inexact_EW", "fp32_precond_relres1e-6"])
def test_whole_run_fivespot_200k(precision, newton):
    """The 200k-cell five-spot case (100x100x20, 4 rate injectors and a BHP
    producer, layered log-normal permeability, chop 0.1) at full size, the
    two runs its configuration asks for: inexact Newton with the
    Eisenstat-Walker forcing term of eq. (26) in FP64, and standard Newton
    at relres 1e-6 with the FP32 preconditioner (FGMRES in FP64); 3 steps
    of 5 days against the FP64 oracle with the same Newton settings."""
    c = I.case1()
    nw = 1 if newton == "inexact" else 0
    opts = dict(newton=nw, decoupling=R.DEC_QI, max_lin=200)
    o = oracle.Sim(c, **opts)
    g = R.Sim(c, precision=precision, **opts)
    o.init_hydrostatic(); g.init_hydrostatic()
    for k in range(3):
        n0o, n0g = o.stats()["newton"], g.stats()["newton"]
        assert o.advance(1) == 0
        g.advance(1)
        po, so, pbo, to = o.get_state()
        pg, sg, pbg, tg = g.get_state()
        assert tg == to
        assert np.max(np.abs(pg - po) / np.abs(po)) <= 1e-6, k
        assert np.max(np.abs(sg - so)) <= 1e-6, k
        assert abs((g.stats()["newton"] - n0g) - (o.stats()["newton"] - n0o)) <= 1, k


# ---- Quasi-IMPES decoupling (the paper's choice for its large SPE10 runs) ----
@pytest.mark.parametrize("mk,opts", SYS[:3])
def test_quasi_impes_matches_oracle(mk, opts):
    """QI decoupling on shared FP64 input: the decoupled matrix and right-hand
    side bit for bit (both sides evaluate the same round-to-nearest
    operations), the level-0 C/F split bit for bit, RAS / CPR applications to
    1e-10, FGMRES iterations within one."""
    c = mk()
    o, gl, _ = _shared_system(c, 410, decoupling=R.DEC_QI, **opts)
    o.ls.setup(); gl.setup()
    _, _, dval, db, _ = o.ls.get()
    np.testing.assert_array_equal(gl.export(R.X_VALS), dval)
    np.testing.assert_array_equal(gl.export(R.X_RHS), db)
    np.testing.assert_array_equal(gl.amg_level(0)["cf"], o.ls.amg().level(0)["cf"])
    x = np.random.default_rng(41).standard_normal(2 * (c.n + len(c.wells)))
    for op, fo in ((R.OP_RAS, o.ls.ras), (R.OP_CPR, o.ls.cpr)):
        yg, yo = gl.apply(op, x), fo(x)
        assert np.abs(yg - yo).max() <= 1e-10 * np.abs(yo).max(), op
    rco, yo, itso, relo = o.ls.solve(1e-10)
    yg, itsg, relg = gl.solve(1e-10)
    assert rco == 0 and relg <= 1e-10
    assert abs(itsg - itso) <= 1
    assert np.abs(yg - yo).max() <= 1e-7 * np.abs(yo).max()


def test_whole_run_channelised_case_quasi_impes_mixed():
    """The 1M-cell case's physics on a 42x38x8 grid with QI decoupling, mixed
    precision and BF16 RAS values: three steps against the oracle (QI, FP64)."""
    c = I.case2(nx=42, ny=38, nz=8)
    _run_compare(c, 3, precision=R.PREC_MIXED_BF16, decoupling=R.DEC_QI)
