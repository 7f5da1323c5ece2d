"""Host-side checks of the C-ABI library (no GPU calls): it builds for
sm_103a, loads, and exports every entry point that include/resim.h declares."""
import copy
import ctypes
import dataclasses
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "resim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:sim_status|void|const char|long long|sim_ls_t)\s*\*?\s*(sim_\w+)\s*\(",
                           src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sim_create", "sim_destroy", "sim_assemble", "sim_linear_solve", "sim_newton_step", "sim_advance",
              "sim_set_state", "sim_get_state", "sim_ls_create", "sim_ls_setup", "sim_ls_solve", "sim_ls_export",
              "sim_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol():
    import paper_1701_06254_gb300 as R
    path = R.build()
    L = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_default_options_and_error_path_without_gpu():
    """sim_default_options and argument validation run on the host only."""
    import paper_1701_06254_gb300 as R
    o = R.make_options()
    assert o.restart == 50 and o.max_lin == 100 and o.tile_x == 4 and o.amg_coarse_max == 128
    assert abs(o.amg_theta - 0.25) < 1e-15 and o.decoupling == R.DEC_ABF
    L = R.lib()
    h = ctypes.c_void_p()
    rc = L.sim_create(ctypes.byref(h), None, None, None, None, 0, ctypes.byref(o))
    assert rc == 1                                   # SIM_ERR_ARG, no device touched
    assert b"NULL" in L.sim_last_error()
    rc = L.sim_ls_create(ctypes.byref(h), 0, 1, 1, 0, None, None, None, ctypes.byref(o))
    assert rc == 1


def _create(R, case, **kw):
    """sim_create on a case, with option fields overridden; returns the status
    and the library's error text."""
    L = R.lib()
    o = R.make_options(dt=case.dt)
    for k, v in kw.items():
        setattr(o, k, v)
    g, fl, wells, keep = R._case_structs(case)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (case.kx, case.ky, case.kz, case.phi)]
    rock = R.Rock(*(a.ctypes.data for a in arrs))
    h = ctypes.c_void_p()
    rc = L.sim_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(rock), ctypes.byref(fl), wells,
                      len(case.wells), ctypes.byref(o))
    return rc, L.sim_last_error().decode()


@pytest.mark.parametrize("field,value,text", [
    ("precision", 3, "precision"), ("precision", -1, "precision"), ("decoupling", 3, "decoupling"),
    ("reorder", 2, "reorder"), ("newton", 2, "Newton"), ("newton_tol", -1e-8, "newton_tol"),
    ("newton_tol", float("nan"), "newton_tol"), ("lin_tol", float("inf"), "lin_tol"),
    ("amg_theta", 1.5, "amg_theta"), ("amg_theta", float("nan"), "amg_theta"),
    ("max_newton", -1, "limit"), ("max_cuts", -2, "limit"), ("amg_coarse_max", -1, "limit"),
    ("dt", 0.0, "dt"), ("dt", float("inf"), "dt")])
def test_bad_options_are_rejected_before_device_work(field, value, text):
    """Every rejected option value returns SIM_ERR_ARG with its name in the
    message, on a machine without a GPU as on one with it: the checks run
    before any allocation."""
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    rc, msg = _create(R, I.case0(), **{field: value})
    assert rc == 1 and text in msg, (rc, msg)


def test_bad_wells_are_rejected_before_device_work():
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    base = I.case0()
    bad = [
        (0, dict(kind=5), "bad kind"),
        (0, dict(control=I.ORATE), "need a producer"),          # an injector injects water only
        (0, dict(control=I.LRATE), "need a producer"),
        (0, dict(control=7), "unknown control"),
        (0, dict(target=0.0), "positive"),
        (0, dict(target=float("inf")), "positive"),
        (1, dict(bhp_limit=-1.0), "BHP limit"),
        (1, dict(bhp_limit=float("nan")), "BHP limit"),
        (0, dict(perf_cells=np.array([base.n], np.int32)), "outside the grid"),
        (0, dict(perf_cells=np.array([-1], np.int32)), "outside the grid"),
    ]
    for w, change, text in bad:
        c = copy.deepcopy(base)
        c.wells[w] = dataclasses.replace(c.wells[w], **change)
        rc, msg = _create(R, c)
        assert rc == 1 and text in msg, (change, rc, msg)


def test_bad_capillary_tables_are_rejected_before_device_work():
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    for sw, pc, text in (((0.3, 0.2), (1.0, 0.5), "must increase"),
                         ((0.2, 0.3), (1.0, float("nan")), "not finite"),
                         (tuple(np.linspace(0.2, 0.8, 17)), tuple(np.linspace(2.0, 0.0, 17)), "0 to 16 points")):
        c = I.case0()
        c.fluid = dataclasses.replace(c.fluid, pc_sw=sw, pc=pc)
        rc, msg = _create(R, c)
        assert rc == 1 and text in msg, (sw, rc, msg)


def test_ls_create_checks_options():
    import paper_1701_06254_gb300 as R
    L = R.lib()
    o = R.make_options(decoupling=9)
    rp = np.array([0, 1], np.int32)
    ci = np.array([0], np.int32)
    h = ctypes.c_void_p()
    rc = L.sim_ls_create(ctypes.byref(h), 1, 1, 1, 0, rp.ctypes.data, ci.ctypes.data, None, ctypes.byref(o))
    assert rc == 1 and b"decoupling" in L.sim_last_error()


def test_no_cpu_fallback_without_a_gpu():
    """On a machine without a usable GPU the product path raises; it never
    computes on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    with pytest.raises(R.SimError) as e:
        R.Sim(I.case0())
    assert e.value.code == 2                          # SIM_ERR_CUDA
    with pytest.raises(R.SimError):
        R.WarmStart(seed=1)


def test_solve_tolerances_are_checked_on_the_host():
    import paper_1701_06254_gb300 as R
    L = R.lib()
    its, rel = ctypes.c_int(), ctypes.c_double()
    for tol in (-1.0, float("nan"), float("inf")):
        assert L.sim_ls_solve(None, tol, None, ctypes.byref(its), ctypes.byref(rel)) == 1
        assert b"tol" in L.sim_last_error()
        assert L.sim_linear_solve(None, tol, ctypes.byref(its), ctypes.byref(rel)) == 1
        assert b"tol" in L.sim_last_error()
    assert L.sim_ls_solve(None, 1e-8, None, None, None) == 1           # NULL handle
    assert b"NULL" in L.sim_last_error()


def test_every_workload_passes_the_host_checks():
    """The workloads the tests and the benchmark run get past every host-side
    check (without a GPU sim_create then stops at its first CUDA call)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    cases = [I.case0(), I.case1(nx=20, ny=20, nz=4), I.case2(nx=24, ny=24, nz=5), I.ensemble_member(0),
             I.small_case()]
    for c in cases:
        for prec in (R.PREC_FP64, R.PREC_MIXED, R.PREC_MIXED_BF16):
            for dec in (R.DEC_NONE, R.DEC_ABF, R.DEC_QI):
                o = dict(newton=0 if c.newton == "standard" else 1, newton_tol=c.newton_tol, lin_tol=c.lin_tol,
                         sat_chop=c.sat_chop, precision=prec, decoupling=dec)
                rc, msg = _create(R, c, **o)
                assert rc == 2, (c.name, prec, dec, rc, msg)


def test_grid_size_limit():
    """Grids above 50M cells are refused before any device work (the solver
    setup's counts are 32-bit)."""
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    c = I.case0()
    c.nx, c.ny, c.nz = 400, 400, 320                    # 51.2M cells; the rock arrays are never read
    rc, msg = _create(R, c)
    assert rc == 1 and "too large" in msg, (rc, msg)


def test_noalloc_size_rule_on_the_host(tmp_path):
    """The allocation-free residual norm accepts 1 .. 4096 * 4096 block rows
    (one partial sum per 4096 rows in a fixed array of 4096) and refuses
    anything else before it touches the GPU.  The rule is a plain C header
    of the library, compiled and run here without a GPU."""
    import subprocess
    hdr = os.path.join(ROOT, "paper_1701_06254_gb300", "csrc", "noalloc_limit.h")
    src = tmp_path / "rule.c"
    src.write_text('#include <stdio.h>\n#include "%s"\nint main(void) {\n'
                   '  long long v[] = {0, 1, 4096, 4097, 16002, 4096LL * 4096, 4096LL * 4096 + 1, -5};\n'
                   '  for (int i = 0; i < 8; i++) printf("%%lld\\n", rs_noalloc_blocks(v[i]));\n'
                   '  return 0;\n}\n' % hdr)
    exe = tmp_path / "rule"
    subprocess.run(["gcc", "-O2", "-o", str(exe), str(src)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out == [-1, 1, 1, 2, 4, 4096, -1, -1]
