"""Host-side checks of the C-ABI library (no GPU calls): it builds for
sm_103a, loads, and exports every entry point that include/resim.h declares."""
import ctypes
import os
import re

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
