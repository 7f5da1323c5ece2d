"""The allocation-free residual norm, sim_ls_residual_norm_noalloc.

Some callers must not allocate device memory (code running under another
allocator's budget, latency-sensitive loops where cudaMalloc/cudaFree would
synchronise the device).  For them the library offers a variant of its
residual norm whose scratch is a fixed array inside the library.  This test
calls it through the C ABI twice in a row, with different vectors, and
checks each result against the allocating entry point sim_ls_residual_norm
to 1e-12 relative (the two sum the same squares in different orders).

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _system():
    import oracle
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    c = I.small_case(9, 7, 4, seed=91)
    o = oracle.Sim(c)
    p0, s0, pb0 = I.random_state(c, 900)
    p1, s1, pb1 = I.random_state(c, 901)
    o.set_state(p0, s0, pb0); o.store_old(); o.set_dt(1.5)
    o.set_state(p1, s1, pb1); o.assemble()
    rp, ci, val, b, key = o.system()
    gl = R.LinearSystem(c.nx, c.ny, c.nz, len(c.wells), rp, ci, [w.perf_cells[0] for w in c.wells])
    gl.set(val, b, key)
    gl.setup()
    return gl, 2 * (c.n + len(c.wells))


def test_noalloc_residual_norm_matches_allocating_entry_point():
    import torch
    import paper_1701_06254_gb300 as R
    gl, nu = _system()
    fn = R.lib().sim_ls_residual_norm_noalloc
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (11, 12):                      # two calls in a row share the scratch array
        x = np.random.default_rng(seed).standard_normal(nu)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        rc = fn(gl.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert rc == 0, R.lib().sim_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        ref = gl.residual_norm(x)
        assert ref > 0
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def test_noalloc_residual_norm_rejects_host_memory():
    import torch
    import paper_1701_06254_gb300 as R
    gl, nu = _system()
    x = np.zeros(nu)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = R.lib().sim_ls_residual_norm_noalloc(gl.h, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(out.data_ptr()))
    assert rc == 1                              # SIM_ERR_ARG
    assert b"device memory" in R.lib().sim_last_error()
