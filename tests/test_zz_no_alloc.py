"""The allocation-free residual norm, sim_ls_residual_norm_noalloc.

Some callers must not allocate device memory: code running under another
allocator's budget (a framework whose caching allocator already holds the
GPU's memory, so a fresh cudaMalloc can fail) and latency-sensitive loops in
which the device-wide synchronisation of cudaMalloc / cudaFree is not
acceptable.  For them the library offers a variant of its residual norm
whose scratch is a fixed array inside the library.

The tests call it through the C ABI, several times in a row on the same
shared array, first on a system large enough to need several partial sums
(16,000 cells: 4 partials) and then on a small one (1 partial), and check
every result against the allocating entry point sim_ls_residual_norm and
against ||b - A x|| of the same decoupled system computed by the CPU oracle,
to 1e-12 relative (the three sum the same squares in different orders).

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _system(nx, ny, nz, seed):
    """The Jacobian of a random state of a small heterogeneous case, set up
    (decoupled) on the GPU and in the oracle."""
    import oracle
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    c = I.small_case(nx, ny, nz, seed=seed)
    o = oracle.Sim(c)
    p0, s0, pb0 = I.random_state(c, seed + 900)
    p1, s1, pb1 = I.random_state(c, seed + 901)
    o.set_state(p0, s0, pb0); o.store_old(); o.set_dt(1.5)
    o.set_state(p1, s1, pb1); o.assemble()
    rp, ci, val, b, key = o.system()
    wc0 = [w.perf_cells[0] for w in c.wells]
    gl = R.LinearSystem(c.nx, c.ny, c.nz, len(c.wells), rp, ci, wc0)
    gl.set(val, b, key)
    gl.setup()
    ol = oracle.LinearSystem(c.nx, c.ny, c.nz, len(c.wells), rp, ci, wc0)
    ol.set(val, b, key)
    ol.setup()
    return gl, ol, 2 * (c.n + len(c.wells))


def _oracle_norm(ol, x):
    db = ol.get()[3]                          # decoupled right-hand side
    return float(np.linalg.norm(db - ol.mv(x)))


def test_noalloc_residual_norm_matches_allocating_entry_point_and_oracle():
    import torch
    import paper_1701_06254_gb300 as R
    big = _system(40, 40, 10, 91)             # 16,002 block rows: 4 partial sums
    small = _system(9, 7, 4, 92)              # 254 block rows: 1 partial sum
    assert big[2] // 2 > 3 * 4096 and small[2] // 2 < 4096
    fn = R.lib().sim_ls_residual_norm_noalloc
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # the large system first, then the small one twice: later calls read
    # fewer partials than an earlier call left in the shared array
    for (gl, ol, nu), seed in ((big, 11), (small, 12), (small, 13), (big, 14)):
        x = np.random.default_rng(seed).standard_normal(nu)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        rc = fn(gl.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert rc == 0, R.lib().sim_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        ref = gl.residual_norm(x)
        orc = _oracle_norm(ol, x)
        assert ref > 0 and orc > 0
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)
        assert abs(got - orc) <= 1e-12 * orc, (got, orc)


def test_noalloc_residual_norm_rejects_host_memory():
    import torch
    import paper_1701_06254_gb300 as R
    gl, _, nu = _system(9, 7, 4, 92)
    x = np.zeros(nu)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = R.lib().sim_ls_residual_norm_noalloc(gl.h, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(out.data_ptr()))
    assert rc == 1                              # SIM_ERR_ARG
    assert b"device memory" in R.lib().sim_last_error()


def test_noalloc_residual_norm_rejects_another_devices_memory():
    import torch
    import paper_1701_06254_gb300 as R
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second visible GPU")
    gl, _, nu = _system(9, 7, 4, 92)
    x1 = torch.zeros(nu, dtype=torch.float64, device="cuda:1")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    rc = R.lib().sim_ls_residual_norm_noalloc(gl.h, ctypes.c_void_p(x1.data_ptr()), ctypes.c_void_p(out.data_ptr()))
    assert rc == 1                              # SIM_ERR_ARG, before any launch
    assert b"current device" in R.lib().sim_last_error()
