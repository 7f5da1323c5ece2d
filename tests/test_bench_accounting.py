"""The algorithmic byte counts behind bench.py's roofline fractions, on small
hand-made sizes (no GPU): each formula against its terms written out."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_spmv_bytes():
    # 10 block rows, 30 blocks: values + column per block, row pointers,
    # two unknowns per row for each vector
    assert bench.spmv_bytes(10, 30, 16, 4, 4, 4) == 30 * 20 + 11 * 4 + 20 * 12
    assert bench.spmv_bytes(10, 30, 32, 4, 0, 8) == 30 * 36 + 11 * 4 + 20 * 12


class _FakeAMG:
    """Two levels: a 100-row level with 700 entries and 400-entry P to 30
    coarse rows, and a dense 30-row coarsest level."""

    def amg_nlev(self):
        return 2

    def amg_level(self, l):
        if l == 0:
            return dict(n=100, nnz=700, nc=30, nnzP=400, coarse_dense=0)
        return dict(n=30, nnz=300, nc=0, nnzP=0, coarse_dense=1)


def test_vcycle_bytes_fp32():
    vb = 4
    a = 700 * (vb + 4) + 101 * 4
    level0 = 2 * a + 8 * 100 * vb                                   # pre + post smoothing
    level0 += 400 * (vb + 4) + 31 * 4 + 100 * vb + 3 * 30 * vb      # restriction (R = P^T)
    level0 += 400 * (vb + 4) + 101 * 4 + 2 * 100 * vb + 30 * vb     # prolongation
    coarsest = 30 * 30 * 8 + 2 * 30 * vb                            # dense FP64 inverse
    assert bench.vcycle_bytes(_FakeAMG(), "mixed_bf16") == level0 + coarsest


class _FakeRAS:
    """Two subdomains: (owned rows, extended rows, local entries)."""

    def ras_count(self):
        return 2

    def ras_sizes(self, s):
        return [(16, 40, 200), (12, 30, 150)][s]


def test_ras_bytes_bf16():
    own, nxt, nnz = 28, 70, 350
    off = nnz - nxt                                  # off-diagonal blocks
    expect = off * (8 + 2) + nxt * (4 + 12 + 8) + nxt * 8.0 + own * 12.0
    assert bench.ras_bytes(_FakeRAS(), "mixed_bf16") == expect



def test_decoupling_codes_agree():
    """bench.py's decoupling codes are those of the CUDA library's header and
    of the oracle's (both arms must run the same configuration)."""
    import re
    lib = open(os.path.join(ROOT, "include", "resim.h")).read()
    orc = open(os.path.join(ROOT, "oracle", "or_internal.h")).read()
    for name, code in bench.DECOUPLING.items():
        assert int(re.search(r"SIM_DEC_%s = (\d+)" % name.upper(), lib).group(1)) == code
        assert int(re.search(r"OR_DEC_%s = (\d+)" % name.upper(), orc).group(1)) == code


def test_clock_record_parsing():
    """The nvidia-smi samples taken during the timed region: median SM
    clock, the maximum, and every throttle reason seen active at least once
    (what decides whether a run is kept)."""
    c = bench.Clocks(0)

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    rows = [
        "0, 2070, 2070, 310.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 402.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 398.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    c.f.write("\n".join(rows) + "\n")
    c.f.flush()
    c.p = _Done()
    d = c.stop()
    assert d["sm_mhz"] == 2070.0 and d["sm_max_mhz"] == 2070.0 and d["samples"] == 3
    assert d["power_w_max"] == 402.0 and d["reasons"] == ["sw_power_cap"]


def test_clock_record_without_nvidia_smi():
    c = bench.Clocks(0)
    try:
        assert c.stop() is None                   # never started: no record, no exception
    finally:
        c.f.close()
        os.unlink(c.f.name)


def test_state_difference():
    """Mixed-precision and FP64 end states: relative in pressure, absolute
    in saturation, largest over the cells."""
    import numpy as np
    ref = (np.array([200.0, 100.0, 150.0]), np.array([0.2, 0.5, 0.8]))
    run = (np.array([200.0, 100.0002, 150.0]), np.array([0.2, 0.5, 0.8000003]))
    d = bench.state_difference(run, ref)
    assert abs(d["p_rel_max"] - 2e-6) < 1e-12 and abs(d["sw_abs_max"] - 3e-7) < 1e-12
    assert bench.state_difference(ref, ref) == {"p_rel_max": 0.0, "sw_abs_max": 0.0}


def test_host_state_never_raises():
    class _Broken:
        def get_state(self):
            raise RuntimeError("no device")
    assert bench._host_state(_Broken()) is None
