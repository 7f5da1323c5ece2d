"""The synthetic workloads against the recipe the benchmark and the tests
rely on (seeded; no GPU): facies fractions and permeability distributions of
the channelised case, its anisotropic correlation, well layout, the ensemble's
size ranges, and reproducibility from the seed."""
import math

import numpy as np

from paper_1701_06254_gb300 import inputs as I


def test_channelised_case_facies_and_permeability():
    c = I.case2(nx=100, ny=100, nz=20)
    lnk = np.log(c.kx)
    sand = c.phi > 0.2
    assert abs(sand.mean() - 0.35) < 0.005                        # thresholded at the 0.65 quantile
    assert abs(lnk[sand].mean() - math.log(500.0)) < 0.02
    assert abs(lnk[~sand].mean() - math.log(5.0)) < 0.02
    assert abs(lnk[sand].std() - 0.5) < 0.02 and abs(lnk[~sand].std() - 0.5) < 0.02
    np.testing.assert_allclose(c.kz, 0.1 * c.kx)
    np.testing.assert_array_equal(c.kx, c.ky)
    assert set(np.unique(c.phi)) == {0.10, 0.25}


def test_channelised_case_is_anisotropic():
    """Correlation lengths 40 / 8 / 2 cells: neighbouring cells along x share
    their facies more often than along y, and along y more than along z."""
    c = I.case2(nx=100, ny=100, nz=20)
    s = (c.phi > 0.2).reshape(c.nz, c.ny, c.nx)
    same_x = (s[:, :, 1:] == s[:, :, :-1]).mean()
    same_y = (s[:, 1:, :] == s[:, :-1, :]).mean()
    same_z = (s[1:, :, :] == s[:-1, :, :]).mean()
    assert same_x > same_y > same_z > 0.5


def test_channelised_case_wells():
    c = I.case2()
    prod = [w for w in c.wells if w.kind == I.PROD]
    inj = [w for w in c.wells if w.kind == I.INJ]
    assert len(prod) == 9 and len(inj) == 4
    assert all(w.control == I.BHP and w.target == 150.0 for w in prod)
    assert all(w.control == I.WRATE and w.target == 800.0 for w in inj)
    for w in c.wells:                                            # whole columns, top to bottom
        assert len(w.perf_cells) == c.nz
        assert np.all(np.diff(w.perf_cells) == c.nx * c.ny)


def test_ensemble_sizes_and_seeds():
    cases = I.ensemble(16)
    for c in cases:
        assert 32 <= c.nx <= 128 and 32 <= c.ny <= 128 and 8 <= c.nz <= 32
        assert c.dt == 10.0
    assert len({(c.nx, c.ny, c.nz) for c in cases}) > 8            # uneven sizes
    a, b = I.ensemble_member(3), I.ensemble_member(3)
    np.testing.assert_array_equal(a.kx, b.kx)                      # reproducible from the seed
    assert not np.array_equal(I.case2(seed=5, nx=40, ny=40, nz=8).kx, I.case2(seed=6, nx=40, ny=40, nz=8).kx)


def test_plain_case_recipe():
    c = I.case0()
    lnk = np.log(c.kx)
    assert (c.nx, c.ny, c.nz) == (20, 20, 5)
    assert abs(lnk.mean() - math.log(100.0)) < 0.06 and abs(lnk.std() - 1.0) < 0.05
    assert np.all(c.phi == 0.2)
    assert len(c.wells) == 2 and c.dt == 1.0 and c.n_steps == 10
