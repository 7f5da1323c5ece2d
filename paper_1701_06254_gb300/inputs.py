"""Seeded synthetic inputs for the oil-water reservoir workloads.

This module only draws data: grids, permeability / porosity fields, well
placements and the fluid constants.  It contains none of the method's
arithmetic (no PVT, no transmissibility, no well index, no residual), so the
CUDA path and the CPU oracle can both take their inputs from it without
sharing any solver code.

The paper's own workloads (SPE10 and two CMG IMEX decks, Sec. "Numerical
experiments") are not available; the cases below are synthetic stand-ins
with the sizes and the kind of heterogeneity those models have.

Units: lengths in m, permeability in mD, pressure in bar, time in days,
density in kg/m3, viscosity in cP, compressibility in 1/bar, well rates in
standard m3/day.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# well kinds / controls (Sec. "Two-phase oil-water flow model", eqs. 11-14)
INJ, PROD = 0, 1
BHP, WRATE, ORATE, LRATE, SHUT = 0, 1, 2, 3, 4


@dataclass
class Fluid:
    """Fluid and rock-compressibility constants; index 0 = water, 1 = oil."""
    rho_ref: tuple = (1000.0, 800.0)
    c_f: tuple = (4.5e-5, 1.0e-4)
    mu_ref: tuple = (0.5, 2.0)
    c_mu: tuple = (0.0, 0.0)
    p_ref: float = 200.0
    c_r: float = 4.5e-5
    swc: float = 0.2
    sor: float = 0.2
    nw: float = 2.0
    no: float = 2.0
    krw_max: float = 1.0
    kro_max: float = 1.0
    g: float = 9.80665
    pc_sw: tuple = ()          # capillary pressure table (eq. 9): s_w ascending ...
    pc: tuple = ()             # ... and p_c in bar; empty = no capillary pressure


@dataclass
class Well:
    kind: int
    control: int
    target: float          # bar (BHP) or sm3/day (rate)
    perf_cells: list       # natural cell indices, top to bottom
    r_w: float = 0.1
    skin: float = 0.0
    z_ref: float | None = None  # reference depth of p_b; None -> top perforation depth
    bhp_limit: float = 0.0      # rate wells: injector maximum / producer minimum p_b (bar), 0 = none


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    top: float
    kx: np.ndarray
    ky: np.ndarray
    kz: np.ndarray
    phi: np.ndarray
    fluid: Fluid
    wells: list
    dt: float
    n_steps: int
    p_init: float = 200.0      # oil pressure at the top datum
    sw_init: float = 0.2
    newton: str = "standard"   # or "inexact"
    newton_tol: float = 1e-8
    lin_tol: float = 1e-8
    sat_chop: float = 0.0      # max |ds_w| per Newton update (0: full step)
    opts: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def cell(self, i: int, j: int, k: int) -> int:
        return i + self.nx * (j + self.ny * k)

    def column(self, i: int, j: int) -> list:
        return [self.cell(i, j, k) for k in range(self.nz)]

    def well_z_ref(self, w: Well) -> float:
        if w.z_ref is not None:
            return w.z_ref
        k0 = w.perf_cells[0] // (self.nx * self.ny)
        return self.top + (k0 + 0.5) * self.dz


def _lognormal_iid(rng, n, mean_ln, sigma):
    return np.exp(mean_ln + sigma * rng.standard_normal(n))


def _gauss_kernel(sig):
    r = int(math.ceil(3.0 * sig))
    x = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (x / sig) ** 2)
    return w / w.sum()


def _grf(rng, nx, ny, nz, lx, ly, lz):
    """Gaussian random field: white noise convolved with a separable Gaussian
    kernel (sigma = correlation length / 2 per axis, truncated at 3 sigma,
    zero padded), rescaled to zero mean and unit variance.  Array order is
    [k, j, i] so that ravel() gives the natural cell index i + nx(j + ny k)."""
    f = rng.standard_normal((nz, ny, nx))
    for axis, ell in ((2, lx), (1, ly), (0, lz)):
        w = _gauss_kernel(max(ell / 2.0, 1e-3))
        r = (len(w) - 1) // 2            # centred "same" window, also when the kernel is longer than the axis
        f = np.apply_along_axis(lambda v: np.convolve(v, w)[r:r + len(v)], axis, f)
    f = (f - f.mean()) / f.std()
    return f.ravel()


def case0(seed: int = 0) -> Case:
    """Plain-method case: 20x20x5, i.i.d. log-normal k (ln 100 mD, sigma 1),
    kv/kh = 0.1, phi = 0.2, rate injector at (0,0), BHP producer at (19,19),
    10 steps of 1 day, standard Newton 1e-8, linear relres 1e-8."""
    nx, ny, nz = 20, 20, 5
    rng = np.random.default_rng(seed)
    kh = _lognormal_iid(rng, nx * ny * nz, math.log(100.0), 1.0)
    c = Case("lognormal_20x20x5", nx, ny, nz, 20.0, 20.0, 5.0, 2000.0,
             kh.copy(), kh.copy(), 0.1 * kh, np.full(nx * ny * nz, 0.2),
             Fluid(), [], dt=1.0, n_steps=10)
    c.wells = [Well(INJ, WRATE, 200.0, c.column(0, 0)),
               Well(PROD, BHP, 150.0, c.column(nx - 1, ny - 1))]
    return c


def case1(seed: int = 1, nx=100, ny=100, nz=20) -> Case:
    """200k-cell case: log-normal k (sigma 1.5) with a per-layer multiplier
    10^U(-1,1), porosity 0.1-0.3 rising with ln k, five-spot wells
    (4 corner injectors at 500 sm3/d, central producer at 150 bar),
    30 steps of 5 days."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    z = rng.standard_normal(n)
    layer_mult = 10.0 ** rng.uniform(-1.0, 1.0, nz)
    lnk = math.log(100.0) + 1.5 * z + np.log(np.repeat(layer_mult, nx * ny))
    kh = np.exp(lnk)
    # porosity: normal CDF of the standardised ln k mapped to [0.1, 0.3]
    zs = (lnk - lnk.mean()) / lnk.std()
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(zs / math.sqrt(2.0)))
    phi = 0.1 + 0.2 * cdf
    c = Case(f"fivespot_{nx}x{ny}x{nz}", nx, ny, nz, 20.0, 20.0, 5.0, 2000.0,
             kh.copy(), kh.copy(), 0.1 * kh, phi, Fluid(), [], dt=5.0, n_steps=30,
             newton="inexact", newton_tol=1e-8, lin_tol=1e-6, sat_chop=0.1)
    c.wells = [Well(INJ, WRATE, 500.0, c.column(i, j))
               for (i, j) in ((0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1))]
    c.wells.append(Well(PROD, BHP, 150.0, c.column(nx // 2, ny // 2)))
    return c


def case2(seed: int = 2, nx=200, ny=200, nz=25) -> Case:
    """1M-cell channelised case: anisotropic Gaussian random field
    (correlation lengths 40/8/2 cells) thresholded at its 0.65 quantile into
    sand (35 %, ln k ~ N(ln 500, 0.5)) and shale (ln k ~ N(ln 5, 0.5)),
    kv/kh = 0.1, phi 0.25 / 0.10; 9 BHP producers (150 bar) on a 3x3
    lattice and 4 rate injectors (800 sm3/d); 50 steps of 10 days."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    f = _grf(rng, nx, ny, nz, 40.0 * nx / 200.0, 8.0 * ny / 200.0, 2.0 * nz / 25.0)
    thr = np.quantile(f, 0.65)
    sand = f > thr
    noise = rng.standard_normal(n)
    lnk = np.where(sand, math.log(500.0), math.log(5.0)) + 0.5 * noise
    kh = np.exp(lnk)
    phi = np.where(sand, 0.25, 0.10)
    c = Case(f"channelised_{nx}x{ny}x{nz}", nx, ny, nz, 20.0, 20.0, 5.0, 2000.0,
             kh.copy(), kh.copy(), 0.1 * kh, phi, Fluid(), [], dt=10.0, n_steps=50,
             newton="standard", newton_tol=1e-6, lin_tol=1e-6, sat_chop=0.1)
    pi = [round(x * nx / 200.0) for x in (33, 100, 166)]
    pj = [round(x * ny / 200.0) for x in (33, 100, 166)]
    for j in pj:
        for i in pi:
            c.wells.append(Well(PROD, BHP, 150.0, c.column(i, j)))
    for (i, j) in ((66, 66), (133, 66), (66, 133), (133, 133)):
        c.wells.append(Well(INJ, WRATE, 800.0 * (nx * ny) / 40000.0,
                            c.column(round(i * nx / 200.0), round(j * ny / 200.0))))
    return c


def ensemble_member(k: int, seed0: int = 2000, size_lo=(32, 32, 8), size_hi=(128, 128, 32),
                    n_steps: int = 20) -> Case:
    """Member k of the ensemble workload: the channelised two-facies field,
    wells and Newton settings of case2 on a grid drawn from
    U{32..128} x U{32..128} x U{8..32} (seed seed0 + k; correlation lengths,
    well positions and injection rates scale with the grid), 10-day steps.
    size_lo / size_hi narrow the draw for tests."""
    rng = np.random.default_rng(seed0 + k)
    nx = int(rng.integers(size_lo[0], size_hi[0] + 1))
    ny = int(rng.integers(size_lo[1], size_hi[1] + 1))
    nz = int(rng.integers(size_lo[2], size_hi[2] + 1))
    c = case2(seed=seed0 + k, nx=nx, ny=ny, nz=nz)
    c.name = f"ens{k}_{nx}x{ny}x{nz}"
    c.dt, c.n_steps = 10.0, n_steps
    return c


def ensemble(members: int = 128, seed0: int = 2000, **kw) -> list:
    """The ensemble workload: `members` independent models (default 128,
    seeds 2000..2127, about 16M cells in all)."""
    return [ensemble_member(k, seed0, **kw) for k in range(members)]


def small_case(nx=6, ny=5, nz=3, seed=7, sigma=1.0, gravity=True, dt=1.0) -> Case:
    """Tiny heterogeneous case used by parity tests: i.i.d. log-normal k,
    one rate injector and one BHP producer in opposite corner columns."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    kh = _lognormal_iid(rng, n, math.log(100.0), sigma)
    fl = Fluid()
    if not gravity:
        fl.g = 0.0
    c = Case(f"small_{nx}x{ny}x{nz}", nx, ny, nz, 20.0, 20.0, 5.0, 2000.0,
             kh.copy(), kh.copy(), 0.1 * kh, 0.15 + 0.1 * rng.random(n), fl, [],
             dt=dt, n_steps=3)
    c.wells = [Well(INJ, WRATE, 100.0, c.column(0, 0)),
               Well(PROD, BHP, 150.0, c.column(nx - 1, ny - 1))]
    return c


def random_state(case: Case, seed: int, s_lo=0.3, s_hi=0.7, p_lo=170.0, p_hi=230.0):
    """A random iterate (p, s_w, p_b) away from relative-permeability kinks,
    used to check Jacobians and single linear systems."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(p_lo, p_hi, case.n)
    sw = rng.uniform(s_lo, s_hi, case.n)
    pb = np.array([(p_hi + 30.0) if w.kind == INJ else (p_lo - 30.0) for w in case.wells])
    return p, sw, pb


CASES = {"lognormal": case0, "fivespot": case1, "channelised": case2}
