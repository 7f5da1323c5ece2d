"""ctypes binding of the CPU oracle (plain C, FP64).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The CUDA product path never imports it.

The C sources follow arXiv 1701.06254 step by step (model: eqs. 3-18,
Newton: Algorithm 1 and eq. 26, processing: eqs. 28-32, preconditioner:
Algorithm 2); each C function names the passage it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["or_model.c", "or_solve.c", "or_amg.c"]
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_LIB_OMP = os.path.join(_LIBDIR, "liboracle_omp.so")
_lib = None
_lib_omp = None

DEFAULT_OPTS = dict(decoupling=1, reorder=1, newton=0, newton_tol=1e-8, lin_tol=1e-8,
                    max_newton=20, restart=50, max_lin=100, tile_x=4, tile_y=4,
                    amg_theta=0.25, amg_max_levels=25, amg_coarse_max=128,
                    seed=0x5EED, max_cuts=6, dt=1.0, sat_chop=0.0, krylov=0, overlap=1, interp=0)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle into oracle/_lib/liboracle.so (gcc, -O2,
    -ffp-contract=off so that no multiply-add is fused); omp=True builds
    liboracle_omp.so, the same sources with OpenMP on the loops that write
    disjoint outputs (bit-identical results, for timing on all cores)."""
    out = _LIB_OMP if omp else _LIB
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "or_internal.h")]
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return out
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    compile_sources(_HERE, tmp, omp=omp)
    os.replace(tmp, out)
    return out


def compile_sources(src_dir: str, out: str, omp: bool = False) -> None:
    """gcc the oracle's C files found in src_dir into the shared library out
    (also used by the tests that build a copy with a planted mistake)."""
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC", "-shared",
           "-Wno-unknown-pragmas"] + (["-fopenmp"] if omp else []) + \
        ["-o", out] + [os.path.join(src_dir, s) for s in _SRC] + ["-lm"]
    subprocess.run(cmd, check=True)


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("top", C.c_double)]


class Fluid(C.Structure):
    _fields_ = [("rho_ref", C.c_double * 2), ("c_f", C.c_double * 2), ("mu_ref", C.c_double * 2),
                ("c_mu", C.c_double * 2), ("p_ref", C.c_double), ("c_r", C.c_double),
                ("swc", C.c_double), ("sor", C.c_double), ("nw", C.c_double), ("no", C.c_double),
                ("krw_max", C.c_double), ("kro_max", C.c_double), ("g", C.c_double),
                ("pc_n", C.c_int), ("pc_sw", C.POINTER(C.c_double)), ("pc_val", C.POINTER(C.c_double))]


class Well(C.Structure):
    _fields_ = [("kind", C.c_int), ("control", C.c_int), ("target", C.c_double),
                ("r_w", C.c_double), ("skin", C.c_double), ("z_ref", C.c_double),
                ("n_perf", C.c_int), ("perf_cell", C.POINTER(C.c_int)),
                ("wi", C.POINTER(C.c_double)), ("bhp_limit", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("decoupling", C.c_int), ("reorder", C.c_int), ("newton", C.c_int),
                ("newton_tol", C.c_double), ("lin_tol", C.c_double),
                ("max_newton", C.c_int), ("restart", C.c_int), ("max_lin", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("amg_theta", C.c_double),
                ("amg_max_levels", C.c_int), ("amg_coarse_max", C.c_int),
                ("seed", C.c_uint64), ("max_cuts", C.c_int), ("dt", C.c_double), ("sat_chop", C.c_double),
                ("krylov", C.c_int), ("overlap", C.c_int), ("interp", C.c_int)]


def make_opts(**kw) -> Opts:
    d = dict(DEFAULT_OPTS)
    d.update(kw)
    o = Opts()
    for k, v in d.items():
        setattr(o, k, v)
    return o


P = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def _sig(lib):
    s = {
        "or_sim_create": (P, [C.POINTER(Grid), _dp, _dp, _dp, _dp, C.POINTER(Fluid), C.POINTER(Well), C.c_int, C.POINTER(Opts)]),
        "or_sim_destroy": (None, [P]),
        "or_sim_init_hydrostatic": (None, [P, C.c_double, C.c_double]),
        "or_sim_set_state": (None, [P, _dp, _dp, _dp, C.c_double]),
        "or_sim_get_state": (None, [P, _dp, _dp, _dp, _dp]),
        "or_sim_store_old": (None, [P]),
        "or_sim_assemble": (None, [P]),
        "or_sim_residual_norm": (C.c_double, [P]),
        "or_sim_newton": (C.c_int, [P, _ip]),
        "or_sim_advance": (C.c_int, [P, C.c_int]),
        "or_sim_linear_solve": (C.c_int, [P, C.c_double, _dp, _ip, _dp]),
        "or_sim_lsys": (P, [P]),
        "or_sim_set_dt": (None, [P, C.c_double]),
        "or_sim_stats": (None, [P, _dp]),
        "or_sim_well_rates": (None, [P, _dp, _dp]),
        "or_sim_mass": (None, [P, _dp, _dp]),
        "or_sim_get_wi": (None, [P, _dp]),
        "or_sim_set_well": (None, [P, C.c_int, C.c_int, C.c_double, C.c_double]),
        "or_sim_well_controls": (None, [P, _ip, _dp]),
        "or_ls_create": (P, [C.c_int, C.c_int, C.c_int, C.c_int, _ip, _ip, _ip, C.POINTER(Opts)]),
        "or_ls_destroy": (None, [P]),
        "or_ls_set": (None, [P, _dp, _dp, _dp]),
        "or_ls_set_opts": (None, [P, C.POINTER(Opts)]),
        "or_ls_setup": (C.c_int, [P]),
        "or_ls_solve": (C.c_int, [P, C.c_double, _dp, _ip, _dp]),
        "or_ls_get": (None, [P, _ip, _ip, _dp, _dp, _dp]),
        "or_ls_sizes": (None, [P, _ip]),
        "or_ls_mv": (None, [P, _dp, _dp]),
        "or_ls_cpr": (None, [P, _dp, _dp]),
        "or_ls_ras": (None, [P, _dp, _dp]),
        "or_ls_amg": (P, [P]),
        "or_ls_sub_sizes": (None, [P, C.c_int, _ip]),
        "or_ls_sub_get": (None, [P, C.c_int, _ip, _ip, _ip, _ip, _dp, _dp]),
        "or_amg_new": (P, [C.c_int, _ip, _ip, _dp, C.c_double, C.c_uint64, C.c_int, C.c_int, C.c_int]),
        "or_interp_given": (None, [C.c_int, _ip, _ip, _dp, C.c_double, C.c_void_p, C.c_int, _ip, _ip, _ip, _dp]),
        "or_amg_delete": (None, [P]),
        "or_amg_nlev": (C.c_int, [P]),
        "or_amg_level_sizes": (None, [P, C.c_int, _ip]),
        "or_amg_level_get": (None, [P, C.c_int, _ip, _ip, _dp, C.c_void_p, C.c_void_p, _ip, _ip, _dp, _dp]),
        "or_amg_apply": (None, [P, _dp, _dp]),
        "or_hash": (C.c_double, [C.c_uint64, C.c_int, C.c_int]),
        "or_potential_rank": (None, [C.c_int, _dp, _ip, _ip]),
        "or_splitmix64": (C.c_uint64, [C.c_uint64]),
        "or_forcing": (C.c_double, [C.c_int, C.c_double, C.c_double, C.c_double]),
        "or_reorth_count": (C.c_long, []),
    }
    for name, (res, args) in s.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib(omp: bool = False):
    """The oracle library; omp=True the OpenMP build (same results)."""
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            build(omp=True)
            _lib_omp = C.CDLL(_LIB_OMP)
            _sig(_lib_omp)
        return _lib_omp
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _sig(_lib)
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def omp_threads() -> int:
    """Threads the OpenMP build of the oracle runs its parallel loops on."""
    lib(omp=True)
    try:
        return int(C.CDLL("libgomp.so.1").omp_get_max_threads())
    except OSError:
        return os.cpu_count() or 1


def potential_order(key, idx=None):
    """Positions in descending-potential order (ties: lower idx first)."""
    key = np.ascontiguousarray(key, dtype=np.float64)
    idx = np.arange(len(key), dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    order = np.zeros(len(key), dtype=np.int32)
    lib().or_potential_rank(len(key), _d(key), _i(idx), _i(order))
    return order


def pm_mapping(key):
    """Pm of eq. (30): 1-based rank of each item in the descending sort."""
    order = potential_order(key)
    pm = np.empty(len(key), dtype=np.int64)
    pm[order] = np.arange(1, len(key) + 1)
    return pm


def interpolation(rp, ci, v, cf, theta=0.25, interp=0):
    """P of a scalar CSR matrix for a given C/F split (cf: 1 = C, -1 = F):
    direct (interp=0) or extended+i (interp=1).  Returns (prp, pci, pv)."""
    rp = np.ascontiguousarray(rp, np.int32); ci = np.ascontiguousarray(ci, np.int32)
    v = np.ascontiguousarray(v, np.float64); cf = np.ascontiguousarray(cf, np.int8)
    n = len(rp) - 1
    nnz = C.c_int()
    lib().or_interp_given(n, _i(rp), _i(ci), _d(v), theta, cf.ctypes.data, interp, C.byref(nnz), None, None, None)
    prp = np.zeros(n + 1, np.int32); pci = np.zeros(max(nnz.value, 1), np.int32); pv = np.zeros(max(nnz.value, 1))
    lib().or_interp_given(n, _i(rp), _i(ci), _d(v), theta, cf.ctypes.data, interp, C.byref(nnz), _i(prp), _i(pci),
                          _d(pv))
    return prp, pci[:nnz.value], pv[:nnz.value]


def forcing(l, bn, rprev, bprev):
    """eta_l of eq. (26), second choice, clamped to [0.01, 0.1]."""
    return lib().or_forcing(l, bn, rprev, bprev)


def pmis_hash(seed, level, i):
    return lib().or_hash(seed, level, i)


def splitmix64(x):
    return lib().or_splitmix64(x)


class AMG:
    """Standalone AMG hierarchy on a scalar CSR matrix."""

    def __init__(self, rp, ci, v, theta=0.25, seed=0x5EED, coarse_max=128, max_levels=25, interp=0, _handle=None,
                 _owner=None):
        self._lib = lib()
        if _handle is not None:
            self.h, self._own, self._owner = _handle, False, _owner
            return
        self._rp = np.ascontiguousarray(rp, dtype=np.int32)
        self._ci = np.ascontiguousarray(ci, dtype=np.int32)
        self._v = np.ascontiguousarray(v, dtype=np.float64)
        n = len(self._rp) - 1
        self.h = self._lib.or_amg_new(n, _i(self._rp), _i(self._ci), _d(self._v), theta, seed, coarse_max, max_levels,
                                      interp)
        self._own = True

    def __del__(self):
        if getattr(self, "_own", False) and self.h:
            self._lib.or_amg_delete(self.h)
            self.h = None

    @property
    def nlev(self):
        return self._lib.or_amg_nlev(self.h)

    def sizes(self, l):
        out = np.zeros(6, dtype=np.int32)
        self._lib.or_amg_level_sizes(self.h, l, _i(out))
        return dict(n=int(out[0]), nnz=int(out[1]), nnzP=int(out[2]), nc=int(out[3]), rounds=int(out[4]),
                    coarse_dense=int(out[5]))

    def level(self, l):
        s = self.sizes(l)
        n, nnz = s["n"], s["nnz"]
        rp = np.zeros(n + 1, np.int32); ci = np.zeros(max(nnz, 1), np.int32); v = np.zeros(max(nnz, 1))
        cf = np.zeros(max(n, 1), np.int8); st = np.zeros(max(nnz, 1), np.uint8)
        last = l == self.nlev - 1
        prp = np.zeros(n + 1, np.int32); pci = np.zeros(max(s["nnzP"], 1), np.int32); pv = np.zeros(max(s["nnzP"], 1))
        dl1 = np.zeros(max(n, 1))
        self._lib.or_amg_level_get(self.h, l, _i(rp), _i(ci), _d(v), cf.ctypes.data, st.ctypes.data,
                                   None if last else _i(prp), None if last else _i(pci), None if last else _d(pv), _d(dl1))
        out = dict(n=n, rp=rp, ci=ci[:nnz], v=v[:nnz], cf=cf[:n], strong=st[:nnz].astype(bool), dl1=dl1[:n],
                   rounds=s["rounds"])
        if not last:
            out.update(prp=prp, pci=pci[:s["nnzP"]], pv=pv[:s["nnzP"]], nc=s["nc"])
        return out

    def apply(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros_like(f)
        self._lib.or_amg_apply(self.h, _d(f), _d(x))
        return x


class LinearSystem:
    """A 2x2-block Newton system plus its CPR-FGMRES solver state."""

    def __init__(self, nx, ny, nz, nw, rp, ci, well_cell0, **opts):
        self._lib = lib()
        self._keep = [np.ascontiguousarray(rp, np.int32), np.ascontiguousarray(ci, np.int32),
                      np.ascontiguousarray(well_cell0 if nw else [0], np.int32)]
        self.opts = make_opts(**opts)
        self.h = self._lib.or_ls_create(nx, ny, nz, nw, _i(self._keep[0]), _i(self._keep[1]), _i(self._keep[2]),
                                        C.byref(self.opts))
        self._own = True
        self._fill_sizes()

    @classmethod
    def _wrap(cls, handle, owner, library=None):
        self = cls.__new__(cls)
        self._lib = library or lib(); self.h = handle; self._own = False; self._owner = owner
        self._fill_sizes()
        return self

    def _fill_sizes(self):
        out = np.zeros(5, np.int32)
        self._lib.or_ls_sizes(self.h, _i(out))
        self.n, self.nw, self.nb, self.nnzb, self.nsub = (int(x) for x in out)

    def __del__(self):
        if getattr(self, "_own", False) and self.h:
            self._lib.or_ls_destroy(self.h)
            self.h = None

    def set(self, val, b, key):
        val = np.ascontiguousarray(val, np.float64); b = np.ascontiguousarray(b, np.float64)
        key = np.ascontiguousarray(key, np.float64)
        self._lib.or_ls_set(self.h, _d(val), _d(b), _d(key))

    def set_opts(self, **kw):
        self.opts = make_opts(**kw)
        self._lib.or_ls_set_opts(self.h, C.byref(self.opts))

    def setup(self):
        rc = self._lib.or_ls_setup(self.h)
        self._fill_sizes()
        return rc

    def solve(self, tol):
        y = np.zeros(2 * self.nb); its = C.c_int(); rel = C.c_double()
        rc = self._lib.or_ls_solve(self.h, tol, _d(y), C.byref(its), C.byref(rel))
        return rc, y, its.value, rel.value

    def get(self):
        rp = np.zeros(self.nb + 1, np.int32); ci = np.zeros(self.nnzb, np.int32)
        val = np.zeros(4 * self.nnzb); b = np.zeros(2 * self.nb); key = np.zeros(max(self.n, 1))
        self._lib.or_ls_get(self.h, _i(rp), _i(ci), _d(val), _d(b), _d(key))
        return rp, ci, val, b, key[:self.n]

    def mv(self, x):
        x = np.ascontiguousarray(x, np.float64); y = np.zeros(2 * self.nb)
        self._lib.or_ls_mv(self.h, _d(x), _d(y)); return y

    def cpr(self, f):
        f = np.ascontiguousarray(f, np.float64); x = np.zeros(2 * self.nb)
        self._lib.or_ls_cpr(self.h, _d(f), _d(x)); return x

    def ras(self, f):
        f = np.ascontiguousarray(f, np.float64); x = np.zeros(2 * self.nb)
        self._lib.or_ls_ras(self.h, _d(f), _d(x)); return x

    def amg(self):
        return AMG(None, None, None, _handle=self._lib.or_ls_amg(self.h), _owner=self)

    def sub(self, s):
        if not 0 <= s < self.nsub:
            raise IndexError(f"subdomain {s} of {self.nsub}")
        out = np.zeros(3, np.int32)
        self._lib.or_ls_sub_sizes(self.h, s, _i(out))
        nown, next_, nnz = (int(x) for x in out)
        own = np.zeros(nown, np.int32); ext = np.zeros(next_, np.int32)
        rp = np.zeros(next_ + 1, np.int32); ci = np.zeros(max(nnz, 1), np.int32)
        lu = np.zeros(4 * max(nnz, 1)); dinv = np.zeros(4 * max(next_, 1))
        self._lib.or_ls_sub_get(self.h, s, _i(own), _i(ext), _i(rp), _i(ci), _d(lu), _d(dinv))
        return dict(own=own, ext=ext, rp=rp, ci=ci[:nnz], lu=lu[:4 * nnz], dinv=dinv[:4 * next_])


def _case_structs(case):
    g = Grid(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz, case.top)
    f = case.fluid
    keep = []
    pcs = np.ascontiguousarray(getattr(f, "pc_sw", ()) or [0.0], np.float64)
    pcv = np.ascontiguousarray(getattr(f, "pc", ()) or [0.0], np.float64)
    keep += [pcs, pcv]
    fl = Fluid((C.c_double * 2)(*f.rho_ref), (C.c_double * 2)(*f.c_f), (C.c_double * 2)(*f.mu_ref),
               (C.c_double * 2)(*f.c_mu), f.p_ref, f.c_r, f.swc, f.sor, f.nw, f.no, f.krw_max, f.kro_max, f.g,
               len(getattr(f, "pc", ()) or ()), _d(pcs), _d(pcv))
    wells = (Well * max(len(case.wells), 1))()
    for k, w in enumerate(case.wells):
        pc = np.ascontiguousarray(w.perf_cells, np.int32)
        keep.append(pc)
        wells[k] = Well(w.kind, w.control, w.target, w.r_w, w.skin, case.well_z_ref(w), len(pc), _i(pc), None,
                        getattr(w, "bhp_limit", 0.0) or 0.0)
    return g, fl, wells, keep


class Sim:
    """The oracle simulator for one Case."""

    def __init__(self, case, omp=False, **opts):
        self._lib = lib(omp)
        self.case = case
        o = dict(newton=0 if case.newton == "standard" else 1, newton_tol=case.newton_tol,
                 lin_tol=case.lin_tol, dt=case.dt, sat_chop=case.sat_chop)
        o.update(opts)
        self.opts = make_opts(**o)
        g, fl, wells, keep = _case_structs(case)
        self._keep = keep
        self._k = [np.ascontiguousarray(a, np.float64) for a in (case.kx, case.ky, case.kz, case.phi)]
        self.h = self._lib.or_sim_create(C.byref(g), *(_d(a) for a in self._k), C.byref(fl), wells,
                                         len(case.wells), C.byref(self.opts))
        self.n, self.nw = case.n, len(case.wells)
        self.ls = LinearSystem._wrap(self._lib.or_sim_lsys(self.h), self, self._lib)

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.or_sim_destroy(self.h)
            self.h = None

    def init_hydrostatic(self, p_datum=None, sw0=None):
        self._lib.or_sim_init_hydrostatic(self.h, self.case.p_init if p_datum is None else p_datum,
                                          self.case.sw_init if sw0 is None else sw0)

    def set_state(self, p, s, pb, t=0.0):
        p = np.ascontiguousarray(p, np.float64); s = np.ascontiguousarray(s, np.float64)
        pb = np.ascontiguousarray(pb if self.nw else [0.0], np.float64)
        self._lib.or_sim_set_state(self.h, _d(p), _d(s), _d(pb), t)

    def get_state(self):
        p = np.zeros(self.n); s = np.zeros(self.n); pb = np.zeros(max(self.nw, 1)); t = C.c_double()
        self._lib.or_sim_get_state(self.h, _d(p), _d(s), _d(pb), C.byref(t))
        return p, s, pb[:self.nw], t.value

    def store_old(self):
        self._lib.or_sim_store_old(self.h)

    def set_dt(self, dt):
        self._lib.or_sim_set_dt(self.h, dt)

    def assemble(self):
        self._lib.or_sim_assemble(self.h)

    def system(self):
        return self.ls.get()

    def residual_norm(self):
        return self._lib.or_sim_residual_norm(self.h)

    def newton(self):
        its = C.c_int()
        rc = self._lib.or_sim_newton(self.h, C.byref(its))
        return rc, its.value

    def advance(self, nsteps):
        return self._lib.or_sim_advance(self.h, nsteps)

    def linear_solve(self, tol):
        y = np.zeros(2 * (self.n + self.nw)); its = C.c_int(); rel = C.c_double()
        rc = self._lib.or_sim_linear_solve(self.h, tol, _d(y), C.byref(its), C.byref(rel))
        return rc, y, its.value, rel.value

    def stats(self):
        out = np.zeros(9)
        self._lib.or_sim_stats(self.h, _d(out))
        return dict(steps=int(out[0]), newton=int(out[1]), lin=int(out[2]), cuts=int(out[3]),
                    relres=out[4], its=int(out[5]), norm=out[6], t=out[7], switches=int(out[8]))

    def set_well(self, w, control, target, bhp_limit=0.0):
        """A schedule change: well w's control, target and BHP limit from now on."""
        if not 0 <= w < self.nw:
            raise IndexError(f"well {w} of {self.nw}")
        self._lib.or_sim_set_well(self.h, w, control, target, bhp_limit)

    def well_controls(self):
        """Current control and target of every well (after limit switching)."""
        c = np.zeros(max(self.nw, 1), np.int32); tg = np.zeros(max(self.nw, 1))
        self._lib.or_sim_well_controls(self.h, _i(c), _d(tg))
        return c[:self.nw], tg[:self.nw]

    def well_rates(self):
        qw = np.zeros(max(self.nw, 1)); qo = np.zeros(max(self.nw, 1))
        self._lib.or_sim_well_rates(self.h, _d(qw), _d(qo))
        return qw[:self.nw], qo[:self.nw]

    def mass(self):
        mw = C.c_double(); mo = C.c_double()
        self._lib.or_sim_mass(self.h, C.byref(mw), C.byref(mo))
        return mw.value, mo.value

    def well_index(self):
        npf = sum(len(w.perf_cells) for w in self.case.wells)
        wi = np.zeros(max(npf, 1))
        self._lib.or_sim_get_wi(self.h, _d(wi))
        return wi[:npf]
