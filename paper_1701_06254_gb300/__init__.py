"""Python binding of libresim.so, the sm_103a CPR-FGMRES reservoir solver.

Thin ctypes marshalling over the C ABI declared in include/resim.h: every
step of the Newton / linear-solve path runs in the library's CUDA kernels.
Arrays may be numpy arrays (host) or CUDA tensors (device); the library
accepts either.  Importing this package does not load the library; the
first call does, and raises if the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs  # noqa: F401  (synthetic workloads)

_lib = None

PREC_FP64, PREC_MIXED, PREC_MIXED_BF16 = 0, 1, 2
KRYLOV_FGMRES, KRYLOV_BICGSTAB = 0, 1
INTERP_DIRECT, INTERP_EXTI = 0, 1
DEC_NONE, DEC_ABF, DEC_QI = 0, 1, 2
OP_SPMV, OP_RAS, OP_VCYCLE, OP_CPR = 0, 1, 2, 3
T_NONE, T_SPMV64, T_SPMV_PREC, T_RAS, T_VCYCLE, T_ORTHO, T_ASSEMBLE = 0, 1, 2, 3, 4, 5, 6
T_AMG_SETUP, T_RAS_SETUP, T_DECOUPLE, T_WARMSTART, T_NETWORK, T_NFAMILIES = 7, 8, 9, 10, 11, 12
T_NAMES = {1: "spmv64", 2: "spmv_prec", 3: "ras_apply", 4: "vcycle", 5: "ortho", 6: "assemble",
           7: "amg_setup", 8: "ras_setup", 9: "decouple", 10: "warm_start", 11: "network"}
X_VALS, X_RHS, X_SOLUTION, X_ROWPTR, X_COLS, X_KEY = 0, 1, 2, 3, 4, 5
X_AMG_SIZES, X_AMG_RP, X_AMG_CI, X_AMG_V, X_AMG_CF, X_AMG_PRP, X_AMG_PCI, X_AMG_PV = 10, 11, 12, 13, 14, 15, 16, 17
X_RAS_SIZES, X_RAS_EXT, X_RAS_LEVELS = 20, 21, 22
STATUS = {0: "SIM_OK", 1: "SIM_ERR_ARG", 2: "SIM_ERR_CUDA", 3: "SIM_ERR_OOM", 4: "SIM_ERR_NOT_CONVERGED",
          5: "SIM_ERR_NAN", 6: "SIM_ERR_TIMEOUT", 7: "SIM_ERR_STATE"}


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dz", C.c_double), ("top_depth", C.c_double)]


class Rock(C.Structure):
    _fields_ = [("kx", C.c_void_p), ("ky", C.c_void_p), ("kz", C.c_void_p), ("phi", C.c_void_p)]


class Fluid(C.Structure):
    _fields_ = [("rho_ref", C.c_double * 2), ("c_f", C.c_double * 2), ("mu_ref", C.c_double * 2),
                ("c_mu", C.c_double * 2), ("p_ref", C.c_double), ("c_r", C.c_double), ("swc", C.c_double),
                ("sor", C.c_double), ("nw", C.c_double), ("no", C.c_double), ("krw_max", C.c_double),
                ("kro_max", C.c_double), ("g", C.c_double), ("pc_n", C.c_int), ("pc_sw", C.c_void_p),
                ("pc_val", C.c_void_p)]


class Well(C.Structure):
    _fields_ = [("kind", C.c_int), ("control", C.c_int), ("target", C.c_double), ("r_w", C.c_double),
                ("skin", C.c_double), ("z_ref", C.c_double), ("n_perf", C.c_int),
                ("perf_cell", C.POINTER(C.c_int)), ("wi", C.POINTER(C.c_double)), ("bhp_limit", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("decoupling", C.c_int), ("reorder", C.c_int), ("newton", C.c_int),
                ("newton_tol", C.c_double), ("lin_tol", C.c_double), ("max_newton", C.c_int),
                ("restart", C.c_int), ("max_lin", C.c_int), ("tile_x", C.c_int), ("tile_y", C.c_int),
                ("amg_theta", C.c_double), ("amg_max_levels", C.c_int), ("amg_coarse_max", C.c_int),
                ("seed", C.c_uint64), ("max_cuts", C.c_int), ("dt", C.c_double), ("cuda_stream", C.c_void_p),
                ("sat_chop", C.c_double), ("krylov", C.c_int), ("overlap", C.c_int), ("interp", C.c_int),
                ("fp64_basis", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("newton", C.c_longlong), ("linear_its", C.c_longlong),
                ("cuts", C.c_longlong), ("linear_solves", C.c_longlong), ("last_relres", C.c_double),
                ("last_norm", C.c_double), ("t", C.c_double), ("last_its", C.c_int), ("last_newton", C.c_int),
                ("ms_assemble", C.c_double), ("ms_setup", C.c_double), ("ms_solve", C.c_double),
                ("ws_used", C.c_longlong), ("ws_fallback", C.c_longlong), ("ws_r0", C.c_double),
                ("switches", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libresim.so")


def build(force=False):
    from . import _build
    return _build.build(force=force)


def lib():
    """Load libresim.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        sig = {
            "sim_default_options": (None, [C.POINTER(Options)]),
            "sim_create": (I, [C.POINTER(P), C.POINTER(Grid), C.POINTER(Rock), C.POINTER(Fluid), C.POINTER(Well), I,
                               C.POINTER(Options)]),
            "sim_destroy": (None, [P]),
            "sim_init_hydrostatic": (I, [P, D, D]),
            "sim_set_state": (I, [P, P, P, P, D]),
            "sim_get_state": (I, [P, P, P, P, C.POINTER(D)]),
            "sim_begin_step": (I, [P, D]),
            "sim_assemble": (I, [P, C.POINTER(D)]),
            "sim_linear_solve": (I, [P, D, C.POINTER(I), C.POINTER(D)]),
            "sim_newton_step": (I, [P, C.POINTER(I), C.POINTER(Stats)]),
            "sim_advance": (I, [P, I, C.POINTER(Stats)]),
            "sim_get_stats": (I, [P, C.POINTER(Stats)]),
            "sim_set_well": (I, [P, I, I, D, D]),
            "sim_get_well_controls": (I, [P, P, P]),
            "sim_linear_system": (P, [P]),
            "sim_ls_create": (I, [C.POINTER(P), I, I, I, I, P, P, P, C.POINTER(Options)]),
            "sim_ls_destroy": (None, [P]),
            "sim_ls_set": (I, [P, P, P, P]),
            "sim_ls_setup": (I, [P]),
            "sim_ls_solve": (I, [P, D, P, C.POINTER(I), C.POINTER(D)]),
            "sim_ls_apply": (I, [P, I, P, P]),
            "sim_ls_export": (I, [P, I, I, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "sim_ls_residual_norm": (I, [P, P, C.POINTER(D)]),
            "sim_ls_residual_norm_noalloc": (I, [P, P, P]),
            "sim_kernel_timer": (I, [P, C.c_uint]),
            "sim_ls_step_graph": (I, [P, C.c_int]),
            "sim_ls_graph_mode": (I, [P, C.POINTER(C.c_int)]),
            "sim_kernel_time": (I, [P, I, C.POINTER(C.c_longlong), C.POINTER(D)]),
            "sim_batch_create": (I, [C.POINTER(P), I, C.POINTER(Grid), C.POINTER(Rock), C.POINTER(Fluid),
                                     C.POINTER(C.POINTER(Well)), C.POINTER(I), C.POINTER(Options), I]),
            "sim_batch_destroy": (None, [P]),
            "sim_batch_member": (I, [P, I, C.POINTER(P)]),
            "sim_batch_size": (I, [P, C.POINTER(I), C.POINTER(I)]),
            "sim_batch_advance": (I, [P, I, C.POINTER(Stats), C.POINTER(I)]),
            "sim_batch_autotune": (I, [P, C.POINTER(I), I, I, C.POINTER(I), C.POINTER(D)]),
            "sim_ws_create": (I, [C.POINTER(P), C.c_uint64]),
            "sim_ws_destroy": (None, [P]),
            "sim_ws_use_tcgen05": (I, [P, I]),
            "sim_ws_params": (I, [P, I, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "sim_ws_set_params": (I, [P, P, C.c_size_t]),
            "sim_ws_forward": (I, [P, I, I, I, P, P]),
            "sim_ws_backward": (I, [P, I, I, I, P, P, C.POINTER(D)]),
            "sim_ws_zero_grad": (I, [P]),
            "sim_ws_adam": (I, [P, D]),
            "sim_ws_record": (I, [P, P]),
            "sim_ws_dataset": (I, [P, C.POINTER(I)]),
            "sim_ws_train": (I, [P, I, I, D, C.c_uint64, C.POINTER(D)]),
            "sim_ws_eval": (I, [P, C.POINTER(D)]),
            "sim_ws_attach": (I, [P, P]),
            "sim_launch_count": (C.c_longlong, []),
            "sim_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise SimError(rc, lib().sim_last_error().decode(errors="replace"))


def _ptr(a):
    """Raw address of a numpy array or a CUDA tensor (anything with data_ptr)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _vec(a, n, name, dtype=np.float64, out=False, at_least=False):
    """a as a buffer of n values of dtype for a C call: a numpy array (an
    input is converted to a contiguous copy of that type; an output must
    already be one) or a contiguous tensor with that element type.  A wrong
    count, type or layout raises ValueError here instead of letting the
    library read or write past the caller's buffer."""
    dt = np.dtype(dtype)
    if hasattr(a, "data_ptr"):
        ok = (a.is_contiguous() and a.element_size() == dt.itemsize
              and bool(a.is_floating_point()) == bool(np.issubdtype(dt, np.floating)))
        cnt = a.numel()
    else:
        if out:
            ok = isinstance(a, np.ndarray) and a.dtype == dt and a.flags.c_contiguous and a.flags.writeable
        else:
            a = np.ascontiguousarray(a, dt)
            ok = True
        cnt = a.size if ok else 0
    if not ok:
        raise ValueError(f"{name}: expected a contiguous, writable buffer of {dt.name} values" if out else
                         f"{name}: expected a contiguous buffer of {dt.name} values")
    if (cnt < n) if at_least else (cnt != n):
        raise ValueError(f"{name}: expected {'at least ' if at_least else ''}{n} values, got {cnt}")
    return a


def launch_count():
    return lib().sim_launch_count()


OPT_KEYS = ("precision", "decoupling", "reorder", "newton", "newton_tol", "lin_tol", "max_newton", "restart",
            "max_lin", "tile_x", "tile_y", "amg_theta", "amg_max_levels", "amg_coarse_max", "seed", "max_cuts", "dt",
            "sat_chop", "krylov", "overlap", "interp", "fp64_basis")


def make_options(stream=None, **kw):
    o = Options()
    lib().sim_default_options(C.byref(o))
    for k, v in kw.items():
        if k not in OPT_KEYS:
            raise KeyError(k)
        setattr(o, k, v)
    o.cuda_stream = stream
    return o


class LinearSystem:
    """A 2x2-block Newton system with its CPR-FGMRES solver (sim_ls_*)."""

    def __init__(self, nx=None, ny=None, nz=None, nw=0, rp=None, ci=None, well_cell0=None, stream=None,
                 _handle=None, _owner=None, **opts):
        self._L = lib()
        if _handle is not None:
            self.h, self._own, self._owner = _handle, False, _owner
        else:
            rp = np.ascontiguousarray(rp, np.int32); ci = np.ascontiguousarray(ci, np.int32)
            wc = np.ascontiguousarray(well_cell0 if nw else [0], np.int32)
            self.opts = make_options(stream, **opts)
            h = C.c_void_p()
            _check(self._L.sim_ls_create(C.byref(h), nx, ny, nz, nw, _ptr(rp), _ptr(ci), _ptr(wc), C.byref(self.opts)))
            self.h, self._own = h, True
            self.n, self.nw, self.nb, self.nnzb = nx * ny * nz, nw, nx * ny * nz + nw, int(rp[-1])

    def __del__(self):
        if getattr(self, "_own", False) and self.h:
            self._L.sim_ls_destroy(self.h)
            self.h = None

    def set(self, val, b, key):
        nnzb = getattr(self, "nnzb", None)
        val = _vec(val, 4 * nnzb, "val") if nnzb is not None else _vec(val, 0, "val", at_least=True)
        b = _vec(b, 2 * self.nb, "b")
        key = _vec(key, self.n, "key")
        _check(self._L.sim_ls_set(self.h, _ptr(val), _ptr(b), _ptr(key)))

    def setup(self):
        _check(self._L.sim_ls_setup(self.h))

    def solve(self, tol, y=None):
        nb = self._nb()
        out = np.zeros(2 * nb) if y is None else _vec(y, 2 * nb, "y", out=True)
        its, rel = C.c_int(), C.c_double()
        _check(self._L.sim_ls_solve(self.h, tol, _ptr(out), C.byref(its), C.byref(rel)))
        return out, its.value, rel.value

    def apply(self, op, x):
        x = np.ascontiguousarray(x, np.float64)
        if op in (OP_SPMV, OP_RAS, OP_CPR, OP_VCYCLE):         # an unknown op is the library's to reject
            x = _vec(x, self.n if op == OP_VCYCLE else 2 * self.nb, "x")
        y = np.zeros_like(x)
        _check(self._L.sim_ls_apply(self.h, op, _ptr(x), _ptr(y)))
        return y

    def residual_norm(self, x):
        """||b - A x||_2 of the current (decoupled after setup) system."""
        x = _vec(x, 2 * self.nb, "x")
        nrm = C.c_double()
        _check(self._L.sim_ls_residual_norm(self.h, _ptr(x), C.byref(nrm)))
        return nrm.value

    def residual_norm_noalloc(self, x_dev, norm_dev):
        """Same norm without allocating: x_dev and norm_dev are CUDA tensors;
        the result is written to norm_dev on the library stream."""
        _check(self._L.sim_ls_residual_norm_noalloc(self.h, _ptr(x_dev), _ptr(norm_dev)))

    def export(self, what, index=0, dtype=np.float64):
        need = C.c_size_t()
        _check(self._L.sim_ls_export(self.h, what, index, None, 0, C.byref(need)))
        out = np.zeros(need.value // np.dtype(dtype).itemsize, dtype)
        if need.value:
            _check(self._L.sim_ls_export(self.h, what, index, _ptr(out), need.value, C.byref(need)))
        return out

    def _nb(self):
        return len(self.export(X_RHS)) // 2

    def amg_nlev(self):
        return int(self.export(X_AMG_SIZES, -1, np.int32)[0])

    def amg_level(self, l):
        sz = self.export(X_AMG_SIZES, l, np.int32)
        d = dict(n=int(sz[0]), nnz=int(sz[1]), nnzP=int(sz[2]), nc=int(sz[3]), rounds=int(sz[4]),
                 coarse_dense=int(sz[5]))
        d["rp"] = self.export(X_AMG_RP, l, np.int32)
        d["ci"] = self.export(X_AMG_CI, l, np.int32)
        d["v"] = self.export(X_AMG_V, l, np.float64)
        d["cf"] = self.export(X_AMG_CF, l, np.int8)
        if l < self.amg_nlev() - 1:
            d["prp"] = self.export(X_AMG_PRP, l, np.int32)
            d["pci"] = self.export(X_AMG_PCI, l, np.int32)
            d["pv"] = self.export(X_AMG_PV, l, np.float64)
        return d

    def ras_count(self):
        return int(self.export(X_RAS_SIZES, -1, np.int32)[0])

    def ras_ext(self, s):
        return self.export(X_RAS_EXT, s, np.int32)

    def ras_levels(self, s):
        v = self.export(X_RAS_LEVELS, s, np.int32)
        return int(v[0]), int(v[1]), v[2::2].copy(), v[3::2].copy()

    def ras_sizes(self, s):
        v = self.export(X_RAS_SIZES, s, np.int32)
        return int(v[0]), int(v[1]), int(v[2])

    def kernel_timer(self, families):
        """Enable CUDA-event timing for the given T_* families (iterable)."""
        mask = 0
        for f in families:
            mask |= 1 << f
        _check(self._L.sim_kernel_timer(self.h, mask))

    def step_graph(self, mode):
        """Launch mode of the Arnoldi steps: 2 a whole restart cycle from
        one graph launch with a device-side WHILE node, 1 (or True, the
        default) one graph replay per step, 0 (or False) separate kernel
        launches; same results in all three."""
        mode = 1 if mode is True else 0 if mode is False else int(mode)
        _check(self._L.sim_ls_step_graph(self.h, mode))

    def graph_mode(self):
        """The launch mode the last FGMRES solve used (-1 before any)."""
        m = C.c_int()
        _check(self._L.sim_ls_graph_mode(self.h, C.byref(m)))
        return m.value

    def kernel_time(self, which):
        n, ms = C.c_longlong(), C.c_double()
        _check(self._L.sim_kernel_time(self.h, which, C.byref(n), C.byref(ms)))
        return n.value, ms.value


def _case_structs(case):
    g = Grid(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz, case.top)
    f = case.fluid
    keep = []
    pcs = np.ascontiguousarray(getattr(f, "pc_sw", ()) or [0.0], np.float64)
    pcv = np.ascontiguousarray(getattr(f, "pc", ()) or [0.0], np.float64)
    keep += [pcs, pcv]
    fl = Fluid((C.c_double * 2)(*f.rho_ref), (C.c_double * 2)(*f.c_f), (C.c_double * 2)(*f.mu_ref),
               (C.c_double * 2)(*f.c_mu), f.p_ref, f.c_r, f.swc, f.sor, f.nw, f.no, f.krw_max, f.kro_max, f.g,
               len(getattr(f, "pc", ()) or ()), _ptr(pcs), _ptr(pcv))
    wells = (Well * max(len(case.wells), 1))()
    for k, w in enumerate(case.wells):
        pc = np.ascontiguousarray(w.perf_cells, np.int32)
        keep.append(pc)
        wells[k] = Well(w.kind, w.control, w.target, w.r_w, w.skin, case.well_z_ref(w), len(pc),
                        pc.ctypes.data_as(C.POINTER(C.c_int)), None, getattr(w, "bhp_limit", 0.0) or 0.0)
    return g, fl, wells, keep


class Sim:
    """GPU simulator for one inputs.Case (sim_* entry points)."""

    def __init__(self, case, stream=None, **opts):
        self._L = lib()
        self.case = case
        o = dict(newton=0 if case.newton == "standard" else 1, newton_tol=case.newton_tol, lin_tol=case.lin_tol,
                 dt=case.dt, sat_chop=case.sat_chop)
        o.update(opts)
        self.opts = make_options(stream, **o)
        g, fl, wells, keep = _case_structs(case)
        self._k = [np.ascontiguousarray(a, np.float64) for a in (case.kx, case.ky, case.kz, case.phi)]
        rock = Rock(*(_ptr(a) for a in self._k))
        h = C.c_void_p()
        _check(self._L.sim_create(C.byref(h), C.byref(g), C.byref(rock), C.byref(fl), wells, len(case.wells),
                                  C.byref(self.opts)))
        self.h = h
        self.n, self.nw = case.n, len(case.wells)
        self.ls = LinearSystem(_handle=self._L.sim_linear_system(h), _owner=self)
        self.ls.n, self.ls.nw, self.ls.nb = self.n, self.nw, self.n + self.nw

    def __del__(self):
        if getattr(self, "h", None):
            self._L.sim_destroy(self.h)
            self.h = None

    def init_hydrostatic(self, p_datum=None, sw0=None):
        _check(self._L.sim_init_hydrostatic(self.h, self.case.p_init if p_datum is None else p_datum,
                                            self.case.sw_init if sw0 is None else sw0))

    def set_state(self, p, sw, pb, t=0.0):
        p, sw = _vec(p, self.n, "p"), _vec(sw, self.n, "sw")
        pb = _vec(pb, self.nw, "pb", at_least=True) if self.nw else np.zeros(1)
        _check(self._L.sim_set_state(self.h, _ptr(p), _ptr(sw), _ptr(pb), t))

    def get_state(self, out=None):
        if out is None:
            p, sw, pb = np.zeros(self.n), np.zeros(self.n), np.zeros(max(self.nw, 1))
        else:
            p, sw = _vec(out[0], self.n, "p", out=True), _vec(out[1], self.n, "sw", out=True)
            pb = _vec(out[2], self.nw, "pb", out=True, at_least=True)
        t = C.c_double()
        _check(self._L.sim_get_state(self.h, _ptr(p), _ptr(sw), _ptr(pb), C.byref(t)))
        return p, sw, pb[:self.nw] if out is None else pb, t.value

    def begin_step(self, dt):
        _check(self._L.sim_begin_step(self.h, dt))

    def assemble(self):
        nr = C.c_double()
        _check(self._L.sim_assemble(self.h, C.byref(nr)))
        return nr.value

    def linear_solve(self, tol):
        its, rel = C.c_int(), C.c_double()
        _check(self._L.sim_linear_solve(self.h, tol, C.byref(its), C.byref(rel)))
        return its.value, rel.value

    def newton_step(self):
        conv, st = C.c_int(), Stats()
        _check(self._L.sim_newton_step(self.h, C.byref(conv), C.byref(st)))
        return bool(conv.value), st.as_dict()

    def advance(self, n_steps):
        st = Stats()
        _check(self._L.sim_advance(self.h, n_steps, C.byref(st)))
        return st.as_dict()

    def stats(self):
        st = Stats()
        _check(self._L.sim_get_stats(self.h, C.byref(st)))
        return st.as_dict()

    def set_well(self, w, control, target, bhp_limit=0.0):
        """A schedule change: well w's control, target and BHP limit from now on."""
        if not 0 <= w < self.nw:
            raise IndexError(f"well {w} of {self.nw}")
        _check(self._L.sim_set_well(self.h, w, control, target, bhp_limit))

    def well_controls(self):
        """Current control and target of every well (after limit switching)."""
        c = np.zeros(max(self.nw, 1), np.int32); tg = np.zeros(max(self.nw, 1))
        _check(self._L.sim_get_well_controls(self.h, _ptr(c), _ptr(tg)))
        return c[:self.nw], tg[:self.nw]

    def attach_warm_start(self, ws):
        """Use a WarmStart network for the initial guess of every solve (None detaches)."""
        self._ws = ws
        _check(self._L.sim_ws_attach(self.h, ws.h if ws is not None else None))

    def record_to(self, ws):
        """Append every solve's (features, update) pair to ws's dataset (None stops)."""
        self._rec = ws
        _check(self._L.sim_ws_record(self.h, ws.h if ws is not None else None))


class _Member(Sim):
    """A batch member: the single-model calls on a handle the batch owns."""

    def __init__(self, batch, k, case, h):
        self._L = batch._L
        self.case = case
        self.h = h
        self._owned = False
        self.n, self.nw = case.n, len(case.wells)
        self.ls = LinearSystem(_handle=self._L.sim_linear_system(h), _owner=self)
        self.ls.n, self.ls.nw, self.ls.nb = self.n, self.nw, self.n + self.nw
        self._batch = batch                    # keeps the batch (and so the handle) alive

    def __del__(self):
        pass


class Batch:
    """An ensemble of independent models advanced together on one GPU
    (sim_batch_* entry points).  cases: a list of inputs.Case; options are
    taken from each case as Sim does, plus the keyword overrides."""

    def __init__(self, cases, workers=0, **opts):
        self._L = lib()
        self.cases = list(cases)
        m = len(self.cases)
        grids, rocks, fluids = (Grid * m)(), (Rock * m)(), (Fluid * m)()
        wptr = (C.POINTER(Well) * m)()
        nwell = (C.c_int * m)()
        ops = (Options * m)()
        self._keep = []
        for k, case in enumerate(self.cases):
            o = dict(newton=0 if case.newton == "standard" else 1, newton_tol=case.newton_tol,
                     lin_tol=case.lin_tol, dt=case.dt, sat_chop=case.sat_chop)
            o.update(opts)
            ops[k] = make_options(None, **o)
            g, fl, wells, keep = _case_structs(case)
            arrs = [np.ascontiguousarray(a, np.float64) for a in (case.kx, case.ky, case.kz, case.phi)]
            grids[k], fluids[k] = g, fl
            rocks[k] = Rock(*(_ptr(a) for a in arrs))
            wptr[k] = C.cast(wells, C.POINTER(Well))
            nwell[k] = len(case.wells)
            self._keep += [wells, keep, arrs]
        h = C.c_void_p()
        _check(self._L.sim_batch_create(C.byref(h), m, grids, rocks, fluids, wptr, nwell, ops, workers))
        self.h = h
        self._keep = None                      # everything was copied at creation
        self.members = []
        for k, case in enumerate(self.cases):
            mh = C.c_void_p()
            _check(self._L.sim_batch_member(h, k, C.byref(mh)))
            self.members.append(_Member(self, k, case, mh))

    def __del__(self):
        if getattr(self, "h", None):
            self.members = []
            self._L.sim_batch_destroy(self.h)
            self.h = None

    def __len__(self):
        return len(self.cases)

    @property
    def workers(self):
        w = C.c_int()
        _check(self._L.sim_batch_size(self.h, None, C.byref(w)))
        return w.value

    def init_hydrostatic(self):
        for mem in self.members:
            mem.init_hydrostatic()

    def advance(self, n_steps):
        m = len(self.cases)
        st = (Stats * m)()
        rc = (C.c_int * m)()
        _check(self._L.sim_batch_advance(self.h, n_steps, st, rc))
        return [s.as_dict() for s in st]

    def autotune(self, candidates=(2, 4, 8, 16), sample=0):
        c = (C.c_int * len(candidates))(*candidates)
        sec = (C.c_double * len(candidates))()
        chosen = C.c_int()
        _check(self._L.sim_batch_autotune(self.h, c, len(candidates), sample, C.byref(chosen), sec))
        return chosen.value, dict(zip(candidates, list(sec)))


class WarmStart:
    """The learned warm start's network (sim_ws_* entry points)."""

    def __init__(self, seed=0):
        self._L = lib()
        h = C.c_void_p()
        _check(self._L.sim_ws_create(C.byref(h), seed))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            self._L.sim_ws_destroy(self.h)
            self.h = None

    def params(self, which=0):
        """Flat FP32 vector: per layer W[27][Co][Ci] then b[Co] (which=1: mean gradients)."""
        n = C.c_size_t()
        _check(self._L.sim_ws_params(self.h, which, None, 0, C.byref(n)))
        out = np.zeros(n.value, np.float32)
        _check(self._L.sim_ws_params(self.h, which, _ptr(out), n.value, None))
        return out

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, np.float32)
        _check(self._L.sim_ws_set_params(self.h, _ptr(a), a.size))

    @staticmethod
    def _grid(a, name):
        a = np.ascontiguousarray(a, np.float32)
        if a.ndim != 4 or a.shape[3] != 8 or min(a.shape[:3]) < 1:
            raise ValueError(f"{name}: expected shape (nz, ny, nx, 8), got {a.shape}")
        return a

    def forward(self, feat):
        """feat (nz, ny, nx, 8) -> output (nz, ny, nx, 8), FP32."""
        f = self._grid(feat, "feat")
        nz, ny, nx = f.shape[:3]
        y = np.zeros((nz, ny, nx, 8), np.float32)
        _check(self._L.sim_ws_forward(self.h, nx, ny, nz, _ptr(f), _ptr(y)))
        return y

    def backward(self, feat, target):
        """Forward + loss + backward for one sample (feat (nz, ny, nx, 8),
        target (nz, ny, nx, 2)); gradients accumulate."""
        f = self._grid(feat, "feat")
        t = np.ascontiguousarray(target, np.float32)
        if t.shape != f.shape[:3] + (2,):
            raise ValueError(f"target: expected shape {f.shape[:3] + (2,)}, got {t.shape}")
        nz, ny, nx = f.shape[:3]
        loss = C.c_double()
        _check(self._L.sim_ws_backward(self.h, nx, ny, nz, _ptr(f), _ptr(t), C.byref(loss)))
        return loss.value

    def zero_grad(self):
        _check(self._L.sim_ws_zero_grad(self.h))

    def use_tcgen05(self, on=True):
        """tcgen05 or mma.sync (default) kernels for the forward / data-gradient convolutions."""
        _check(self._L.sim_ws_use_tcgen05(self.h, 1 if on else 0))

    def adam(self, lr):
        _check(self._L.sim_ws_adam(self.h, lr))

    def dataset_size(self):
        n = C.c_int()
        _check(self._L.sim_ws_dataset(self.h, C.byref(n)))
        return n.value

    def train(self, epochs, batch=4, lr=1e-3, seed=0):
        loss = C.c_double()
        _check(self._L.sim_ws_train(self.h, epochs, batch, lr, seed, C.byref(loss)))
        return loss.value

    def eval(self):
        loss = C.c_double()
        _check(self._L.sim_ws_eval(self.h, C.byref(loss)))
        return loss.value
