"""FP64 CPU oracle of the symmetric MG-preconditioned SQMR Stokes solver (arXiv 2312.10615).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference leg may import this module; the product package never does.  The oracle is the plain
C file ``stokes_oracle.c`` next to this one (loops over single degrees of freedom, written from the
paper's Eq. 2, Alg. 1-4 and Sec. 5) plus this ctypes shim.  It shares no code with the CUDA path.

Every oracle function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_pins.py``
against something other than itself (Table 1 DOF counts, dense matrices built independently,
Thm 1-4 symmetry, MINRES equivalence, second-order manufactured-solution convergence).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stokes_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_ARG, ERR_OOM, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_UNSUPPORTED, ERR_SINGULAR = 0, -1, -2, -4, -5, -8, -9


def build(force=False):
    """Compile the oracle with gcc (plain -O2; OpenMP for the order-free loops, one thread by default)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None
_d = ctypes.POINTER(ctypes.c_double)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_l = ctypes.POINTER(ctypes.c_long)
_i = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    vp = ctypes.c_void_p
    sig = {
        "og_auto_levels": (ctypes.c_int, [ctypes.c_int] * 4),
        "og_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8,
                                     ctypes.POINTER(vp)]),
        "og_destroy": (None, [vp]),
        "og_nlevels": (ctypes.c_int, [vp]),
        "og_has_neumann": (ctypes.c_int, [vp]),
        "og_set_threads": (ctypes.c_int, [ctypes.c_int]),
        "og_level_n": (ctypes.c_long, [vp, ctypes.c_int]),
        "og_level_dims": (None, [vp, ctypes.c_int, _i]),
        "og_level_masks": (None, [vp, ctypes.c_int, _u8, _u8]),
        "og_level_order": (None, [vp, ctypes.c_int, _l, _l]),
        "og_count_dofs": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8, _l, _l]),
        "og_apply": (None, [vp, ctypes.c_int, ctypes.c_int, _d, _d]),
        "og_rhs": (None, [vp, _d, _d, _d]),
        "og_dgs": (None, [vp, ctypes.c_int, ctypes.c_int, _d, _d]),
        "og_vanka": (None, [vp, ctypes.c_int, ctypes.c_int, _d, _d]),
        "og_smooth_level": (None, [vp, ctypes.c_int, _d, _d]),
        "og_restrict_level": (None, [vp, ctypes.c_int, _d, _d]),
        "og_prolong_level": (None, [vp, ctypes.c_int, _d, _d]),
        "og_coarse": (None, [vp, _d, _d]),
        "og_dgs_diag": (None, [vp, ctypes.c_int, _d]),
        "og_vcycle": (None, [vp, _d, _d]),
        "og_set_variant": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "og_sqmr": (ctypes.c_int, [vp, _d, _d, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i,
                                   _d, _d]),
        "og_vcycle_x0": (None, [vp, _d, _d]),
        "og_mg_solve": (ctypes.c_int, [vp, _d, _d, ctypes.c_double, ctypes.c_int, _i, _d, _d]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_d)


def set_threads(n):
    """Threads of the oracle's order-free loops (operator rows, prolongation, one Vanka colour's patch
    corrections); results are bit-identical for every count.  Returns the count in effect."""
    return _load().og_set_threads(int(n))


def auto_levels(nx, ny, nz, coarsest_max=8):
    return _load().og_auto_levels(nx, ny, nz, coarsest_max)


def count_dofs(nx, ny, nz, labels=None):
    """(active DOFs, V1 DOFs) of an nx x ny x nz grid (Sec. 5; Table 1)."""
    lib = _load()
    na, nv = ctypes.c_long(), ctypes.c_long()
    lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8).ctypes.data_as(_u8)
    rc = lib.og_count_dofs(nx, ny, nz, lab, ctypes.byref(na), ctypes.byref(nv))
    if rc:
        raise RuntimeError(f"og_count_dofs failed: {rc}")
    return na.value, nv.value


class Oracle:
    """Multigrid hierarchy of the oracle (FP64)."""

    def __init__(self, nx, ny=None, nz=None, h=None, eta=1.0, gamma=1e-3, levels=0, coarsest_max=8, kb=1,
                 labels=None, additive=False, cycle=1, dwj=False):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        h = 1.0 / nx if h is None else h
        self.lib = _load()
        self._h = ctypes.c_void_p()
        self._lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8)
        lab = None if self._lab is None else self._lab.ctypes.data_as(_u8)
        rc = self.lib.og_create(nx, ny, nz, h, eta, gamma, levels, coarsest_max, kb, lab, ctypes.byref(self._h))
        if rc:
            raise RuntimeError(f"og_create failed: {rc}")
        rc = self.lib.og_set_variant(self._h, int(bool(additive)), int(cycle), int(bool(dwj)))
        if rc:
            raise RuntimeError(f"og_set_variant failed: {rc}")
        self.dims, self.h, self.eta, self.gamma, self.kb = (nx, ny, nz), h, eta, gamma, kb
        self.nlevels = self.lib.og_nlevels(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.og_destroy(self._h)
            self._h = ctypes.c_void_p()

    # -- sizes / classification ----------------------------------------------------------
    def has_neumann(self):
        """True when some unknown face borders an exterior cell (Sec. 5): no pressure null space."""
        return bool(self.lib.og_has_neumann(self._h))

    def n(self, level=0):
        return self.lib.og_level_n(self._h, level)

    def level_dims(self, level):
        d = (ctypes.c_int * 3)()
        self.lib.og_level_dims(self._h, level, d)
        return tuple(d)

    def masks(self, level=0):
        n = self.n(level)
        a, v = np.zeros(n, np.uint8), np.zeros(n, np.uint8)
        self.lib.og_level_masks(self._h, level, a.ctypes.data_as(_u8), v.ctypes.data_as(_u8))
        return a.astype(bool), v.astype(bool)

    def dgs_order(self, level=0):
        n = self.n(level)
        o, m = np.zeros(n + 1, np.int64), ctypes.c_long()
        self.lib.og_level_order(self._h, level, o.ctypes.data_as(_l), ctypes.byref(m))
        return o[: m.value].copy()

    def dgs_diag(self, level=0):
        d = np.zeros(self.n(level))
        self.lib.og_dgs_diag(self._h, level, _dp(d))
        return d

    # -- operators -------------------------------------------------------------------------
    def apply(self, x, level=0, penalised=False):
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros(self.n(level))
        self.lib.og_apply(self._h, level, int(penalised), _dp(x), _dp(y))
        return y

    def rhs(self, f=None, g=None):
        b = np.zeros(self.n(0))
        fp = None if f is None else _dp(np.ascontiguousarray(f, np.float64))
        gp = None if g is None else _dp(np.ascontiguousarray(g, np.float64))
        self.lib.og_rhs(self._h, fp, gp, _dp(b))
        return b

    def dgs(self, x, b, level=0, direction=0):
        x = np.array(x, np.float64, copy=True)
        self.lib.og_dgs(self._h, level, direction, _dp(x), _dp(np.ascontiguousarray(b, np.float64)))
        return x

    def vanka(self, x, b, level=0, colour=-1):
        x = np.array(x, np.float64, copy=True)
        self.lib.og_vanka(self._h, level, colour, _dp(x), _dp(np.ascontiguousarray(b, np.float64)))
        return x

    def smooth(self, x, b, level=0):
        x = np.array(x, np.float64, copy=True)
        self.lib.og_smooth_level(self._h, level, _dp(x), _dp(np.ascontiguousarray(b, np.float64)))
        return x

    def restrict(self, r, level=0):
        bc = np.zeros(self.n(level + 1))
        self.lib.og_restrict_level(self._h, level, _dp(np.ascontiguousarray(r, np.float64)), _dp(bc))
        return bc

    def prolong_add(self, e, x, level=0):
        x = np.array(x, np.float64, copy=True)
        self.lib.og_prolong_level(self._h, level, _dp(np.ascontiguousarray(e, np.float64)), _dp(x))
        return x

    def coarse_solve(self, b):
        x = np.zeros(self.n(self.nlevels - 1))
        self.lib.og_coarse(self._h, _dp(np.ascontiguousarray(b, np.float64)), _dp(x))
        return x

    def vcycle(self, s):
        t = np.zeros(self.n(0))
        self.lib.og_vcycle(self._h, _dp(np.ascontiguousarray(s, np.float64)), _dp(t))
        return t

    def vcycle_x0(self, b, x0):
        """One V-cycle of Alg. 1 on L~ from the initial guess x0 (not zero)."""
        x = np.array(x0, np.float64, copy=True)
        self.lib.og_vcycle_x0(self._h, _dp(np.ascontiguousarray(b, np.float64)), _dp(x))
        return x

    def mg_solve(self, b, x0=None, tol=1e-8, maxit=200):
        """Alg. 1 iterated as a solver on L~ x = b.  Returns (x, status, cycles, relative L~ residual, history)."""
        x = np.zeros(self.n(0)) if x0 is None else np.array(x0, np.float64, copy=True)
        hist = np.zeros(maxit + 1)
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = self.lib.og_mg_solve(self._h, _dp(np.ascontiguousarray(b, np.float64)), _dp(x), tol, maxit,
                                  ctypes.byref(it), ctypes.byref(rr), _dp(hist))
        return x, rc, it.value, rr.value, hist[: it.value + 1].copy()

    def sqmr(self, b, x0=None, tol=1e-8, maxit=200, precond=True, fixed_iters=0):
        """Alg. 4.  Returns (x, status, iterations, true relative residual, history)."""
        x = np.zeros(self.n(0)) if x0 is None else np.array(x0, np.float64, copy=True)
        hist = np.zeros(maxit + 2)
        it, rr = ctypes.c_int(), ctypes.c_double()
        rc = self.lib.og_sqmr(self._h, _dp(np.ascontiguousarray(b, np.float64)), _dp(x), tol, maxit, int(precond),
                              fixed_iters, ctypes.byref(it), ctypes.byref(rr), _dp(hist))
        return x, rc, it.value, rr.value, hist[: it.value + 1].copy()
