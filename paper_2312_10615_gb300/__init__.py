"""Python binding of libstokesmg -- the GB300 symmetric multigrid-preconditioned SQMR solver for the
3D MAC Stokes system (Tao & Sifakis, arXiv 2312.10615).

Argument marshalling only: every numerical step runs in the library's CUDA kernels.  Functions carry
the C-ABI names of ``include/stokesmg.h``; vectors may be torch tensors (CUDA or CPU, float64,
contiguous) or numpy float64 arrays.  ``Stokes`` wraps a handle for convenience.

If the native library is missing, the first call raises ImportError: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstokesmg.so")

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_NAN, ERR_TIMEOUT, ERR_UNSUPPORTED = \
    -1, -2, -3, -4, -5, -6, -7, -8
PREC_FP64, PREC_FP32, PREC_MIXED_BF16 = 0, 1, 2

# every entry point declared in include/stokesmg.h
EXPORTS = ["stokes_opts_default", "stokes_create", "stokes_destroy", "stokes_vector_length", "stokes_ghost_length",
           "stokes_num_levels", "stokes_rhs", "stokes_apply", "mg_precondition", "sqmr_solve",
           "stokes_residual_norm", "stokes_smooth", "stokes_restrict", "stokes_prolong_add", "stokes_coarse_solve",
           "stokes_profile_iteration", "stokes_residual_norm_noalloc", "sqmr_solve_batch", "stokes_level_schedule",
           "stokes_set_level_schedule", "stokes_level_tiles", "stokes_set_level_tiles", "stokes_level_dgs",
           "stokes_set_level_dgs", "sqmr_solve_unpreconditioned", "stokes_create_batch", "stokes_batch_size",
           "sqmr_solve_batched", "stokes_device_loop", "stokes_set_device_loop",
           "mg_solve",
           "stokes_measure_fma_peak", "stokes_label_flags", "stokes_test_grid_barrier", "stokes_strerror",
           # learned initial guess (include/warmstart.h)
           "warmstart_num_weights", "warmstart_create", "warmstart_destroy", "warmstart_set_scale",
           "warmstart_set_weights", "warmstart_get_weights", "warmstart_predict", "warmstart_loss_grad",
           "warmstart_adam_step", "warmstart_solve", "warmstart_set_engine", "warmstart_conv_check",
           "warmstart_mma_check"]

# kernel kinds reported by stokes_profile_iteration (STOKES_K_* in the header)
KERNEL_KINDS = ["apply_dot", "update_s", "dot2", "update_x", "scalars", "memset", "vanka_compute", "vanka_apply",
                "dgs_u", "dgs_p_fwd", "dgs_p_gather", "dgs_p_bwd", "residual", "restrict", "prolong", "coarse",
                "dgs_p_bwd_prep"]


class stokes_grid_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("levels", ctypes.c_int), ("coarsest_max", ctypes.c_int)]


class stokes_bc_t(ctypes.Structure):
    _fields_ = [("cell_labels", ctypes.POINTER(ctypes.c_uint8))]


class stokes_opts_t(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("kb_vanka", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("vanka_persistent", ctypes.c_int), ("autotune", ctypes.c_int),
                ("vanka_additive", ctypes.c_int), ("cycle", ctypes.c_int), ("distributive_jacobi", ctypes.c_int)]


class sqmr_info_t(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double), ("status", ctypes.c_int),
                ("vcycles", ctypes.c_int)]


class StokesError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {stokes_strerror(code)} ({code})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libstokesmg.so not built ({LIB_PATH}); run paper_2312_10615_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, d, i, ll = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_longlong
    sig = {
        "stokes_opts_default": (None, [ctypes.POINTER(stokes_opts_t)]),
        "stokes_create": (i, [ctypes.POINTER(stokes_grid_t), ctypes.POINTER(stokes_bc_t), d,
                              ctypes.POINTER(stokes_opts_t), ctypes.POINTER(vp)]),
        "stokes_destroy": (i, [vp]),
        "stokes_vector_length": (ll, [vp, i]),
        "stokes_ghost_length": (ll, [vp]),
        "stokes_num_levels": (i, [vp]),
        "stokes_rhs": (i, [vp, vp, vp, vp, vp]),
        "stokes_apply": (i, [vp, vp, vp, vp]),
        "mg_precondition": (i, [vp, vp, vp, vp]),
        "sqmr_solve": (i, [vp, vp, vp, d, i, ctypes.POINTER(sqmr_info_t), vp]),
        "sqmr_solve_unpreconditioned": (i, [vp, vp, vp, d, i, ctypes.POINTER(sqmr_info_t), vp]),
        "mg_solve": (i, [vp, vp, vp, d, i, ctypes.POINTER(sqmr_info_t), vp]),
        "stokes_residual_norm": (i, [vp, vp, vp, ctypes.POINTER(d), vp]),
        "stokes_smooth": (i, [vp, i, i, vp, vp, vp]),
        "stokes_restrict": (i, [vp, i, vp, vp, vp]),
        "stokes_prolong_add": (i, [vp, i, vp, vp, vp]),
        "stokes_coarse_solve": (i, [vp, vp, vp, vp]),
        "stokes_profile_iteration": (i, [vp, i, ctypes.POINTER(d), ctypes.POINTER(i), ctypes.POINTER(d),
                                         ctypes.POINTER(i), vp]),
        "stokes_residual_norm_noalloc": (i, [i, i, i, d, d, vp, vp, vp, vp]),
        "stokes_measure_fma_peak": (i, [i, ctypes.POINTER(d), vp]),
        "stokes_test_grid_barrier": (i, [vp, i, i, i, vp]),
        "stokes_label_flags": (i, [ctypes.POINTER(stokes_grid_t), ctypes.POINTER(stokes_bc_t), i,
                                   ctypes.POINTER(ctypes.c_uint8), ll]),
        "sqmr_solve_batch": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), d, i,
                                 ctypes.POINTER(sqmr_info_t), ctypes.POINTER(d), i]),
        "stokes_create_batch": (i, [i, ctypes.POINTER(stokes_grid_t), ctypes.POINTER(stokes_bc_t), d,
                                    ctypes.POINTER(stokes_opts_t), ctypes.POINTER(vp)]),
        "stokes_batch_size": (i, [vp]),
        "stokes_device_loop": (i, [vp]),
        "stokes_set_device_loop": (i, [vp, i]),
        "sqmr_solve_batched": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), d, i, ctypes.POINTER(sqmr_info_t), vp]),
        "stokes_level_schedule": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float)]),
        "stokes_set_level_schedule": (i, [vp, i, i, i]),
        "stokes_level_tiles": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float)]),
        "stokes_set_level_tiles": (i, [vp, i, ctypes.POINTER(i)]),
        "stokes_level_dgs": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float)]),
        "stokes_set_level_dgs": (i, [vp, i, i]),
        "stokes_strerror": (ctypes.c_char_p, [i]),
        "warmstart_num_weights": (ll, []),
        "warmstart_create": (i, [i, i, d, ctypes.POINTER(vp)]),
        "warmstart_destroy": (i, [vp]),
        "warmstart_set_scale": (i, [vp, d]),
        "warmstart_set_weights": (i, [vp, vp]),
        "warmstart_get_weights": (i, [vp, vp]),
        "warmstart_predict": (i, [vp, vp, vp, vp]),
        "warmstart_loss_grad": (i, [vp, vp, vp, vp, ctypes.POINTER(d), vp, vp]),
        "warmstart_adam_step": (i, [vp, d, d, d, d, vp]),
        "warmstart_solve": (i, [vp, vp, vp, vp, d, i, ctypes.POINTER(sqmr_info_t), ctypes.POINTER(i), vp]),
        "warmstart_set_engine": (i, [vp, i]),
        "warmstart_conv_check": (i, [i, i, i, i, vp, vp, vp, vp, vp]),
        "warmstart_mma_check": (i, [vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    """The loaded native library (loaded on first use; ImportError if it was never built)."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def stokes_strerror(code):
    return lib().stokes_strerror(int(code)).decode()


def _ptr(a):
    """Raw pointer of a float64 contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy vectors must be float64 and C-contiguous")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("torch vectors must be float64 and contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported vector type {type(a)}")


def _numel(a):
    """Number of entries of a torch tensor or numpy array."""
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _check(rc, where):
    if rc != OK:
        raise StokesError(rc, where)


def stokes_opts_default():
    o = stokes_opts_t()
    lib().stokes_opts_default(ctypes.byref(o))
    return o


def stokes_create(nx, ny=None, nz=None, viscosity=1.0, h=0.0, levels=0, coarsest_max=8, gamma=1e-3, kb_vanka=1,
                  precision=PREC_FP64, use_graphs=True, vanka_persistent=False, autotune=True, additive=False, cycle=1,
                  dwj=False, labels=None, batch=1):
    """labels: None (the box) or a uint8 array of (nx+2)(ny+2)(nz+2) cell labels, x fastest (0 interior,
    1 Dirichlet, 2 exterior); it is copied by the library.  batch > 1: a batched handle of that many
    problems on this grid (stokes_create_batch; solve with sqmr_solve_batched)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    g = stokes_grid_t(nx, ny, nz, h, levels, coarsest_max)
    o = stokes_opts_t(gamma, kb_vanka, precision, int(bool(use_graphs)), int(bool(vanka_persistent)),
                      int(bool(autotune)), int(bool(additive)), int(cycle), int(bool(dwj)))
    bc = None
    if labels is not None:
        import numpy as np
        lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8).reshape(-1))
        if lab.size != (nx + 2) * (ny + 2) * (nz + 2):
            raise ValueError("labels must hold (nx+2)(ny+2)(nz+2) entries")
        bc = stokes_bc_t(lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    hdl = ctypes.c_void_p()
    if batch > 1:
        _check(lib().stokes_create_batch(int(batch), ctypes.byref(g), None if bc is None else ctypes.byref(bc),
                                         viscosity, ctypes.byref(o), ctypes.byref(hdl)), "stokes_create_batch")
    else:
        _check(lib().stokes_create(ctypes.byref(g), None if bc is None else ctypes.byref(bc), viscosity,
                                   ctypes.byref(o), ctypes.byref(hdl)), "stokes_create")
    return hdl


def stokes_label_flags(labels, nx, ny=None, nz=None, level=0):
    """Per-entry flags of a labelled domain on one level, computed by the library's host code (no GPU):
    bit 0 unknown, bit 1 V2, bit 2 Dirichlet face, bits 3-5 dropped terms, bits 6/7 dropped normal
    neighbours (see include/stokesmg.h)."""
    import numpy as np
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8).reshape(-1))
    if lab.size != (nx + 2) * (ny + 2) * (nz + 2):
        raise ValueError("labels must hold (nx+2)(ny+2)(nz+2) entries")
    g = stokes_grid_t(nx, ny, nz, 0.0, 0, 8)
    bc = stokes_bc_t(lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    m = [nx, ny, nz]
    for _ in range(level):
        m = [a // 2 for a in m]
    n = (m[0] + 1) * m[1] * m[2] + m[0] * (m[1] + 1) * m[2] + m[0] * m[1] * (m[2] + 1) + m[0] * m[1] * m[2]
    out = np.zeros(n, np.uint8)
    _check(lib().stokes_label_flags(ctypes.byref(g), ctypes.byref(bc), level,
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n), "stokes_label_flags")
    return out


def stokes_destroy(h):
    _check(lib().stokes_destroy(h), "stokes_destroy")


def stokes_vector_length(h, level=0):
    return int(lib().stokes_vector_length(h, level))


def stokes_ghost_length(h):
    return int(lib().stokes_ghost_length(h))


def stokes_num_levels(h):
    return int(lib().stokes_num_levels(h))


def stokes_rhs(h, f, g, b, stream=None):
    _check(lib().stokes_rhs(h, _ptr(f), _ptr(g), _ptr(b), _stream(stream)), "stokes_rhs")


def stokes_apply(h, x, y, stream=None):
    _check(lib().stokes_apply(h, _ptr(x), _ptr(y), _stream(stream)), "stokes_apply")


def mg_precondition(h, s, t, stream=None):
    _check(lib().mg_precondition(h, _ptr(s), _ptr(t), _stream(stream)), "mg_precondition")


def sqmr_solve(h, rhs, x, tol=1e-8, max_iter=200, stream=None, check=True):
    info = sqmr_info_t()
    rc = lib().sqmr_solve(h, _ptr(rhs), _ptr(x), tol, max_iter, ctypes.byref(info), _stream(stream))
    if check:
        _check(rc, "sqmr_solve")
    return info


def stokes_residual_norm(h, b, x, stream=None):
    out = ctypes.c_double()
    _check(lib().stokes_residual_norm(h, _ptr(b), _ptr(x), ctypes.byref(out), _stream(stream)), "stokes_residual_norm")
    return out.value


def stokes_smooth(h, level, which, x, b, stream=None):
    _check(lib().stokes_smooth(h, level, which, _ptr(x), _ptr(b), _stream(stream)), "stokes_smooth")


def stokes_restrict(h, level, r_fine, b_coarse, stream=None):
    _check(lib().stokes_restrict(h, level, _ptr(r_fine), _ptr(b_coarse), _stream(stream)), "stokes_restrict")


def stokes_prolong_add(h, level, e_coarse, x_fine, stream=None):
    _check(lib().stokes_prolong_add(h, level, _ptr(e_coarse), _ptr(x_fine), _stream(stream)), "stokes_prolong_add")


def stokes_coarse_solve(h, b, x, stream=None):
    _check(lib().stokes_coarse_solve(h, _ptr(b), _ptr(x), _stream(stream)), "stokes_coarse_solve")


def stokes_profile_iteration(h, stream=None):
    """Per kernel kind: (ms all levels, launches all levels, ms level 0, launches level 0)."""
    k = len(KERNEL_KINDS)
    ma, ca, m0, c0 = (ctypes.c_double * k)(), (ctypes.c_int * k)(), (ctypes.c_double * k)(), (ctypes.c_int * k)()
    _check(lib().stokes_profile_iteration(h, k, ma, ca, m0, c0, _stream(stream)), "stokes_profile_iteration")
    return {name: (ma[j], ca[j], m0[j], c0[j]) for j, name in enumerate(KERNEL_KINDS)}


def stokes_level_schedule(h, level):
    """(mode, blocks, ms per symmetric sweep) of the Vanka schedule of a smoothed level."""
    m, b, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().stokes_level_schedule(h, level, ctypes.byref(m), ctypes.byref(b), ctypes.byref(t)),
           "stokes_level_schedule")
    return m.value, b.value, t.value


def stokes_set_level_schedule(h, level, mode, blocks=0):
    _check(lib().stokes_set_level_schedule(h, level, mode, blocks), "stokes_set_level_schedule")


def stokes_level_tiles(h, level):
    """((restrict bx, by, kz), (prolong bx, by, kz), (ms restrict, ms prolong)) of the transfers between
    level and level + 1."""
    t, m = (ctypes.c_int * 6)(), (ctypes.c_float * 2)()
    _check(lib().stokes_level_tiles(h, level, t, m), "stokes_level_tiles")
    return tuple(t[0:3]), tuple(t[3:6]), (m[0], m[1])


def stokes_set_level_tiles(h, level, restrict_tile, prolong_tile):
    t = (ctypes.c_int * 6)(*restrict_tile, *prolong_tile)
    _check(lib().stokes_set_level_tiles(h, level, t), "stokes_set_level_tiles")


def stokes_level_dgs(h, level):
    """(fused, (ms in place, ms fused)) of the symmetric DGS velocity passes on a smoothed level."""
    f, m = ctypes.c_int(), (ctypes.c_float * 2)()
    _check(lib().stokes_level_dgs(h, level, ctypes.byref(f), m), "stokes_level_dgs")
    return f.value, (m[0], m[1])


def stokes_set_level_dgs(h, level, fused):
    _check(lib().stokes_set_level_dgs(h, level, int(fused)), "stokes_set_level_dgs")


def stokes_residual_norm_noalloc(nx, ny, nz, h, viscosity, b, x, out, stream=None):
    """||b - L x||_2 written into the 1-element device tensor `out`, without any allocation in the
    library (for callers that cannot allocate; see include/stokesmg.h)."""
    n = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1) + nx * ny * nz
    for name, t in (("b", b), ("x", x)):
        if _numel(t) < n:
            raise StokesError(ERR_INVALID_ARG, f"stokes_residual_norm_noalloc: {name} holds {_numel(t)} < {n} entries")
    if _numel(out) < 1:
        raise StokesError(ERR_INVALID_ARG, "stokes_residual_norm_noalloc: out holds no entry")
    _check(lib().stokes_residual_norm_noalloc(nx, ny, nz, h, viscosity, _ptr(b), _ptr(x), _ptr(out),
                                              _stream(stream)), "stokes_residual_norm_noalloc")


def stokes_test_grid_barrier(h, level, missing_blocks, spin_limit, stream=None):
    """Status of one cooperative Vanka sweep whose barrier waits for missing_blocks extra blocks
    (STOKES_ERR_TIMEOUT expected for missing_blocks > 0); returns the raw status code."""
    return int(lib().stokes_test_grid_barrier(h, level, missing_blocks, spin_limit, _stream(stream)))


def stokes_measure_fma_peak(fp64=True, stream=None):
    """Measured FMA rate of the CUDA cores in flop/s (FP64 or FP32), the roof of the FP64 kernels."""
    r = ctypes.c_double()
    _check(lib().stokes_measure_fma_peak(1 if fp64 else 0, ctypes.byref(r), _stream(stream)), "stokes_measure_fma_peak")
    return r.value


def sqmr_solve_batch(handles, rhs, xs, tol=1e-8, max_iter=200, nstreams=8, check=True):
    """Solve independent problems concurrently (one stream per host thread).  Returns (infos, done_ms)."""
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h.value if hasattr(h, "value") else h for h in handles])
    R = (ctypes.c_void_p * n)(*[_ptr(b) for b in rhs])
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    infos = (sqmr_info_t * n)()
    done = (ctypes.c_double * n)()
    rc = lib().sqmr_solve_batch(n, H, R, X, tol, max_iter, infos, done, nstreams)
    if check:
        _check(rc, "sqmr_solve_batch")
    return list(infos), list(done)


def sqmr_solve_batched(h, rhs, xs, tol=1e-8, max_iter=200, stream=None, check=True):
    """All problems of a batched handle (one launch per step for all of them).  Returns the list of infos."""
    n = len(rhs)
    R = (ctypes.c_void_p * n)(*[_ptr(b) for b in rhs])
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    infos = (sqmr_info_t * n)()
    rc = lib().sqmr_solve_batched(h, R, X, tol, max_iter, infos, _stream(stream))
    if check:
        _check(rc, "sqmr_solve_batched")
    return list(infos)


def stokes_batch_size(h):
    return int(lib().stokes_batch_size(h))


def stokes_device_loop(h):
    """0 host loop, 1 device-side graph with programmatic launch edges, 2 without them."""
    return int(lib().stokes_device_loop(h))


def stokes_set_device_loop(h, enable):
    _check(lib().stokes_set_device_loop(h, 1 if enable else 0), "stokes_set_device_loop")


def sqmr_solve_unpreconditioned(h, rhs, x, tol=1e-8, max_iter=200, stream=None, check=True):
    info = sqmr_info_t()
    rc = lib().sqmr_solve_unpreconditioned(h, _ptr(rhs), _ptr(x), tol, max_iter, ctypes.byref(info), _stream(stream))
    if check:
        _check(rc, "sqmr_solve_unpreconditioned")
    return info


def mg_solve(h, rhs, x, tol=1e-8, max_iter=200, stream=None, check=True):
    info = sqmr_info_t()
    rc = lib().mg_solve(h, _ptr(rhs), _ptr(x), tol, max_iter, ctypes.byref(info), _stream(stream))
    if check:
        _check(rc, "mg_solve")
    return info


class Stokes:
    """Owning wrapper of a solver handle (one box problem on the current CUDA device)."""

    def __init__(self, nx, ny=None, nz=None, viscosity=1.0, **kw):
        self.h = stokes_create(nx, ny, nz, viscosity, **kw)
        self.dims = (nx, nx if ny is None else ny, nx if nz is None else nz)
        self.n = stokes_vector_length(self.h)
        self.levels = stokes_num_levels(self.h)

    def close(self):
        if self.h is not None and self.h.value:
            stokes_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def length(self, level=0):
        return stokes_vector_length(self.h, level)

    def rhs(self, f, g=None, out=None):
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device="cuda") if out is None else out
        stokes_rhs(self.h, f, g, out)
        return out

    def apply(self, x, out=None):
        import torch
        out = torch.empty_like(x) if out is None else out
        stokes_apply(self.h, x, out)
        return out

    def precondition(self, s, out=None):
        import torch
        out = torch.empty_like(s) if out is None else out
        mg_precondition(self.h, s, out)
        return out

    def solve(self, b, x0=None, tol=1e-8, max_iter=200, check=True):
        import torch
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        info = sqmr_solve(self.h, b, x, tol, max_iter, check=check)
        return x, info

    def residual_norm(self, b, x):
        return stokes_residual_norm(self.h, b, x)


# ------------------------------------------------------------------------------------------------
# learned initial guess (include/warmstart.h)

STORE_FP32, STORE_BF16 = 0, 1


def _fptr(a):
    """Raw pointer of a float32 contiguous torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("weight arrays must be float32 and C-contiguous")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("weight tensors must be float32 and contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def warmstart_num_weights():
    return int(lib().warmstart_num_weights())


class WarmStart:
    """Owning wrapper of the initial-guess network for n^3 problems (activations FP32 or BF16)."""

    def __init__(self, n, storage=STORE_BF16, scale=1.0):
        self.n = n
        self.h = ctypes.c_void_p()
        _check(lib().warmstart_create(n, storage, float(scale), ctypes.byref(self.h)), "warmstart_create")

    def close(self):
        if self.h is not None and self.h.value:
            _check(lib().warmstart_destroy(self.h), "warmstart_destroy")
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scale(self, scale):
        _check(lib().warmstart_set_scale(self.h, float(scale)), "warmstart_set_scale")

    def set_engine(self, tensor_cores):
        """BF16 storage: convolutions on the tensor cores (True, the default) or the CUDA cores."""
        _check(lib().warmstart_set_engine(self.h, 1 if tensor_cores else 0), "warmstart_set_engine")

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32) if isinstance(w, np.ndarray) else w
        assert (w.size if isinstance(w, np.ndarray) else w.numel()) == warmstart_num_weights()
        _check(lib().warmstart_set_weights(self.h, _fptr(w)), "warmstart_set_weights")

    def get_weights(self):
        w = np.zeros(warmstart_num_weights(), dtype=np.float32)
        _check(lib().warmstart_get_weights(self.h, _fptr(w)), "warmstart_get_weights")
        return w

    def predict(self, b, out=None, stream=None):
        import torch
        out = torch.empty_like(b) if out is None else out
        _check(lib().warmstart_predict(self.h, _ptr(b), _ptr(out), _stream(stream)), "warmstart_predict")
        return out

    def loss_grad(self, b, xstar, S=None, want_loss=True, want_grad=False, stream=None):
        """S None: error-form loss; S a Stokes handle: residual-form loss ||L (x0 - x*)||^2 / ||b||^2."""
        loss = ctypes.c_double(0.0)
        g = np.zeros(warmstart_num_weights(), dtype=np.float32) if want_grad else None
        hs = None if S is None else (S.h if isinstance(S, Stokes) else S)
        _check(lib().warmstart_loss_grad(self.h, hs, _ptr(b), _ptr(xstar), ctypes.byref(loss) if want_loss else None,
                                         _fptr(g) if want_grad else None, _stream(stream)), "warmstart_loss_grad")
        return (loss.value if want_loss else None), g

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(lib().warmstart_adam_step(self.h, lr, beta1, beta2, eps, _stream(stream)), "warmstart_adam_step")

    def train_step(self, b, xstar, lr, S=None, want_loss=False, stream=None):
        loss, _ = self.loss_grad(b, xstar, S=S, want_loss=want_loss, stream=stream)
        self.adam_step(lr, stream=stream)
        return loss

    def solve(self, S, b, x=None, tol=1e-8, max_iter=200, check=True, stream=None):
        """SQMR solve of Stokes handle S from the network's guess; returns (x, info, used_guess)."""
        import torch
        x = torch.empty_like(b) if x is None else x
        info = sqmr_info_t()
        used = ctypes.c_int(0)
        rc = lib().warmstart_solve(self.h, S.h if isinstance(S, Stokes) else S, _ptr(b), _ptr(x), tol, max_iter,
                                   ctypes.byref(info), ctypes.byref(used), _stream(stream))
        if check:
            _check(rc, "warmstart_solve")
        return x, info, bool(used.value)


def _raw(a):
    """Raw pointer of a contiguous torch tensor of any dtype (None -> NULL)."""
    if a is None:
        return None
    if not a.is_contiguous():
        raise TypeError("tensors must be contiguous")
    return a.data_ptr()


def warmstart_conv_check(n, ci, op, engine, x, w, out, g=None, stream=None):
    """One network operation on device tensors (op 0 convolution + activation, 1 data gradient, 2 weight
    gradient) on the CUDA cores (engine 0) or the tensor cores (engine 1); returns the status code."""
    return int(lib().warmstart_conv_check(n, ci, op, engine, _raw(x), _raw(g), _raw(w), _raw(out), _stream(stream)))


def warmstart_mma_check(a, b, d, stream=None):
    """d = a b^T by one tcgen05 MMA (a BF16 [128, 16], b BF16 [16, 16], d FP32 [128, 16]); status code."""
    return int(lib().warmstart_mma_check(_raw(a), _raw(b), _raw(d), _stream(stream)))
