"""Thin ctypes binding of ``libschur.so`` (see include/schur.h).

Marshalling only: every step of the solve runs in the CUDA library.  Device buffers are
passed as raw pointers taken from PyTorch CUDA tensors (PyTorch supplies device memory
and the stream); host masks are passed as numpy pointers.  There is no CPU fallback:
``load()`` raises when the library is missing.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

SCHUR_OK, SCHUR_EINVAL, SCHUR_ENOMEM, SCHUR_ENOTCONV = 0, 1, 2, 3
SCHUR_EBREAKDOWN, SCHUR_ECUDA, SCHUR_ESTATE = 4, 5, 6
UZAWA, SIMPLE = 0, 1
PRECOND_AUTO = 2          # server only: SIMPLE below AUTO_SIMPLE_BELOW fluid fraction
AUTO_SIMPLE_BELOW = 0.25
STOP_UNPRECOND, STOP_PRECOND = 0, 1
FP64, MIXED = 0, 1
LOOP_GRAPH, LOOP_HOST = 0, 1
INNER_JACOBI, INNER_MG = 0, 1
FIELD_P, FIELD_U, FIELD_FLAGS, FIELD_MASK, FIELD_G = 0, 1, 2, 3, 4

EXPORTED = [
    "schur_opts_default", "schur_create_geometry", "schur_set_force", "schur_solve",
    "schur_recover_velocity", "schur_permeability", "schur_get_field",
    "schur_geometry_info", "schur_apply_A", "schur_apply_B", "schur_apply_BT",
    "schur_apply_simple", "schur_solve_A", "schur_time_kernel", "schur_destroy",
    "schur_last_error", "schur_permeability_noalloc", "schur_solve_async", "schur_query",
    "schur_finish", "schur_batch_create", "schur_batch_run", "schur_batch_autotune",
    "schur_batch_destroy", "schur_footprint_bytes", "schur_server_create",
    "schur_server_submit", "schur_server_progress", "schur_server_take", "schur_server_info",
    "schur_server_destroy",
    "schur_set_launch", "schur_permeability_diag", "schur_history", "schur_cond_estimate",
    "schur_lanczos_extremes", "schur_set_barrier_limit", "schur_fp64_peak", "schur_mg_levels",
]
KERNELS = {"cgA_dir": 0, "cgA_matvec": 1, "cgA_update": 2, "cgS_dir": 3, "cgS_matvec": 4,
           "cgS_update": 5, "cgA_dir_f32": 6, "cgA_matvec_f32": 7, "cgA_update_f32": 8,
           "cgS_dir_f32": 9, "cgS_matvec_f32": 10, "cgS_update_f32": 11,
           "cgA_loop": 12, "cgS_loop": 13, "cgA_loop_f32": 14, "cgS_loop_f32": 15,
           "mgA_loop": 16, "mgS_loop": 17, "mgA_loop_f32": 18, "mgS_loop_f32": 19}
# iterations of one timed launch of the persistent loop kernels (ids 12-15)
TIMED_LOOP_ITERS = 20


class Opts(C.Structure):
    _fields_ = [("precond", C.c_int), ("stop_norm", C.c_int), ("precision", C.c_int),
                ("loop_mode", C.c_int), ("max_outer", C.c_int), ("max_inner", C.c_int),
                ("tol", C.c_double), ("tol_inner_A", C.c_double), ("tol_inner_S", C.c_double),
                ("tol_inner_f32", C.c_double), ("refine_factor", C.c_double),
                ("max_refine", C.c_int), ("step_max", C.c_int), ("inner_precond", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("zero_rhs", C.c_int),
                ("inner_status", C.c_int), ("inner_iters_A", C.c_longlong),
                ("inner_iters_S", C.c_longlong), ("rel_res", C.c_double),
                ("rel_res_precond", C.c_double), ("g_norm", C.c_double),
                ("kernel_launches", C.c_longlong), ("inner_iters_A_f32", C.c_longlong),
                ("inner_iters_S_f32", C.c_longlong), ("refinements", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class JobResult(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("outer_iters", C.c_int),
                ("inner_iters", C.c_int64), ("k", C.c_double), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("bytes", C.c_int64),
                ("precond", C.c_int), ("pad", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class GeomInfo(C.Structure):
    _fields_ = [("ndim", C.c_int), ("dims", C.c_int64 * 3), ("periodic", C.c_int * 3),
                ("n_cells", C.c_int64), ("face_stride", C.c_int64),
                ("n_unknown", C.c_int64 * 3), ("n_fluid", C.c_int64), ("h", C.c_double),
                ("device_bytes", C.c_int64)]


_LIB = None


def load(build_if_missing: bool = True):
    """Load the library (building it in-tree first when it is absent)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libschur.so not built at {path}")
        _build.build()
    lib = C.CDLL(path)
    vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
    sig = {
        "schur_opts_default": (None, [C.POINTER(Opts)]),
        "schur_create_geometry": (C.c_int, [vp, C.c_int, i64p, C.POINTER(C.c_int), vp,
                                            C.POINTER(vp)]),
        "schur_set_force": (C.c_int, [vp, C.POINTER(C.c_double)]),
        "schur_solve": (C.c_int, [vp, C.POINTER(Opts), C.POINTER(Stats)]),
        "schur_recover_velocity": (C.c_int, [vp, C.POINTER(Stats)]),
        "schur_permeability": (C.c_int, [vp, C.c_int, C.POINTER(C.c_double)]),
        "schur_get_field": (C.c_int, [vp, C.c_int, C.POINTER(vp), i64p, C.POINTER(C.c_int)]),
        "schur_geometry_info": (C.c_int, [vp, C.POINTER(GeomInfo)]),
        "schur_apply_A": (C.c_int, [vp, vp, vp]),
        "schur_apply_B": (C.c_int, [vp, vp, vp]),
        "schur_apply_BT": (C.c_int, [vp, vp, vp]),
        "schur_apply_simple": (C.c_int, [vp, vp, vp]),
        "schur_solve_A": (C.c_int, [vp, vp, vp, C.c_double, C.c_int, C.POINTER(C.c_int)]),
        "schur_time_kernel": (C.c_int, [vp, C.c_int, C.POINTER(C.c_float)]),
        "schur_set_launch": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
        "schur_set_barrier_limit": (C.c_int, [vp, C.c_uint, C.c_int]),
        "schur_fp64_peak": (C.c_int, [vp, C.c_int, C.POINTER(C.c_double)]),
        "schur_mg_levels": (C.c_int, [vp, C.c_int, i64p, C.c_int, C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]),
        "schur_history": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, C.POINTER(C.c_int)]),
        "schur_cond_estimate": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
        "schur_lanczos_extremes": (C.c_int, [vp, vp, C.c_int, C.POINTER(C.c_double),
                                             C.POINTER(C.c_double)]),
        "schur_permeability_diag": (C.c_int, [vp, C.POINTER(Opts), C.POINTER(C.c_double),
                                              C.POINTER(Stats)]),
        "schur_permeability_noalloc": (C.c_int, [vp, vp, C.c_int, i64p, C.c_int64, vp, vp]),
        "schur_solve_async": (C.c_int, [vp, C.POINTER(Opts)]),
        "schur_query": (C.c_int, [vp, C.POINTER(C.c_int)]),
        "schur_finish": (C.c_int, [vp, C.POINTER(Stats), C.POINTER(Stats)]),
        "schur_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(Opts), C.c_int, vp,
                                         C.POINTER(vp)]),
        "schur_batch_run": (C.c_int, [vp, C.POINTER(Stats), C.POINTER(Stats),
                                      C.POINTER(C.c_double)]),
        "schur_batch_autotune": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(Opts), vp,
                                           C.POINTER(C.c_int * 3), C.POINTER(C.c_double)]),
        "schur_batch_destroy": (None, [vp]),
        "schur_footprint_bytes": (C.c_int64, [C.c_int, i64p, C.c_int]),
        "schur_server_create": (C.c_int, [C.POINTER(Opts), C.c_int64, C.c_int, C.POINTER(vp)]),
        "schur_server_submit": (C.c_int, [vp, vp, C.c_int, i64p, C.POINTER(C.c_int), C.c_int,
                                          C.POINTER(C.c_int64)]),
        "schur_server_progress": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "schur_server_take": (C.c_int, [vp, C.POINTER(JobResult), C.c_int, C.POINTER(C.c_int)]),
        "schur_server_info": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
        "schur_server_destroy": (None, [vp]),
        "schur_destroy": (None, [vp]),
        "schur_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class SchurError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"schur error {code}: {msg}")
        self.code = code


def _check(rc, allow=(SCHUR_OK,)):
    if rc not in allow:
        raise SchurError(rc, load().schur_last_error().decode())
    return rc


def default_opts(**kw) -> Opts:
    o = Opts()
    load().schur_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    """Raw device pointer of a contiguous CUDA tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


class _CudaArray:
    """Zero-copy view of a library-owned device buffer (CUDA array interface)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None, "stream": None}


class Geometry:
    """Owner of one ``schur_geom_t``: mask -> flags -> solve -> velocity -> permeability.

    ``mask`` is a numpy uint8 array (host) or a CUDA uint8 tensor (device), C order
    ``[z][y][x]`` or ``[y][x]``.  ``periodic`` lists one flag per physical axis (x, y, z).
    """

    def __init__(self, mask, periodic=None, stream=None):
        lib = load()
        shape = tuple(int(s) for s in mask.shape)
        ndim = len(shape)
        if ndim not in (2, 3):
            raise ValueError("mask must be 2D or 3D")
        dims = (C.c_int64 * 3)(*(list(reversed(shape)) + [1] * (3 - ndim)))
        per = periodic if periodic is not None else (True,) * ndim
        per_c = (C.c_int * 3)(*([int(bool(p)) for p in per] + [1] * (3 - len(per))))
        if isinstance(mask, np.ndarray):
            self._host_mask = np.ascontiguousarray(mask, dtype=np.uint8)
            mptr = self._host_mask.ctypes.data_as(C.c_void_p)
        else:
            if mask.dtype.itemsize != 1:
                raise ValueError("mask tensor must be uint8")
            self._dev_mask = mask.contiguous()
            mptr = _ptr(self._dev_mask)
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:          # no torch: legacy default stream
                stream = 0
        self.stream = stream
        h = C.c_void_p()
        _check(lib.schur_create_geometry(mptr, ndim, dims, per_c, C.c_void_p(stream),
                                         C.byref(h)))
        self._h = h
        self.shape = shape
        self.ndim = ndim
        self.info = self.geometry_info()

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_h", None):
            load().schur_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- calls ----
    def geometry_info(self):
        gi = GeomInfo()
        _check(load().schur_geometry_info(self._h, C.byref(gi)))
        return gi

    def set_force(self, f):
        f3 = (C.c_double * 3)(*(list(f) + [0.0] * (3 - len(f))))
        _check(load().schur_set_force(self._h, f3))

    def solve(self, opts=None, allow_fail=False, **kw):
        o = opts if opts is not None else default_opts(**kw)
        st = Stats()
        rc = load().schur_solve(self._h, C.byref(o), C.byref(st))
        _check(rc, (SCHUR_OK, SCHUR_ENOTCONV, SCHUR_EBREAKDOWN) if allow_fail else (SCHUR_OK,))
        return st

    def recover_velocity(self, allow_fail=False):
        st = Stats()
        rc = load().schur_recover_velocity(self._h, C.byref(st))
        _check(rc, (SCHUR_OK, SCHUR_ENOTCONV, SCHUR_EBREAKDOWN) if allow_fail else (SCHUR_OK,))
        return st

    def permeability(self, axis: int) -> float:
        k = C.c_double()
        _check(load().schur_permeability(self._h, axis, C.byref(k)))
        return k.value

    def field(self, which):
        """Borrowed zero-copy torch view of a library field (valid until the next call)."""
        import torch
        p, n, dt = C.c_void_p(), C.c_int64(), C.c_int()
        _check(load().schur_get_field(self._h, which, C.byref(p), C.byref(n), C.byref(dt)))
        typestr = {0: "|u1", 1: "<f4", 2: "<f8"}[dt.value]
        return torch.as_tensor(_CudaArray(p.value, n.value, typestr), device="cuda")

    # ---- single operators on torch CUDA float64 buffers ----
    def apply_A(self, x, y):
        _check(load().schur_apply_A(self._h, _ptr(x), _ptr(y)))

    def apply_B(self, u, p):
        _check(load().schur_apply_B(self._h, _ptr(u), _ptr(p)))

    def apply_BT(self, p, u):
        _check(load().schur_apply_BT(self._h, _ptr(p), _ptr(u)))

    def apply_simple(self, p, q):
        _check(load().schur_apply_simple(self._h, _ptr(p), _ptr(q)))

    def set_barrier_limit(self, polls=0, skip_block=-1):
        """Poll limit of the loop kernels' grid-barrier waits (0: default) and the block
        that leaves out its arrivals for testing the bounded wait (-1: none)."""
        _check(load().schur_set_barrier_limit(self._h, polls, skip_block))

    def solve_async(self, **kw):
        _check(load().schur_solve_async(self._h, C.byref(default_opts(**kw))))

    def query(self):
        d = C.c_int()
        _check(load().schur_query(self._h, C.byref(d)))
        return bool(d.value)

    def finish(self, allow_fail=False):
        st, rs = Stats(), Stats()
        rc = load().schur_finish(self._h, C.byref(st), C.byref(rs))
        _check(rc, (SCHUR_OK, SCHUR_ENOTCONV, SCHUR_EBREAKDOWN) if allow_fail else (SCHUR_OK,))
        return st, rs

    def solve_A(self, b, x, tol=1e-12, max_iter=20000):
        it = C.c_int()
        _check(load().schur_solve_A(self._h, _ptr(b), _ptr(x), tol, max_iter, C.byref(it)))
        return it.value

    def permeability_diag(self, allow_fail=False, **kw):
        """(k_xx, k_yy, k_zz) and the solve stats of each axis (schur_permeability_diag)."""
        o = default_opts(**kw)
        k = (C.c_double * 3)()
        st = (Stats * 3)()
        rc = load().schur_permeability_diag(self._h, C.byref(o), k, st)
        _check(rc, (SCHUR_OK, SCHUR_ENOTCONV, SCHUR_EBREAKDOWN) if allow_fail else (SCHUR_OK,))
        return tuple(k), list(st)[:self.info.ndim]

    def history(self):
        """Per-iteration record of the last solve: dict of numpy arrays alpha, beta, rel,
        relz (schur_history)."""
        import numpy as np
        n = C.c_int()
        _check(load().schur_history(self._h, 0, None, None, None, None, C.byref(n)))
        out = {k: np.full(n.value, np.nan) for k in ("alpha", "beta", "rel", "relz")}
        if n.value:
            ptr = [out[k].ctypes.data_as(C.c_void_p) for k in ("alpha", "beta", "rel", "relz")]
            _check(load().schur_history(self._h, n.value, *ptr, C.byref(n)))
        return out

    def cond_estimate(self):
        """(lambda_min, lambda_max, cond) from the last FP64 solve's CG coefficients."""
        lo, hi, c = C.c_double(), C.c_double(), C.c_double()
        _check(load().schur_cond_estimate(self._h, C.byref(lo), C.byref(hi), C.byref(c)))
        return lo.value, hi.value, c.value

    def set_launch(self, blocks_per_sm=8, entries_per_thread=1, persistent=1):
        """Launch shape of this geometry's kernels (see schur_set_launch)."""
        _check(load().schur_set_launch(self._h, blocks_per_sm, entries_per_thread, persistent))

    def mg_levels(self, simple=False):
        """(entries per level, first one-block level) of the multigrid hierarchy of A or
        S-hat; ([], 0) before the first multigrid solve (schur_mg_levels)."""
        sizes = (C.c_int64 * 64)()
        nlev, tail = C.c_int(), C.c_int()
        _check(load().schur_mg_levels(self._h, int(simple), sizes, 64, C.byref(nlev), C.byref(tail)))
        return [int(sizes[i]) for i in range(min(nlev.value, 64))], tail.value

    def time_kernel(self, name) -> float:
        """Milliseconds of one launch of a hot kernel (CUDA events on the handle stream)."""
        ms = C.c_float()
        _check(load().schur_time_kernel(self._h, KERNELS[name], C.byref(ms)))
        return ms.value

    def permeability_noalloc(self, k_out, u=None, flags=None):
        """Darcy permeability of a face velocity field through the allocation-free entry
        point; k_out is a CUDA float64 tensor of 3 entries (written asynchronously)."""
        u = self.field(FIELD_U) if u is None else u
        flags = self.field(FIELD_FLAGS) if flags is None else flags
        dims = (C.c_int64 * 3)(*(list(reversed(self.shape)) + [1] * (3 - self.ndim)))
        _check(load().schur_permeability_noalloc(_ptr(u), _ptr(flags), self.ndim, dims,
                                                 self.face_stride, C.c_void_p(self.stream),
                                                 _ptr(k_out)))

    # ---- layout helpers ----
    @property
    def face_stride(self) -> int:
        return int(self.info.face_stride)

    @property
    def n_cells(self) -> int:
        return int(self.info.n_cells)

    def faces_to_grid(self, t):
        """Face-space tensor [d*stride] -> [d, *shape] view (drops the padding)."""
        d, s, n = self.ndim, self.face_stride, self.n_cells
        return t.view(d, s)[:, :n].reshape((d,) + self.shape)


def _dims(shape):
    return (C.c_int64 * 3)(*(list(reversed(shape)) + [1] * (3 - len(shape))))


def _per(periodic, ndim):
    per = periodic if periodic is not None else (True,) * ndim
    return (C.c_int * 3)(*([int(bool(p)) for p in per] + [1] * (3 - len(per))))


class Batch:
    """Many geometries solved by one CUDA graph launch (see schur_batch_create)."""

    def __init__(self, geoms, blocks_per_sm=8, stream=None, **opts):
        self.geoms = list(geoms)
        self.opts = default_opts(**opts)
        self.stream = geoms[0].stream if stream is None else stream
        arr = (C.c_void_p * len(self.geoms))(*[g._h.value for g in self.geoms])
        self._arr = arr
        h = C.c_void_p()
        _check(load().schur_batch_create(arr, len(self.geoms), C.byref(self.opts),
                                         blocks_per_sm, C.c_void_p(self.stream), C.byref(h)))
        self._h = h

    @staticmethod
    def autotune(geoms, stream=None, **opts):
        """Times the batch for a few launch shapes and leaves the geometries on the fastest;
        returns ((blocks_per_sm, entries_per_thread, persistent), ms).  Run the batch with
        blocks_per_sm=0 to keep that shape."""
        o = default_opts(**opts)
        arr = (C.c_void_p * len(geoms))(*[g._h.value for g in geoms])
        best, ms = (C.c_int * 3)(), C.c_double()
        st = geoms[0].stream if stream is None else stream
        _check(load().schur_batch_autotune(arr, len(geoms), C.byref(o), C.c_void_p(st),
                                           C.byref(best), C.byref(ms)))
        return tuple(best), ms.value

    def run(self, allow_fail=False):
        n = len(self.geoms)
        ss, rs = (Stats * n)(), (Stats * n)()
        k = (C.c_double * (3 * n))()
        rc = load().schur_batch_run(self._h, ss, rs, k)
        _check(rc, (SCHUR_OK, SCHUR_ENOTCONV, SCHUR_EBREAKDOWN) if allow_fail else (SCHUR_OK,))
        return list(ss), list(rs), [tuple(k[3 * i:3 * i + 3]) for i in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            load().schur_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with admission by device footprint (see schur_server_create)."""

    def __init__(self, mem_budget_bytes, max_active=16, **opts):
        self.opts = default_opts(**opts)
        h = C.c_void_p()
        _check(load().schur_server_create(C.byref(self.opts), int(mem_budget_bytes),
                                          int(max_active), C.byref(h)))
        self._h = h

    def submit(self, mask, axis=0, periodic=None):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        jid = C.c_int64()
        _check(load().schur_server_submit(self._h, m.ctypes.data_as(C.c_void_p), m.ndim,
                                          _dims(m.shape), _per(periodic, m.ndim), axis,
                                          C.byref(jid)))
        return jid.value

    def progress(self):
        a, p = C.c_int(), C.c_int()
        _check(load().schur_server_progress(self._h, C.byref(a), C.byref(p)))
        return a.value, p.value

    def take(self, max_results=1024):
        out = (JobResult * max_results)()
        n = C.c_int()
        _check(load().schur_server_take(self._h, out, max_results, C.byref(n)))
        return [out[i].as_dict() for i in range(n.value)]

    def info(self):
        b, a = C.c_int64(), C.c_int()
        _check(load().schur_server_info(self._h, C.byref(b), C.byref(a)))
        return {"peak_bytes": b.value, "peak_active": a.value}

    def close(self):
        if getattr(self, "_h", None):
            load().schur_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lanczos_extremes(alpha, beta):
    """(lambda_min, lambda_max) of the Lanczos tridiagonal of a CG run (host computation of
    the library, see schur_lanczos_extremes)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    lo, hi = C.c_double(), C.c_double()
    _check(load().schur_lanczos_extremes(a.ctypes.data_as(C.c_void_p),
                                         b.ctypes.data_as(C.c_void_p) if b.size else None,
                                         len(a), C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def footprint_bytes(shape, precision=FP64):
    return load().schur_footprint_bytes(len(shape), _dims(shape), precision)


def fp64_peak(iters=1 << 16, stream=None):
    """Measured FP64 DFMA lane-operations per second of the current device
    (schur_fp64_peak)."""
    v = C.c_double()
    _check(load().schur_fp64_peak(C.c_void_p(stream or 0), iters, C.byref(v)))
    return v.value
