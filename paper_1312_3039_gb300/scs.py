"""Python binding of the C ABI in ``include/scs_gpu.h`` (argument marshalling only).

Every step of the solve runs in the CUDA library ``libscs_gb300.so``; this
module converts arrays, fills the C structs and calls the entry points of the
same names.  There is no fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libscs_gb300.so")

SOLVED = 1
SOLVED_INACCURATE = 2
UNFINISHED = 0
INFEASIBLE = -1
UNBOUNDED = -2
INFEASIBLE_INACCURATE = -3
UNBOUNDED_INACCURATE = -4
INVALID_INPUT = -10
DEVICE_ERROR = -11
TIMEOUT = -12
NUMERICAL = -13
UNSUPPORTED = -14


class CSC(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("colptr", C.POINTER(C.c_int64)),
                ("rowidx", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double))]


class ConeC(C.Structure):
    _fields_ = [("z", C.c_int32), ("l", C.c_int32), ("q", C.POINTER(C.c_int32)), ("nq", C.c_int32),
                ("s", C.POINTER(C.c_int32)), ("ns", C.c_int32), ("ep", C.c_int32), ("ed", C.c_int32),
                ("p", C.POINTER(C.c_double)), ("np", C.c_int32)]


class Settings(C.Structure):
    _fields_ = [("eps_pri", C.c_double), ("eps_dual", C.c_double), ("eps_gap", C.c_double),
                ("eps_infeas", C.c_double), ("eps_unbdd", C.c_double), ("alpha", C.c_double),
                ("cg_rate", C.c_double), ("cg_adapt", C.c_double), ("cg_tol_rel", C.c_double), ("time_limit_s", C.c_double),
                ("psd_fp64_cond", C.c_double),
                ("max_iters", C.c_int32), ("check_interval", C.c_int32), ("cg_max_iters", C.c_int32),
                ("normalize", C.c_int32), ("scale_passes", C.c_int32), ("block_scale", C.c_int32),
                ("precision", C.c_int32),
                ("use_graph", C.c_int32), ("verbose", C.c_int32), ("device", C.c_int32),
                ("cuda_stream", C.c_void_p), ("linsys", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("cg_iters", C.c_int32),
                ("matvecs", C.c_int32), ("pobj", C.c_double), ("dobj", C.c_double),
                ("res_pri", C.c_double), ("res_dual", C.c_double), ("gap", C.c_double),
                ("tau", C.c_double), ("kappa", C.c_double), ("setup_s", C.c_double),
                ("solve_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib_handle = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run `python -m paper_1312_3039_gb300.build`")
        L = C.CDLL(LIB_PATH)
        P, D, I32, I64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_int64)
        L.scs_default_settings.argtypes = [C.POINTER(Settings)]
        L.scs_default_settings.restype = None
        L.scs_init.argtypes = [C.POINTER(CSC), D, D, C.POINTER(ConeC), C.POINTER(Settings), C.POINTER(I32)]
        L.scs_init.restype = P
        L.scs_solve.argtypes = [P, D, D, D, C.POINTER(Info)]
        L.scs_solve.restype = I32
        L.scs_warm_start.argtypes = [P, D, D, D]
        L.scs_warm_start.restype = I32
        L.scs_finish.argtypes = [P]
        L.scs_finish.restype = None
        L.scs_reset.argtypes = [P]
        L.scs_reset.restype = I32
        L.scs_iterate.argtypes = [P, I32, I32]
        L.scs_iterate.restype = I32
        L.scs_update_bc.argtypes = [P, D, D]
        L.scs_update_bc.restype = I32
        L.scs_iterate_checked.argtypes = [P, I32, C.POINTER(I32)]
        L.scs_iterate_checked.restype = I32
        L.scs_iterate_profiled.argtypes = [P, I32]
        L.scs_iterate_profiled.restype = I32
        L.scs_kernel_time.argtypes = [P, I32, D, I64]
        L.scs_kernel_time.restype = I32
        L.scs_get_iterates.argtypes = [P, D, D]
        L.scs_get_iterates.restype = I32
        L.scs_get_scaling.argtypes = [P, D, D, D, D]
        L.scs_get_scaling.restype = I32
        L.scs_dims.argtypes = [P, C.POINTER(I32), C.POINTER(I32), I64, I64]
        L.scs_dims.restype = I32
        L.scs_counters.argtypes = [P, C.POINTER(I32), I64]
        L.scs_counters.restype = I32
        L.scs_psd_counters.argtypes = [P, I64, I64, I64]
        L.scs_psd_counters.restype = I32
        L.scs_project.argtypes = [C.POINTER(ConeC), I32, C.c_void_p, C.c_void_p, C.c_int64, D, C.c_void_p]
        L.scs_project.restype = I32
        if hasattr(L, "scs_project_noalloc"):
            L.scs_project_noalloc.argtypes = [C.POINTER(ConeC), I32, C.c_void_p, C.c_void_p, C.c_int64, D,
                                              C.c_void_p]
            L.scs_project_noalloc.restype = I32
        L.scs_batch_init.argtypes = [I32, C.POINTER(CSC), D, D, C.POINTER(ConeC), C.POINTER(Settings),
                                     C.POINTER(I32)]
        L.scs_batch_init.restype = P
        L.scs_batch_solve.argtypes = [P, D, D, D, C.POINTER(Info)]
        L.scs_batch_solve.restype = I32
        L.scs_batch_warm_start.argtypes = [P, D, D, D]
        L.scs_batch_warm_start.restype = I32
        L.scs_batch_iterate.argtypes = [P, I32]
        L.scs_batch_iterate.restype = I32
        L.scs_batch_get_iterates.argtypes = [P, I32, D, D]
        L.scs_batch_get_iterates.restype = I32
        L.scs_batch_config.argtypes = [P, C.POINTER(I32), C.POINTER(I32), D, D]
        L.scs_batch_config.restype = I32
        L.scs_batch_finish.argtypes = [P]
        L.scs_batch_finish.restype = None
        L.scs_family_init.argtypes = [C.POINTER(CSC), C.POINTER(ConeC), I32, D, D, C.POINTER(Settings),
                                      C.POINTER(I32)]
        L.scs_family_init.restype = P
        L.scs_family_set_data.argtypes = [P, D, D]
        L.scs_family_set_data.restype = I32
        L.scs_family_warm_start.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p, I32]
        L.scs_family_warm_start.restype = I32
        L.scs_family_solve.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Info), I32]
        L.scs_family_solve.restype = I32
        L.scs_family_iterate.argtypes = [P, I32]
        L.scs_family_iterate.restype = I32
        L.scs_family_get_iterates.argtypes = [P, I32, D, D]
        L.scs_family_get_iterates.restype = I32
        L.scs_family_snapshots.argtypes = [P, C.c_void_p]
        L.scs_family_snapshots.restype = I32
        L.scs_family_unscale.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.scs_family_unscale.restype = I32
        L.scs_family_dims.argtypes = [P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]
        L.scs_family_dims.restype = I32
        L.scs_family_finish.argtypes = [P]
        L.scs_family_finish.restype = None
        V = C.c_void_p
        L.scs_mlp_create.argtypes = [I32, I32, I32, I32, I32, V, C.POINTER(I32)]
        L.scs_mlp_create.restype = P
        L.scs_mlp_param_count.argtypes = [P]
        L.scs_mlp_param_count.restype = C.c_int64
        L.scs_mlp_set_params.argtypes = [P, V]
        L.scs_mlp_set_params.restype = I32
        L.scs_mlp_get_params.argtypes = [P, V]
        L.scs_mlp_get_params.restype = I32
        L.scs_mlp_forward.argtypes = [P, V, V]
        L.scs_mlp_forward.restype = I32
        L.scs_mlp_gradients.argtypes = [P, V, V, V, C.POINTER(C.c_float)]
        L.scs_mlp_gradients.restype = I32
        L.scs_mlp_train_step.argtypes = [P, V, V, C.c_float, C.POINTER(C.c_float)]
        L.scs_mlp_train_step.restype = I32
        L.scs_mlp_destroy.argtypes = [P]
        L.scs_mlp_destroy.restype = None
        L.scs_mlp_set_tensor_path.argtypes = [P, I32]
        L.scs_mlp_set_tensor_path.restype = I32
        L.scs_mlp_error.argtypes = [P]
        L.scs_mlp_error.restype = I32
        L.scs_bf16_gemm.argtypes = [V, I32, V, I32, I32, I32, I32, V, I32, I32, V]
        L.scs_bf16_gemm.restype = I32
        L.scs_bf16_gemm_async.argtypes = [V, I32, V, I32, I32, I32, I32, V, I32, I32, V, V]
        L.scs_bf16_gemm_async.restype = I32
        L.scs_dense_gemm.argtypes = [I32, I32, I32, I32, C.c_double, V, C.c_int64, V, C.c_int64, C.c_double, V,
                                     C.c_int64, V]
        L.scs_dense_gemm.restype = I32
        L.scs_column_stats.argtypes = [V, C.c_int64, I32, V, V, V]
        L.scs_column_stats.restype = I32
        L.scs_standardize.argtypes = [V, C.c_int64, I32, V, V, V]
        L.scs_standardize.restype = I32
        L.scs_gather_rows.argtypes = [V, I32, V, C.c_int64, V, V]
        L.scs_gather_rows.restype = I32
        L.scs_warm_from_prediction.argtypes = [V, C.c_int64, V, V, I32, I32, C.c_int64, C.c_double, V, V, V, V]
        L.scs_warm_from_prediction.restype = I32
        L.scs_last_error.argtypes = []
        L.scs_last_error.restype = C.c_char_p
        _lib_handle = L
    return _lib_handle


def last_error() -> str:
    return lib().scs_last_error().decode()


def default_settings(**kw) -> Settings:
    s = Settings()
    lib().scs_default_settings(C.byref(s))
    for k, v in kw.items():
        if not hasattr(s, k):
            raise AttributeError(k)
        setattr(s, k, v)
    return s


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def cone_struct(cone):
    """ctypes scs_cone for a cone description (keeps its arrays alive)."""
    q = np.ascontiguousarray(list(getattr(cone, "q", ())) or [0], dtype=np.int32)
    s = np.ascontiguousarray(list(getattr(cone, "s", ())) or [0], dtype=np.int32)
    pw = np.ascontiguousarray(list(getattr(cone, "p", ())) or [0.0], dtype=np.float64)
    kc = ConeC(int(cone.z), int(cone.l), q.ctypes.data_as(C.POINTER(C.c_int32)), len(getattr(cone, "q", ())),
               s.ctypes.data_as(C.POINTER(C.c_int32)), len(getattr(cone, "s", ())), int(cone.ep),
               int(getattr(cone, "ed", 0)), pw.ctypes.data_as(C.POINTER(C.c_double)), len(getattr(cone, "p", ())))
    return kc, (q, s, pw)


def project(cone, dual, v_ptr, out_ptr, count, stream=None):
    """scs_project on device pointers (ints); returns the summed ||out - v||^2."""
    kc, keep = cone_struct(cone)
    d2 = C.c_double(0.0)
    rc = lib().scs_project(C.byref(kc), int(dual), C.c_void_p(v_ptr), C.c_void_p(out_ptr), int(count),
                           C.byref(d2), C.c_void_p(stream) if stream else None)
    if rc != 0:
        raise ScsError(rc, last_error())
    return d2.value


def project_noalloc(cone, dual, v_ptr, out_ptr, count, stream=None):
    """scs_project_noalloc (no device allocation; scratch in the library's
    static device array); returns the summed ||out - v||^2."""
    kc, keep = cone_struct(cone)
    d2 = C.c_double(0.0)
    rc = lib().scs_project_noalloc(C.byref(kc), int(dual), C.c_void_p(v_ptr), C.c_void_p(out_ptr), int(count),
                                   C.byref(d2), C.c_void_p(stream) if stream else None)
    if rc != 0:
        raise ScsError(rc, last_error())
    return d2.value


class ScsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"status {code}: {msg}")
        self.code = code


class Solver:
    """One problem on the GPU: ``scs_init`` at construction, ``scs_finish`` at close."""

    def __init__(self, A, b, c, cone, settings: Settings | None = None, **kw):
        import scipy.sparse as sp
        A = sp.csc_matrix(A)
        self.m, self.n = A.shape
        self._colptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self._rowidx = np.ascontiguousarray(A.indices, dtype=np.int32)
        self._val = np.ascontiguousarray(A.data, dtype=np.float64)
        self._b = np.ascontiguousarray(b, dtype=np.float64)
        self._c = np.ascontiguousarray(c, dtype=np.float64)
        csc = CSC(self.m, self.n, self._colptr.ctypes.data_as(C.POINTER(C.c_int64)),
                  self._rowidx.ctypes.data_as(C.POINTER(C.c_int32)),
                  self._val.ctypes.data_as(C.POINTER(C.c_double)))
        kc, self._cone_keep = cone_struct(cone)
        st = settings if settings is not None else default_settings()
        for k, v in kw.items():
            setattr(st, k, v)
        self.settings = st
        err = C.c_int32(0)
        self._w = lib().scs_init(C.byref(csc), _dptr(self._b), _dptr(self._c), C.byref(kc), C.byref(st),
                                 C.byref(err))
        if not self._w:
            raise ScsError(err.value, last_error())

    def _check(self, rc):
        if rc < 0 and rc <= INVALID_INPUT:
            raise ScsError(rc, last_error())
        return rc

    def solve(self):
        """Return ``(status, x, y, s, info_dict)``."""
        x = np.empty(self.n)
        y = np.empty(self.m)
        s = np.empty(self.m)
        info = Info()
        st = lib().scs_solve(self._w, _dptr(x), _dptr(y), _dptr(s), C.byref(info))
        self._check(st)
        return st, x, y, s, info.as_dict()

    def update_bc(self, b, c):
        """scs_update_bc: new b, c with the same A (Sec. 4.2)."""
        self._b = np.ascontiguousarray(b, dtype=np.float64)
        self._c = np.ascontiguousarray(c, dtype=np.float64)
        return self._check(lib().scs_update_bc(self._w, _dptr(self._b), _dptr(self._c)))

    def solve_to(self, x_ptr, y_ptr, s_ptr):
        """scs_solve writing x, y, s to the given addresses (host or device,
        ints; 0 skips one); returns (status, info_dict)."""
        info = Info()
        ptr = lambda a: C.cast(C.c_void_p(a), C.POINTER(C.c_double)) if a else None
        st = lib().scs_solve(self._w, ptr(x_ptr), ptr(y_ptr), ptr(s_ptr), C.byref(info))
        self._check(st)
        return st, info.as_dict()

    def warm_start(self, x=None, y=None, s=None):
        x = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        y = None if y is None else np.ascontiguousarray(y, dtype=np.float64)
        s = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
        return self._check(lib().scs_warm_start(self._w, _dptr(x), _dptr(y), _dptr(s)))

    def reset(self):
        return self._check(lib().scs_reset(self._w))

    def iterate(self, iters, sync=True):
        return self._check(lib().scs_iterate(self._w, int(iters), 1 if sync else 0))

    def iterate_checked(self, iters):
        """scs_iterate_checked: iterations with the Sec. 3.5 tests every
        check_interval (not stopping); returns the last test's status."""
        st = C.c_int32(0)
        self._check(lib().scs_iterate_checked(self._w, int(iters), C.byref(st)))
        return st.value

    def iterate_profiled(self, iters):
        return self._check(lib().scs_iterate_profiled(self._w, int(iters)))

    def kernel_time(self, kind):
        ms = C.c_double(0)
        n = C.c_int64(0)
        self._check(lib().scs_kernel_time(self._w, int(kind), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def iterates(self):
        N = self.n + self.m + 1
        u = np.empty(N)
        v = np.empty(N)
        self._check(lib().scs_get_iterates(self._w, _dptr(u), _dptr(v)))
        return u, v

    def scaling(self):
        D = np.empty(self.m)
        E = np.empty(self.n)
        sg = C.c_double(0)
        rh = C.c_double(0)
        self._check(lib().scs_get_scaling(self._w, _dptr(D), _dptr(E), C.byref(sg), C.byref(rh)))
        return D, E, sg.value, rh.value

    def counters(self):
        it = C.c_int32(0)
        cg = C.c_int64(0)
        self._check(lib().scs_counters(self._w, C.byref(it), C.byref(cg)))
        return it.value, cg.value

    def psd_counters(self):
        """(block projections, Jacobi sweeps, blocks reconstructed in FP64)."""
        a, b, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        self._check(lib().scs_psd_counters(self._w, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def dims(self):
        m, n = C.c_int32(0), C.c_int32(0)
        nnz, by = C.c_int64(0), C.c_int64(0)
        self._check(lib().scs_dims(self._w, C.byref(m), C.byref(n), C.byref(nnz), C.byref(by)))
        return m.value, n.value, nnz.value, by.value

    def close(self):
        if getattr(self, "_w", None):
            lib().scs_finish(self._w)
            self._w = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve(A, b, c, cone, **kw):
    """One-shot solve; returns ``(status, x, y, s, info)``."""
    with Solver(A, b, c, cone, **kw) as S:
        return S.solve()


class Batch:
    """Many independent programs solved by one persistent launch
    (``scs_batch_init`` / ``scs_batch_solve``); ``problems`` is a list of
    ``(A, b, c, cone)``."""

    def __init__(self, problems, settings: Settings | None = None, **kw):
        import scipy.sparse as sp
        self.count = len(problems)
        self._keep = []
        cscs = (CSC * self.count)()
        cones = (ConeC * self.count)()
        self.ns, self.ms = [], []
        bs, cs = [], []
        for i, (A, b, c, cone) in enumerate(problems):
            A = sp.csc_matrix(A)
            m, n = A.shape
            cp = np.ascontiguousarray(A.indptr, dtype=np.int64)
            ri = np.ascontiguousarray(A.indices, dtype=np.int32)
            va = np.ascontiguousarray(A.data, dtype=np.float64)
            cones[i], keep = cone_struct(cone)
            self._keep += [cp, ri, va, keep]
            cscs[i] = CSC(m, n, cp.ctypes.data_as(C.POINTER(C.c_int64)), ri.ctypes.data_as(C.POINTER(C.c_int32)),
                          va.ctypes.data_as(C.POINTER(C.c_double)))
            self.ns.append(n)
            self.ms.append(m)
            bs.append(np.asarray(b, dtype=np.float64))
            cs.append(np.asarray(c, dtype=np.float64))
        self._b = np.ascontiguousarray(np.concatenate(bs))
        self._c = np.ascontiguousarray(np.concatenate(cs))
        self.xoff = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        self.yoff = np.concatenate([[0], np.cumsum(self.ms)]).astype(np.int64)
        st = settings if settings is not None else default_settings()
        for k, v in kw.items():
            setattr(st, k, v)
        self.settings = st
        err = C.c_int32(0)
        self._w = lib().scs_batch_init(self.count, cscs, _dptr(self._b), _dptr(self._c), cones, C.byref(st),
                                       C.byref(err))
        if not self._w:
            raise ScsError(err.value, last_error())

    def _check(self, rc):
        if rc != 0:
            raise ScsError(rc, last_error())
        return rc

    def solve(self):
        """Return ``(xs, ys, ss, infos)``: per-program arrays and info dicts."""
        x = np.empty(int(self.xoff[-1]))
        y = np.empty(int(self.yoff[-1]))
        s = np.empty(int(self.yoff[-1]))
        info = (Info * self.count)()
        self._check(lib().scs_batch_solve(self._w, _dptr(x), _dptr(y), _dptr(s), info))
        xs = [x[self.xoff[i]:self.xoff[i + 1]] for i in range(self.count)]
        ys = [y[self.yoff[i]:self.yoff[i + 1]] for i in range(self.count)]
        ss = [s[self.yoff[i]:self.yoff[i + 1]] for i in range(self.count)]
        return xs, ys, ss, [info[i].as_dict() for i in range(self.count)]

    def warm_start(self, xs=None, ys=None, ss=None):
        cat = lambda parts: None if parts is None else np.ascontiguousarray(np.concatenate(parts), dtype=np.float64)
        x, y, s = cat(xs), cat(ys), cat(ss)
        return self._check(lib().scs_batch_warm_start(self._w, _dptr(x), _dptr(y), _dptr(s)))

    def iterate(self, iters):
        return self._check(lib().scs_batch_iterate(self._w, int(iters)))

    def iterates(self, index):
        N = self.ns[index] + self.ms[index] + 1
        u, v = np.empty(N), np.empty(N)
        self._check(lib().scs_batch_get_iterates(self._w, int(index), _dptr(u), _dptr(v)))
        return u, v

    def config(self):
        t, sp_ = C.c_int32(0), C.c_int32(0)
        tm, sm = C.c_double(0), C.c_double(0)
        self._check(lib().scs_batch_config(self._w, C.byref(t), C.byref(sp_), C.byref(tm), C.byref(sm)))
        return {"threads": t.value, "row_split": sp_.value, "tune_ms": tm.value, "setup_ms": sm.value}

    def close(self):
        if getattr(self, "_w", None):
            lib().scs_batch_finish(self._w)
            self._w = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Family:
    """Members that share A and the cone and differ in b, c
    (``scs_family_*``): one dense direct iteration of all members at once.
    ``B`` (count x m) and ``Cs`` (count x n) hold the members' b and c."""

    def __init__(self, A, cone, B, Cs, settings: Settings | None = None, **kw):
        import scipy.sparse as sp
        A = sp.csc_matrix(A)
        self.m, self.n = A.shape
        B = np.ascontiguousarray(B, dtype=np.float64)
        Cs = np.ascontiguousarray(Cs, dtype=np.float64)
        self.count = B.shape[0]
        assert B.shape == (self.count, self.m) and Cs.shape == (self.count, self.n)
        self._keep = [np.ascontiguousarray(A.indptr, dtype=np.int64), np.ascontiguousarray(A.indices, dtype=np.int32),
                      np.ascontiguousarray(A.data, dtype=np.float64)]
        cp, ri, va = self._keep
        csc = CSC(self.m, self.n, cp.ctypes.data_as(C.POINTER(C.c_int64)), ri.ctypes.data_as(C.POINTER(C.c_int32)),
                  va.ctypes.data_as(C.POINTER(C.c_double)))
        kc, keep = cone_struct(cone)
        self._keep.append(keep)
        st = settings if settings is not None else default_settings()
        for k, v in kw.items():
            setattr(st, k, v)
        self.settings = st
        err = C.c_int32(0)
        self._w = lib().scs_family_init(C.byref(csc), C.byref(kc), self.count, _dptr(B), _dptr(Cs), C.byref(st),
                                        C.byref(err))
        if not self._w:
            raise ScsError(err.value, last_error())

    def _check(self, rc):
        if rc != 0:
            raise ScsError(rc, last_error())
        return rc

    def set_data(self, B, Cs):
        B = np.ascontiguousarray(B, dtype=np.float64)
        Cs = np.ascontiguousarray(Cs, dtype=np.float64)
        return self._check(lib().scs_family_set_data(self._w, _dptr(B), _dptr(Cs)))

    def warm_start(self, X=None, Y=None, S=None):
        """Host arrays (count x n / m / m) in the caller's units (Sec. 4.2)."""
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (X, Y, S)]
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        return self._check(lib().scs_family_warm_start(self._w, *ptrs, 0))

    def warm_start_scaled_device(self, x_ptr, y_ptr, s_ptr):
        """Device pointers (FP64, count x n / m / m) of scaled x^, y^, s^."""
        return self._check(lib().scs_family_warm_start(self._w, x_ptr, y_ptr, s_ptr, 1))

    def solve(self):
        """Return ``(X, Y, S, infos)`` (count x n, count x m, count x m)."""
        X = np.empty((self.count, self.n))
        Y = np.empty((self.count, self.m))
        S = np.empty((self.count, self.m))
        info = (Info * self.count)()
        self._check(lib().scs_family_solve(self._w, X.ctypes.data, Y.ctypes.data, S.ctypes.data, info, 0))
        return X, Y, S, [info[i].as_dict() for i in range(self.count)]

    def solve_info(self):
        """Solve, returning only the per-member infos (outputs stay on the device)."""
        info = (Info * self.count)()
        self._check(lib().scs_family_solve(self._w, None, None, None, info, 0))
        return [info[i].as_dict() for i in range(self.count)]

    def iterate(self, iters):
        return self._check(lib().scs_family_iterate(self._w, int(iters)))

    def iterates(self, index):
        N = self.n + self.m + 1
        u, v = np.empty(N), np.empty(N)
        self._check(lib().scs_family_get_iterates(self._w, int(index), _dptr(u), _dptr(v)))
        return u, v

    def unscale(self, xh_ptr, yh_ptr, sh_ptr, x_ptr, y_ptr, s_ptr):
        """Device FP64 scaled points (count x n, m, m) to the caller's units."""
        return self._check(lib().scs_family_unscale(self._w, xh_ptr, yh_ptr, sh_ptr, x_ptr, y_ptr, s_ptr))

    def snapshots(self, dst_ptr):
        """Copy the members' (u_x, u_y, v_s, u_tau) at their first passing test
        (float32, count x (n + 2m + 1)) to dst_ptr (host or device)."""
        return self._check(lib().scs_family_snapshots(self._w, dst_ptr))

    def close(self):
        if getattr(self, "_w", None):
            lib().scs_family_finish(self._w)
            self._w = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rc(rc):
    if rc != 0:
        raise ScsError(rc, last_error())
    return rc


class MLP:
    """The warm-start network (``scs_mlp_*``): BF16 tensor-core kernels with
    FP32 master weights.  Pointers are device addresses (ints)."""

    def __init__(self, d_in, hidden, layers, d_out, batch, stream=None):
        err = C.c_int32(0)
        self.d_in, self.hidden, self.layers, self.d_out, self.batch = d_in, hidden, layers, d_out, batch
        self._w = lib().scs_mlp_create(d_in, hidden, layers, d_out, batch, stream, C.byref(err))
        if not self._w:
            raise ScsError(err.value, last_error())

    def param_count(self):
        return int(lib().scs_mlp_param_count(self._w))

    def set_tensor_path(self, tcgen05):
        """True: tcgen05 products (the default when the sizes allow); False: mma.sync."""
        return _rc(lib().scs_mlp_set_tensor_path(self._w, 1 if tcgen05 else 0))

    def error(self):
        return lib().scs_mlp_error(self._w)

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.param_count()
        return _rc(lib().scs_mlp_set_params(self._w, flat.ctypes.data))

    def get_params(self):
        out = np.empty(self.param_count(), dtype=np.float32)
        _rc(lib().scs_mlp_get_params(self._w, out.ctypes.data))
        return out

    def forward(self, x_ptr, y_ptr):
        return _rc(lib().scs_mlp_forward(self._w, x_ptr, y_ptr))

    def gradients(self, x_ptr, t_ptr):
        g = np.empty(self.param_count(), dtype=np.float32)
        loss = C.c_float(0)
        _rc(lib().scs_mlp_gradients(self._w, x_ptr, t_ptr, g.ctypes.data, C.byref(loss)))
        return loss.value, g

    def train_step(self, x_ptr, t_ptr, lr, want_loss=False):
        loss = C.c_float(0)
        _rc(lib().scs_mlp_train_step(self._w, x_ptr, t_ptr, float(lr), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_w", None):
            lib().scs_mlp_destroy(self._w)
            self._w = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dense_gemm(precision, M, N, K, alpha, a_ptr, lda, b_ptr, ldb, beta, c_ptr, ldc, stream=None):
    """scs_dense_gemm: C = alpha A B + beta C (column-major device arrays),
    enqueued on `stream`."""
    return _rc(lib().scs_dense_gemm(int(precision), int(M), int(N), int(K), float(alpha), a_ptr, int(lda), b_ptr,
                                    int(ldb), float(beta), c_ptr, int(ldc), stream))


def column_stats(data_ptr, rows, cols, mean_ptr, sd_ptr, stream=None):
    return _rc(lib().scs_column_stats(data_ptr, rows, cols, mean_ptr, sd_ptr, stream))


def standardize(data_ptr, rows, cols, mean_ptr, sd_ptr, stream=None):
    return _rc(lib().scs_standardize(data_ptr, rows, cols, mean_ptr, sd_ptr, stream))


def gather_rows(src_ptr, cols, idx_ptr, count, dst_ptr, stream=None):
    return _rc(lib().scs_gather_rows(src_ptr, cols, idx_ptr, count, dst_ptr, stream))


def warm_from_prediction(pred_ptr, ld, mean_ptr, sd_ptr, n, m, count, tau_min, xh_ptr, yh_ptr, sh_ptr, stream=None):
    return _rc(lib().scs_warm_from_prediction(pred_ptr, ld, mean_ptr, sd_ptr, n, m, count, tau_min, xh_ptr, yh_ptr,
                                              sh_ptr, stream))


def pack_params(params):
    """[(W, b), ...] -> flat float32 in the library's layout."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64)])
                           for W, b in params]).astype(np.float32)


def unpack_params(flat, sizes):
    out, p = [], 0
    for fin, fout in zip(sizes[:-1], sizes[1:]):
        W = flat[p:p + fin * fout].reshape(fout, fin)
        p += fin * fout
        b = flat[p:p + fout]
        p += fout
        out.append((W, b))
    return out
