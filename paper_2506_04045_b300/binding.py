"""Thin ctypes binding of libcluster.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/cluster.h; all
work on the iterate runs in the library's CUDA kernels.  Device buffers are
passed as torch CUDA tensors (their data pointers), host buffers as numpy
arrays.  If the shared library is missing it is built with nvcc; if that is
impossible an ImportError is raised (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CLUSTER_LIB_PATH selects another build of the same library (tuning variants)
_LIB_PATH = os.environ.get("CLUSTER_LIB_PATH") or os.path.join(_HERE, "libcluster.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, EMAXITER, ETIMEOUT, EAGAIN = range(8)
FP32, MIXED_BF16 = 0, 1
STEP_CONST, STEP_INV_L_FROB, STEP_INV_L_SPEC = 0, 1, 2
STOP_LOSS, STOP_PG_REL, STOP_PG_ABS, STOP_NONE = 0, 1, 2, 3


class ClusterError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cluster status {status}: {msg}")
        self.status = status


class CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("index64", ctypes.c_int32),
                ("_pad", ctypes.c_int32), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("step_rule", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("accel", ctypes.c_int32), ("borrow", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("tau", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int64),
                ("graph_chunk", ctypes.c_int32), ("fused_pass", ctypes.c_int32), ("relabel", ctypes.c_int32),
                ("l2_window", ctypes.c_int32), ("update_engine", ctypes.c_int32), ("overlap", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("f_iter", ctypes.c_int64), ("f", ctypes.c_double),
                ("trace_SU", ctypes.c_double), ("gram_fro2", ctypes.c_double), ("pg_norm", ctypes.c_double),
                ("tau", ctypes.c_double), ("L", ctypes.c_double), ("out_iter", ctypes.c_int64),
                ("done", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class KernelTimes(ctypes.Structure):
    _fields_ = [("pass_ms", ctypes.c_double), ("heavy_ms", ctypes.c_double), ("fold_ms", ctypes.c_double),
                ("update_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("launches", ctypes.c_int64), ("heavy_nnz", ctypes.c_int64),
                ("heavy_rows", ctypes.c_int64), ("kernels", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerOptions(ctypes.Structure):
    _fields_ = [("solve", Options), ("hbm_budget", ctypes.c_size_t), ("iters_per_tick", ctypes.c_int32),
                ("max_resident", ctypes.c_int32), ("borrow_host", ctypes.c_int32), ("_pad", ctypes.c_int32),
                ("queue_bytes_max", ctypes.c_size_t)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("ticks", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("queued", ctypes.c_int64), ("resident", ctypes.c_int64), ("resident_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("queued_host_bytes", ctypes.c_size_t), ("uptime_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class RequestTimes(ctypes.Structure):
    _fields_ = [("queue_s", ctypes.c_double), ("run_s", ctypes.c_double), ("total_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_P = ctypes.c_void_p
_SIGS = {
    "cluster_options_default": (None, [ctypes.POINTER(Options)]),
    "cluster_last_error": (ctypes.c_char_p, []),
    "cluster_init": (ctypes.c_int, [ctypes.POINTER(CSR), ctypes.c_int32, _P, ctypes.POINTER(Options), _P,
                                    ctypes.POINTER(_P)]),
    "cluster_step": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(Report)]),
    "cluster_enqueue": (ctypes.c_int, [_P, ctypes.c_int64]),
    "cluster_enqueue_profiled": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(KernelTimes)]),
    "cluster_solve": (ctypes.c_int, [_P, ctypes.POINTER(Report)]),
    "cluster_get_report": (ctypes.c_int, [_P, ctypes.POINTER(Report)]),
    "cluster_get_U": (ctypes.c_int, [_P, _P]),
    "cluster_objective": (ctypes.c_int, [ctypes.POINTER(CSR), ctypes.c_int32, _P, _P,
                                         ctypes.POINTER(ctypes.c_double)]),
    "cluster_objective_static": (ctypes.c_int, [ctypes.POINTER(CSR), ctypes.c_int32, _P, _P,
                                                ctypes.POINTER(ctypes.c_double)]),
    "cluster_hessian_apply": (ctypes.c_int, [ctypes.POINTER(CSR), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]),
    "cluster_state_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "cluster_get_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "cluster_set_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "cluster_destroy": (None, [_P]),
    "cluster_test_hooks": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cluster_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(CSR), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(_P), ctypes.POINTER(Options), _P, ctypes.POINTER(_P)]),
    "cluster_batch_enqueue": (ctypes.c_int, [_P, ctypes.c_int64]),
    "cluster_batch_step": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(Report)]),
    "cluster_batch_get_U": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "cluster_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cluster_batch_describe": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "cluster_batch_destroy": (None, [_P]),
    "cluster_server_options_default": (None, [ctypes.POINTER(ServerOptions)]),
    "cluster_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOptions), ctypes.POINTER(_P)]),
    "cluster_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(CSR), ctypes.c_int32, _P,
                                             ctypes.POINTER(ctypes.c_uint64)]),
    "cluster_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.POINTER(Report),
                                           ctypes.POINTER(RequestTimes)]),
    "cluster_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, _P, ctypes.POINTER(Report),
                                           ctypes.POINTER(RequestTimes)]),
    "cluster_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "cluster_server_destroy": (None, [_P]),
    "cluster_csr_from_edges": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, ctypes.c_int32,
                                              ctypes.POINTER(CSR)]),
    "cluster_csr_free": (None, [ctypes.POINTER(CSR)]),
}


def lib_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load (building first if needed) libcluster.so and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if _LIB_PATH == _build.LIB and not _build.up_to_date():
            try:
                _build.build()
            except Exception as exc:  # no nvcc, or a compile error
                if not os.path.exists(_LIB_PATH):
                    raise ImportError(f"libcluster.so is missing and could not be built: {exc}") from exc
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def last_error() -> str:
    return load().cluster_last_error().decode()


def check(status: int) -> None:
    if status != OK:
        raise ClusterError(status, last_error())


def default_options(**kw) -> Options:
    o = Options()
    load().cluster_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def make_csr(row_ptr, col, val) -> CSR:
    """CSR view of torch tensors (device for the solver, host for nothing else)."""
    import torch
    s = CSR()
    s.n = row_ptr.numel() - 1
    s.nnz = col.numel()
    if row_ptr.dtype == torch.int64:
        s.index64 = 1
    elif row_ptr.dtype == torch.int32:
        s.index64 = 0
    else:
        raise TypeError("row_ptr must be int32 or int64")
    if col.dtype != torch.int32 or val.dtype != torch.float32:
        raise TypeError("col must be int32 and val float32")
    for t in (row_ptr, col, val):
        if not t.is_contiguous():
            raise ValueError("CSR arrays must be contiguous")
    s.row_ptr = _ptr(row_ptr)
    s.col = _ptr(col)
    s.val = _ptr(val)
    return s


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return int(getattr(stream, "cuda_stream", stream))


class Solver:
    """Owns one cluster_ctx.  Inputs are torch CUDA tensors; the CSR tensors
    must stay alive while the solver exists when ``borrow=1``."""

    def __init__(self, row_ptr, col, val, U0, k: int | None = None, stream=None, **opts):
        self._lib = load()
        self._keep = (row_ptr, col, val)
        self.csr = make_csr(row_ptr, col, val)
        if U0.dtype.__str__() != "torch.float32" or not U0.is_contiguous():
            raise TypeError("U0 must be a contiguous float32 tensor")
        self.k = int(U0.shape[1]) if k is None else int(k)
        self.n = int(self.csr.n)
        self.options = default_options(**opts)
        self.stream = _stream_ptr(stream)
        self._ctx = ctypes.c_void_p()
        check(self._lib.cluster_init(ctypes.byref(self.csr), self.k, _ptr(U0), ctypes.byref(self.options),
                                     self.stream, ctypes.byref(self._ctx)))

    def step(self, iters: int) -> dict:
        rep = Report()
        check(self._lib.cluster_step(self._ctx, int(iters), ctypes.byref(rep)))
        return rep.as_dict()

    def enqueue(self, iters: int) -> None:
        check(self._lib.cluster_enqueue(self._ctx, int(iters)))

    def enqueue_profiled(self, iters: int) -> dict:
        kt = KernelTimes()
        check(self._lib.cluster_enqueue_profiled(self._ctx, int(iters), ctypes.byref(kt)))
        return kt.as_dict()

    def solve(self) -> dict:
        rep = Report()
        check(self._lib.cluster_solve(self._ctx, ctypes.byref(rep)))
        return rep.as_dict()

    def report(self) -> dict:
        rep = Report()
        check(self._lib.cluster_get_report(self._ctx, ctypes.byref(rep)))
        return rep.as_dict()

    def get_U(self, out=None):
        import torch
        if out is None:
            out = torch.empty((self.n, self.k), dtype=torch.float32, device="cuda")
        check(self._lib.cluster_get_U(self._ctx, _ptr(out)))
        return out

    def state_size(self) -> int:
        sz = ctypes.c_size_t()
        check(self._lib.cluster_state_size(self._ctx, ctypes.byref(sz)))
        return sz.value

    def get_state(self) -> np.ndarray:
        buf = np.empty(self.state_size(), dtype=np.uint8)
        check(self._lib.cluster_get_state(self._ctx, buf.ctypes.data, buf.nbytes))
        return buf

    def set_state(self, buf: np.ndarray) -> None:
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(self._lib.cluster_set_state(self._ctx, buf.ctypes.data, buf.nbytes))

    def test_hooks(self, flags: int) -> None:
        """cluster_test_hooks: bit 0 makes the tcgen05 update's waits give up."""
        check(self._lib.cluster_test_hooks(self._ctx, int(flags)))

    def close(self) -> None:
        if self._ctx:
            self._lib.cluster_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns one cluster_batch over several (row_ptr, col, val, U0) instances
    (torch CUDA tensors, kept alive by this object)."""

    def __init__(self, instances, stream=None, **opts):
        self._lib = load()
        self._keep = list(instances)
        self.count = len(self._keep)
        csrs = (CSR * self.count)()
        ks = (ctypes.c_int32 * self.count)()
        u0s = (_P * self.count)()
        self.shapes = []
        for i, (rp, c, v, U0) in enumerate(self._keep):
            csrs[i] = make_csr(rp, c, v)
            ks[i] = int(U0.shape[1])
            u0s[i] = _ptr(U0)
            self.shapes.append((int(U0.shape[0]), int(U0.shape[1])))
        self.options = default_options(**opts)
        self._ctx = ctypes.c_void_p()
        check(self._lib.cluster_batch_create(self.count, csrs, ks, u0s, ctypes.byref(self.options),
                                             _stream_ptr(stream), ctypes.byref(self._ctx)))

    def step(self, iters: int) -> list:
        reps = (Report * self.count)()
        check(self._lib.cluster_batch_step(self._ctx, int(iters), reps))
        return [r.as_dict() for r in reps]

    def enqueue(self, iters: int) -> None:
        check(self._lib.cluster_batch_enqueue(self._ctx, int(iters)))

    def autotune(self, trials: int = 1) -> dict:
        check(self._lib.cluster_batch_autotune(self._ctx, int(trials)))
        return self.describe()

    def describe(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        check(self._lib.cluster_batch_describe(self._ctx, buf, len(buf)))
        return json.loads(buf.value.decode())

    def get_U(self, i: int, out=None):
        import torch
        n, k = self.shapes[i]
        if out is None:
            out = torch.empty((n, k), dtype=torch.float32, device="cuda")
        check(self._lib.cluster_batch_get_U(self._ctx, int(i), _ptr(out)))
        return out

    def close(self) -> None:
        if self._ctx:
            self._lib.cluster_batch_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """cluster_server: continuous-batching solves of host-side requests.
    Requests are (row_ptr, col, val, U0) numpy arrays (int64/int32, int32,
    float32, float32 n x k)."""

    def __init__(self, hbm_budget: int = 0, iters_per_tick: int = 16, max_resident: int = 0, borrow_host: bool = False,
                 queue_bytes_max: int = 0, **solve_opts):
        self._lib = load()
        o = ServerOptions()
        self._lib.cluster_server_options_default(ctypes.byref(o))
        o.hbm_budget = int(hbm_budget)
        o.iters_per_tick = int(iters_per_tick)
        o.max_resident = int(max_resident)
        o.borrow_host = 1 if borrow_host else 0
        o.queue_bytes_max = int(queue_bytes_max)
        self._borrowed = {}
        for k, v in solve_opts.items():
            if not hasattr(o.solve, k):
                raise KeyError(k)
            setattr(o.solve, k, v)
        self.options = o
        self._ctx = ctypes.c_void_p()
        self._shapes = {}
        check(self._lib.cluster_server_create(ctypes.byref(o), ctypes.byref(self._ctx)))

    def submit(self, row_ptr, col, val, U0) -> int:
        rp = np.ascontiguousarray(row_ptr)
        if rp.dtype not in (np.int64, np.int32):
            rp = rp.astype(np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float32)
        U0 = np.ascontiguousarray(U0, dtype=np.float32)
        s = CSR()
        s.n = rp.size - 1
        s.nnz = col.size
        s.index64 = 1 if rp.dtype == np.int64 else 0
        s.row_ptr = rp.ctypes.data
        s.col = col.ctypes.data if col.size else 0
        s.val = val.ctypes.data if val.size else 0
        t = ctypes.c_uint64()
        check(self._lib.cluster_server_submit(self._ctx, ctypes.byref(s), int(U0.shape[1]), U0.ctypes.data,
                                              ctypes.byref(t)))
        self._shapes[t.value] = U0.shape
        if self.options.borrow_host:
            self._borrowed[t.value] = (rp, col, val, U0)   # must outlive the request
        return t.value

    def _result(self, ticket, st, U, rep, times):
        self._shapes.pop(ticket, None)
        self._borrowed.pop(ticket, None)
        check(st)
        return U, rep.as_dict(), times.as_dict()

    def poll(self, ticket: int):
        """None while pending, else (U, report, times); raises ClusterError if the solve failed."""
        U = np.empty(self._shapes[ticket], dtype=np.float32)
        rep, times = Report(), RequestTimes()
        st = self._lib.cluster_server_poll(self._ctx, ticket, U.ctypes.data, ctypes.byref(rep), ctypes.byref(times))
        if st == EAGAIN:
            return None
        return self._result(ticket, st, U, rep, times)

    def wait(self, ticket: int, timeout: float = 600.0):
        U = np.empty(self._shapes[ticket], dtype=np.float32)
        rep, times = Report(), RequestTimes()
        st = self._lib.cluster_server_wait(self._ctx, ticket, float(timeout), U.ctypes.data, ctypes.byref(rep),
                                           ctypes.byref(times))
        if st == ETIMEOUT:
            raise ClusterError(st, last_error())
        return self._result(ticket, st, U, rep, times)

    def stats(self) -> dict:
        st = ServerStats()
        check(self._lib.cluster_server_get_stats(self._ctx, ctypes.byref(st)))
        return st.as_dict()

    def close(self) -> None:
        if self._ctx:
            self._lib.cluster_server_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def objective(row_ptr, col, val, U, stream=None) -> float:
    """f(U) through cluster_objective (device tensors)."""
    lib = load()
    csr = make_csr(row_ptr, col, val)
    f = ctypes.c_double()
    check(lib.cluster_objective(ctypes.byref(csr), int(U.shape[1]), _ptr(U), _stream_ptr(stream), ctypes.byref(f)))
    return f.value


def objective_static(row_ptr, col, val, U, stream=None) -> float:
    """f(U) through cluster_objective_static (no device allocation; device tensors)."""
    lib = load()
    csr = make_csr(row_ptr, col, val)
    f = ctypes.c_double()
    check(lib.cluster_objective_static(ctypes.byref(csr), int(U.shape[1]), _ptr(U), _stream_ptr(stream),
                                       ctypes.byref(f)))
    return f.value


def hessian_apply(row_ptr, col, val, U, W, want_hw: bool = True, stream=None):
    """Hessian of f at U applied to W through cluster_hessian_apply (device
    tensors, n x k float32).  Returns (H[W] or None, <W, H[W]>, <grad f(U), W>)."""
    import torch
    lib = load()
    csr = make_csr(row_ptr, col, val)
    HW = torch.empty_like(U) if want_hw else None
    curv, slope = ctypes.c_double(), ctypes.c_double()
    check(lib.cluster_hessian_apply(ctypes.byref(csr), int(U.shape[1]), _ptr(U), _ptr(W), _stream_ptr(stream),
                                    _ptr(HW) if HW is not None else None, ctypes.byref(curv), ctypes.byref(slope)))
    return HW, curv.value, slope.value


def csr_from_edges(n: int, src, dst, w=None, add_unit_diag: bool = True):
    """cluster_csr_from_edges on host arrays; returns numpy (row_ptr, col, val)."""
    lib = load()
    src = np.ascontiguousarray(src, dtype=np.int64)
    dst = np.ascontiguousarray(dst, dtype=np.int64)
    wp = 0
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
        wp = w.ctypes.data
    out = CSR()
    check(lib.cluster_csr_from_edges(int(n), int(src.size), src.ctypes.data if src.size else 0,
                                     dst.ctypes.data if dst.size else 0, wp, 1 if add_unit_diag else 0,
                                     ctypes.byref(out)))
    try:
        rp = np.ctypeslib.as_array(ctypes.cast(out.row_ptr, ctypes.POINTER(ctypes.c_int64)), (n + 1,)).copy()
        nnz = int(out.nnz)
        if nnz:
            col = np.ctypeslib.as_array(ctypes.cast(out.col, ctypes.POINTER(ctypes.c_int32)), (nnz,)).copy()
            val = np.ctypeslib.as_array(ctypes.cast(out.val, ctypes.POINTER(ctypes.c_float)), (nnz,)).copy()
        else:
            col = np.zeros(0, np.int32)
            val = np.zeros(0, np.float32)
    finally:
        lib.cluster_csr_free(ctypes.byref(out))
    return rp, col, val
