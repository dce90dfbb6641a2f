"""ctypes binding of the libpit C-ABI (include/pit.h).

Argument marshalling only: every step of the parallel-in-time path runs in
the CUDA kernels of ``libpit.so``.  Arrays are numpy arrays (host memory,
``on_device = 0``) or CUDA torch tensors (device memory, ``on_device = 1``).
Loading fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpit.so")
_lib: Optional[C.CDLL] = None

# status codes
PIT_OK, PIT_PENDING = 0, 1
PIT_E_INVALID, PIT_E_NOMEM, PIT_E_CUDA, PIT_E_BREAKDOWN = -1, -2, -3, -4
PIT_E_MAXITER, PIT_E_NONFINITE, PIT_E_TIMEOUT, PIT_E_BUSY, PIT_E_UNSUPPORTED = -5, -6, -7, -8, -9
PIT_E_CANCELLED = -10
STATUS_NAMES = {0: "ok", 1: "pending", -1: "invalid", -2: "nomem", -3: "cuda", -4: "breakdown",
                -5: "maxiter", -6: "nonfinite", -7: "timeout", -8: "busy", -9: "unsupported",
                -10: "cancelled"}

PIT_OP = {"heat1d": 1, "heat2d": 2, "advdiff2d": 3, "dense": 4}
PIT_STEP = {"ie": 1, "rk4": 2}
PIT_FP64, PIT_MIXED = 0, 1
PIT_FF, PIT_SPLIT, PIT_MIXED_BF16 = 2, 3, 4
PRECISION = {"fp64": PIT_FP64, "mixed": PIT_MIXED, "ff": PIT_FF, "split": PIT_SPLIT,
             "mixed_bf16": PIT_MIXED_BF16}
TOL_MODE = {"r0": 0, "rhs": 1}
APPLY = {"F": 1, "Ginv": 2, "GinvF": 3, "residual": 4}
X0 = {"coarse": 0, "zero": 1, "given": 2}


class OperatorDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nu", C.c_double),
                ("vx", C.POINTER(C.c_double)), ("vy", C.POINTER(C.c_double)),
                ("A", C.POINTER(C.c_double))]


class StepperDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("steps", C.c_int), ("inner", C.c_int)]


class ProblemDesc(C.Structure):
    _fields_ = [("op", OperatorDesc), ("y0", C.POINTER(C.c_double)), ("batch", C.c_int),
                ("T", C.c_double), ("N", C.c_int), ("fine", StepperDesc),
                ("coarse", StepperDesc), ("precision", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart_eps0", C.c_double), ("max_iter", C.c_int),
                ("x0_mode", C.c_int), ("refine_max", C.c_int), ("inner_tol", C.c_double),
                ("stream", C.c_void_p), ("history", C.POINTER(C.c_double)),
                ("history_len", C.c_int), ("residual_precision", C.c_int), ("tol_mode", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("matvecs", C.c_int), ("restarts", C.c_int),
                ("refinements", C.c_int), ("fine_slice_steps", C.c_longlong),
                ("r0", C.c_double), ("precond_resid", C.c_double), ("seconds", C.c_double),
                ("status", C.c_int), ("history_count", C.c_int),
                ("queue_seconds", C.c_double), ("latency_seconds", C.c_double),
                ("device_bytes", C.c_longlong), ("graph_iterations", C.c_int)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong),
                ("failed", C.c_longlong), ("cancelled", C.c_longlong),
                ("queued", C.c_longlong), ("running", C.c_longlong),
                ("max_running", C.c_int), ("slots", C.c_int),
                ("latency_p50", C.c_double), ("latency_p99", C.c_double),
                ("latency_mean", C.c_double), ("queue_p50", C.c_double),
                ("queue_p99", C.c_double), ("service_p50", C.c_double),
                ("service_p99", C.c_double), ("window_seconds", C.c_double),
                ("solves_per_s", C.c_double), ("slice_steps_per_s", C.c_double),
                ("hbm_budget", C.c_size_t), ("hbm_reserved", C.c_size_t),
                ("hbm_reserved_peak", C.c_size_t), ("pool_peak", C.c_size_t)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PitError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libpit: {STATUS_NAMES.get(status, status)} ({status}): {msg}")
        self.status = status


# every symbol declared in include/pit.h
EXPORTS = ["pit_default_opts", "pit_version", "pit_last_error", "pit_problem_create",
           "pit_problem_destroy", "pit_problem_shape", "pit_apply_operator", "pit_serial_fine",
           "pit_bicgstab_solve", "pit_parareal_solve", "pit_block_reduce",
           "pit_problem_set_y0", "pit_kernel_launches", "pit_set_timing", "pit_get_timing",
           "pit_block_reduce_noalloc", "pit_selftest_convert", "pit_server_create",
           "pit_server_destroy", "pit_serve_submit", "pit_serve_poll", "pit_serve_wait",
           "pit_serve_cancel", "pit_serve_footprint", "pit_server_stats",
           "pit_problem_set_source"]

TIME_CLASSES = {"fine_fp32": 0, "fine_fp64": 1, "sweep_mixed": 2, "sweep_fp64": 3, "krylov": 4,
                "fine_ff": 5, "fine_split": 6, "inner": 7}


def lib_path() -> str:
    return _LIB_PATH


def load() -> C.CDLL:
    """Loads libpit.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libpit.so not found at {_LIB_PATH}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    lib.pit_default_opts.argtypes = [C.POINTER(SolveOpts)]
    lib.pit_default_opts.restype = None
    lib.pit_version.restype = C.c_char_p
    lib.pit_last_error.argtypes = [C.c_char_p, C.c_size_t]
    lib.pit_last_error.restype = C.c_size_t
    lib.pit_problem_create.argtypes = [C.POINTER(ProblemDesc), C.POINTER(P)]
    lib.pit_problem_destroy.argtypes = [P]
    lib.pit_problem_shape.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.pit_apply_operator.argtypes = [P, C.c_int, C.c_int, P, P, C.c_int, P]
    lib.pit_serial_fine.argtypes = [P, C.c_int, P, C.c_int]
    lib.pit_bicgstab_solve.argtypes = [P, C.POINTER(SolveOpts), P, C.c_int, C.POINTER(SolveInfo)]
    lib.pit_parareal_solve.argtypes = [P, C.c_int, C.c_double, P, C.c_int, C.POINTER(SolveInfo)]
    lib.pit_block_reduce.argtypes = [P, P, C.c_int, C.c_int, P, P, P]
    lib.pit_block_reduce_noalloc.argtypes = [P, P, C.c_int, C.c_int, P, P, P]
    lib.pit_problem_set_y0.argtypes = [P, P, C.c_int]
    lib.pit_problem_set_source.argtypes = [P, P, C.c_int]
    lib.pit_selftest_convert.argtypes = [P, C.c_int, P, P]
    lib.pit_kernel_launches.argtypes = []
    lib.pit_kernel_launches.restype = C.c_ulonglong
    lib.pit_set_timing.argtypes = [P, C.c_int]
    lib.pit_get_timing.argtypes = [P, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double)]
    lib.pit_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(P)]
    lib.pit_server_destroy.argtypes = [P]
    lib.pit_serve_submit.argtypes = [P, C.POINTER(ProblemDesc), C.POINTER(SolveOpts),
                                     C.POINTER(C.c_uint64)]
    lib.pit_serve_poll.argtypes = [P, C.c_uint64, P, C.POINTER(SolveInfo)]
    lib.pit_serve_wait.argtypes = [P, C.c_uint64, C.c_double, P, C.POINTER(SolveInfo)]
    lib.pit_serve_cancel.argtypes = [P, C.c_uint64]
    lib.pit_serve_footprint.argtypes = [C.POINTER(ProblemDesc), C.POINTER(C.c_size_t)]
    lib.pit_server_stats.argtypes = [P, C.c_int, C.POINTER(ServerStats)]
    for name in EXPORTS:
        if name not in ("pit_default_opts", "pit_version", "pit_last_error", "pit_kernel_launches"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def last_error() -> str:
    lib = load()
    buf = C.create_string_buffer(1024)
    lib.pit_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(status: int) -> int:
    if status < 0:
        raise PitError(status, last_error())
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _torch_stream(x, stream):
    """The caller's current torch stream for device arrays (unless one is given)."""
    if stream is not None or isinstance(x, np.ndarray):
        return stream
    import torch
    return torch.cuda.current_stream(x.device).cuda_stream


def _array_arg(x, n: Optional[int] = None) -> Tuple[int, int, object]:
    """(pointer, on_device, keepalive) for a numpy array or a CUDA torch
    tensor.  With n, the array must hold exactly n values: the library reads
    or writes that many through the pointer, so a shorter array would be
    accessed out of bounds."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous float64")
        out, size = (x.ctypes.data, 0, x), x.size
    else:
        import torch  # device memory only
        if not isinstance(x, torch.Tensor):
            raise TypeError(f"unsupported array type {type(x)}")
        if x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda:
            raise ValueError("device tensors must be contiguous CUDA float64")
        out, size = (x.data_ptr(), 1, x), x.numel()
    if n is not None and size != n:
        raise ValueError(f"expected an array of {n} values, got {size}")
    return out


def _host_values(a, n: int, what: str) -> np.ndarray:
    """a as a C-contiguous float64 host array of exactly n values."""
    v = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if v.size != n:
        raise ValueError(f"{what}: expected {n} values, got {v.size}")
    return v


def problem_desc(w, precision: int) -> Tuple[ProblemDesc, list]:
    """pit_problem_desc of a workload, and the arrays it points into."""
    keep = []
    M = int(w.nx) * int(w.ny)
    y0 = _host_values(w.y0, int(w.batch) * M, "y0")
    keep.append(y0)
    op = OperatorDesc(PIT_OP[w.kind], w.nx, w.ny, float(w.nu), None, None, None)
    if w.kind == "advdiff2d":
        vx = _host_values(w.vx, M, "vx")
        vy = _host_values(w.vy, M, "vy")
        keep += [vx, vy]
        op.vx, op.vy = _dptr(vx), _dptr(vy)
    if w.kind == "dense":
        A = _host_values(w.A, M * M, "A")
        keep.append(A)
        op.A = _dptr(A)
    desc = ProblemDesc(op, _dptr(y0), int(w.batch), float(w.T), int(w.N),
                       StepperDesc(PIT_STEP[w.fine[0]], int(w.fine[1])),
                       StepperDesc(PIT_STEP[w.coarse[0]], int(w.coarse[1]),
                                   int(getattr(w, "coarse_inner", 0))), precision)
    return desc, keep


def solve_opts(tol: float = 1e-10, eps0: float = 1e-8, max_iter: int = 500,
               x0: str = "coarse", refine_max: int = 8, inner_tol: float = 1e-4,
               tol_mode: str = "r0", residual_precision: str = "split") -> SolveOpts:
    opts = SolveOpts()
    load().pit_default_opts(C.byref(opts))
    opts.tol, opts.restart_eps0, opts.max_iter = tol, eps0, max_iter
    opts.x0_mode = X0[x0]
    opts.refine_max, opts.inner_tol = refine_max, inner_tol
    opts.tol_mode = TOL_MODE[tol_mode]
    opts.residual_precision = PRECISION[residual_precision]
    return opts


class Problem:
    """A libpit problem built from a workload (paper_2203_10148_gb300.inputs.Workload)."""

    def __init__(self, w, precision: Optional[str] = None):
        lib = load()
        self.w = w
        self.precision = PRECISION[precision or w.precision]
        desc, self._keep = problem_desc(w, self.precision)
        if self.precision == PIT_MIXED_BF16:     # a problem setting; applies run as mixed
            self.precision = PIT_MIXED
        h = C.c_void_p()
        check(lib.pit_problem_create(C.byref(desc), C.byref(h)))
        self.handle = h
        if getattr(w, "f", None) is not None:
            self.set_source(np.ascontiguousarray(np.asarray(w.f, dtype=np.float64).reshape(w.batch, -1)))
        self.M, self.N, self.batch = w.M, w.N, w.batch
        self.shape = (self.batch, self.N + 1, self.M)
        self._keep = []

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "handle", None):
            load().pit_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------- calls
    def _out_like(self, x):
        if isinstance(x, np.ndarray):
            return np.empty(self.shape, dtype=np.float64)
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device=x.device)

    def apply(self, which: str, x, precision: Optional[str] = None, out=None, stream=None):
        """pit_apply_operator: which in {'F', 'Ginv', 'GinvF', 'residual'}."""
        prec = self.precision if precision is None else PRECISION[precision]
        y = self._out_like(x) if out is None else out
        n = self.batch * (self.N + 1) * self.M
        px, dev, _ = _array_arg(x, n)
        py, dev2, _ = _array_arg(y, n)
        if dev != dev2:
            raise ValueError("x and y must both be host or both be device arrays")
        check(load().pit_apply_operator(self.handle, APPLY[which], prec, px, py, dev,
                                        _torch_stream(x, stream)))
        return y

    def serial_fine(self, precision: Optional[str] = None, out=None):
        prec = self.precision if precision is None else PRECISION[precision]
        y = np.empty(self.shape, dtype=np.float64) if out is None else out
        py, dev, _ = _array_arg(y, self.batch * (self.N + 1) * self.M)
        check(load().pit_serial_fine(self.handle, prec, py, dev))
        return y

    def bicgstab_solve(self, X=None, tol: float = 1e-10, eps0: float = 1e-8,
                       max_iter: int = 500, x0: str = "coarse", refine_max: int = 8,
                       inner_tol: float = 1e-4, history_len: int = 0, stream=None,
                       raise_on_status: bool = False, tol_mode: str = "r0",
                       residual_precision: str = "split"):
        """pit_bicgstab_solve; returns (X, [info dict per member])."""
        lib = load()
        opts = solve_opts(tol, eps0, max_iter, x0, refine_max, inner_tol, tol_mode,
                          residual_precision)
        hist = None
        if history_len:
            hist = np.zeros(history_len)
            opts.history = _dptr(hist)
            opts.history_len = history_len
        if X is None:
            X = np.zeros(self.shape)
        px, dev, _ = _array_arg(X, self.batch * (self.N + 1) * self.M)
        opts.stream = _torch_stream(X, stream)
        infos = (SolveInfo * self.batch)()
        st = lib.pit_bicgstab_solve(self.handle, C.byref(opts), px, dev, infos)
        if st in (PIT_E_INVALID, PIT_E_NOMEM, PIT_E_CUDA, PIT_E_UNSUPPORTED) or (raise_on_status and st < 0):
            check(st)
        out = [i.as_dict() for i in infos]
        if hist is not None:
            out[0]["history"] = hist[:out[0]["history_count"]].tolist()
        return X, out

    def set_y0(self, y0):
        """pit_problem_set_y0: new initial values (batch x M), host or device."""
        p, dev, _ = _array_arg(y0, self.batch * self.M)
        check(load().pit_problem_set_y0(self.handle, p, dev))

    def set_source(self, f):
        """pit_problem_set_source: time-independent source (batch x M) or None."""
        if f is None:
            check(load().pit_problem_set_source(self.handle, None, 0))
            return
        p, dev, _ = _array_arg(f, self.batch * self.M)
        check(load().pit_problem_set_source(self.handle, p, dev))

    def set_timing(self, enable=True):
        """pit_set_timing: True (or 1) times every operator class; 2 times the
        top-level launches and each launch of the BiCGStab iterations as a
        whole ("inner"), which then run as the uninstrumented loop graph."""
        check(load().pit_set_timing(self.handle, int(enable)))

    def timing(self) -> dict:
        """{class: (calls, milliseconds)} since set_timing(True)."""
        out = {}
        for name, cls in TIME_CLASSES.items():
            calls, ms = C.c_longlong(), C.c_double()
            check(load().pit_get_timing(self.handle, cls, C.byref(calls), C.byref(ms)))
            out[name] = (calls.value, ms.value)
        return out

    def parareal_solve(self, kmax: int, tol: float = 0.0, X=None):
        lib = load()
        if X is None:
            X = np.zeros(self.shape)
        px, dev, _ = _array_arg(X, self.batch * (self.N + 1) * self.M)
        infos = (SolveInfo * self.batch)()
        st = lib.pit_parareal_solve(self.handle, int(kmax), float(tol), px, dev, infos)
        if st in (PIT_E_INVALID, PIT_E_NOMEM, PIT_E_CUDA, PIT_E_UNSUPPORTED):
            check(st)
        return X, [i.as_dict() for i in infos]


class Server:
    """pit_server_*: continuous batching of solves submitted from any thread."""

    def __init__(self, hbm_budget_bytes: int = 0, max_slots: int = 4):
        h = C.c_void_p()
        check(load().pit_server_create(int(hbm_budget_bytes), int(max_slots), C.byref(h)))
        self.handle = h
        self._shapes = {}

    def close(self):
        if getattr(self, "handle", None):
            load().pit_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, w, precision: Optional[str] = None, **opts) -> int:
        """Queues workload ``w`` with solve options (as Problem.bicgstab_solve); a ticket."""
        if getattr(w, "f", None) is not None:
            raise ValueError("the server takes problems without a source term")
        desc, keep = problem_desc(w, PRECISION[precision or w.precision])
        o = solve_opts(**opts)
        t = C.c_uint64()
        check(load().pit_serve_submit(self.handle, C.byref(desc), C.byref(o), C.byref(t)))
        self._shapes[t.value] = (int(w.batch), int(w.N) + 1, int(w.M))
        del keep
        return t.value

    def _take(self, fn, ticket: int, *args):
        shape = self._shapes.get(ticket)
        if shape is None:   # not issued here, or taken: the library reports it
            info = SolveInfo()
            check(fn(self.handle, C.c_uint64(ticket), *args, None, C.byref(info)))
            return None
        X = np.empty(shape, dtype=np.float64)
        infos = (SolveInfo * shape[0])()
        st = fn(self.handle, C.c_uint64(ticket), *args, X.ctypes.data, infos)
        if st == PIT_PENDING:
            return None
        if st == PIT_E_INVALID:
            check(st)
        del self._shapes[ticket]
        out = [i.as_dict() for i in infos]
        if st != PIT_OK:
            msg = last_error()
            for d in out:
                d["error"] = msg
        return st, X, out

    def poll(self, ticket: int):
        """None while pending, else (status, X, [info per member])."""
        return self._take(load().pit_serve_poll, ticket)

    def wait(self, ticket: int, timeout: float = -1.0):
        """Blocks until done (or the timeout: None); as poll."""
        return self._take(load().pit_serve_wait, ticket, C.c_double(timeout))

    def cancel(self, ticket: int):
        check(load().pit_serve_cancel(self.handle, C.c_uint64(ticket)))

    def stats(self, reset: bool = False) -> dict:
        s = ServerStats()
        check(load().pit_server_stats(self.handle, int(reset), C.byref(s)))
        return s.as_dict()


def serve_footprint(w) -> int:
    """pit_serve_footprint: device bytes the server reserves for workload ``w``."""
    desc, keep = problem_desc(w, PRECISION[w.precision])
    b = C.c_size_t()
    check(load().pit_serve_footprint(C.byref(desc), C.byref(b)))
    return int(b.value)


def kernel_launches() -> int:
    return int(load().pit_kernel_launches())


def block_reduce(U, V, nblocks: int, M: int, noalloc: bool = False):
    """pit_block_reduce (or pit_block_reduce_noalloc) on CUDA tensors:
    (dot, per-block norms, max block norm)."""
    import torch
    pu, du, _ = _array_arg(U, nblocks * M)
    pv, dv, _ = _array_arg(V, nblocks * M)
    if not (du and dv):
        raise ValueError("pit_block_reduce takes device tensors")
    out = torch.zeros(2 + nblocks, dtype=torch.float64, device=U.device)
    base = out.data_ptr()
    fn = load().pit_block_reduce_noalloc if noalloc else load().pit_block_reduce
    check(fn(pu, pv, nblocks, M, base, base + 16, base + 8))
    o = out.cpu().numpy()
    return float(o[0]), o[2:], float(o[1])
