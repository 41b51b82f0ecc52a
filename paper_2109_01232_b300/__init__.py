"""Python binding of the B300 GMRES / GMRES-IR library (libgmres_ir.so).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Device memory comes from PyTorch tensors (their data pointers are
passed through the C ABI declared in include/gmres_ir.h) and streams from
torch.cuda.  There is no CPU fallback: if the shared library or a CUDA device
is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgmres_ir.so")

PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
CGS_KERNEL = {"register": 0, "tma": 1}
STATUS = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", 3: "NONFINITE", 4: "ERR_INVALID",
          5: "ERR_OOM", 6: "ERR_CUDA", 7: "ERR_TOO_LARGE", 8: "ERR_DEVICE_TIMEOUT"}
(OK, NOT_CONVERGED, BREAKDOWN, NONFINITE, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TOO_LARGE,
 ERR_DEVICE_TIMEOUT) = range(9)
STATUS_SOLVER = (NOT_CONVERGED, BREAKDOWN, NONFINITE)  # outcomes of a solve, not errors
MAX_RESTART = 512
MAX_BJ_BLOCK = 64
MAX_POLY_DEGREE = 96


class GmresError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})" + (f" [{detail}]" if detail else ""))
        self.code = code


class csr_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


class params_t(ctypes.Structure):
    _fields_ = [("restart_m", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("inner_rtol", ctypes.c_double), ("max_iters", ctypes.c_int64),
                ("inner_prec", ctypes.c_int32), ("poly_degree", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("record_history", ctypes.c_int32),
                ("cgs_kernel", ctypes.c_int32), ("poly_in_fp32", ctypes.c_int32),
                ("bj_block", ctypes.c_int32), ("bj_rcm", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("tma_wait_cycles", ctypes.c_int64),
                ("tma_test_withhold", ctypes.c_int32)]


class stats_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int64),
                ("outer_iters", ctypes.c_int32), ("rel_resid", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double), ("t_setup_ms", ctypes.c_double),
                ("history_len", ctypes.c_int64), ("history", ctypes.c_void_p),
                ("history_cap", ctypes.c_int64)]


class csr_batch_t(ctypes.Structure):
    _fields_ = [("nsys", ctypes.c_int32), ("row_off", ctypes.c_void_p), ("nnz_off", ctypes.c_void_p),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


class selector_t(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("feat_mean", ctypes.c_void_p),
                ("feat_scale", ctypes.c_void_p), ("class_m", ctypes.c_void_p),
                ("class_degree", ctypes.c_void_p), ("class_prec", ctypes.c_void_p),
                ("class_inner_rtol", ctypes.c_void_p), ("min_confidence", ctypes.c_float)]


class batch_stats_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_void_p), ("iters", ctypes.c_void_p), ("outer", ctypes.c_void_p),
                ("rel_resid", ctypes.c_void_p), ("t_solve_ms", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I32, _I64, _U64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_SIGNATURES = {
    "gmres_default_params": (None, [ctypes.POINTER(params_t)]),
    "gmres_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gmres_last_error": (ctypes.c_char_p, []),
    "gmres_solve": (ctypes.c_int, [ctypes.POINTER(csr_t), _P, _P, ctypes.POINTER(params_t),
                                   ctypes.POINTER(stats_t), _P]),
    "gmres_ir_solve": (ctypes.c_int, [ctypes.POINTER(csr_t), _P, _P, ctypes.POINTER(params_t),
                                      ctypes.POINTER(stats_t), _P]),
    "gmres_solve_host": (ctypes.c_int, [ctypes.POINTER(csr_t), _P, _P, ctypes.POINTER(params_t),
                                        ctypes.POINTER(stats_t), _P]),
    "gmres_ir_solve_host": (ctypes.c_int, [ctypes.POINTER(csr_t), _P, _P,
                                           ctypes.POINTER(params_t), ctypes.POINTER(stats_t), _P]),
    "gmres_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(csr_t), _I32,
                                         ctypes.POINTER(params_t), _P]),
    "gmres_plan_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(stats_t), _P]),
    "gmres_plan_destroy": (ctypes.c_int, [_P]),
    "gmres_plan_spmv": (ctypes.c_int, [_P, _P, _P, _P]),
    "gmres_plan_arnoldi": (ctypes.c_int, [_P, _P, _I32, _P, _P, ctypes.POINTER(_I32), _P]),
    "gmres_poly_roots": (ctypes.c_int, [ctypes.POINTER(csr_t), _I32, _U64, _P, _P, _P,
                                        ctypes.POINTER(_I32), _P]),
    "gmres_splitmix64_fill": (ctypes.c_int, [_P, _I64, _U64, _P]),
    "gmres_plan_profile_cycle": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gmres_plan_profile_cycle_graph": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gmres_plan_time_cycle_graph": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gmres_plan_info": (ctypes.c_int, [_P, _P]),
    "gmres_plan_poly_apply": (ctypes.c_int, [_P, _P, _P, _P]),
    "gmres_plan_poly_roots": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_I32)]),
    "gmres_plan_bj_apply": (ctypes.c_int, [_P, _P, _P, _P]),
    "gmres_plan_perm": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I32)]),
    "gmres_rcm": (ctypes.c_int, [_I32, _P, _P, _P]),
    "gmres_spmv_fp64_noalloc": (ctypes.c_int, [ctypes.POINTER(csr_t), _P, _P, _P]),
    "gmres_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(csr_batch_t),
                                               ctypes.POINTER(params_t), _I32, _P]),
    "gmres_batch_plan_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(batch_stats_t), _P]),
    "gmres_batch_plan_info": (ctypes.c_int, [_P, _P]),
    "gmres_batch_plan_destroy": (ctypes.c_int, [_P]),
    "gmres_fd_solve": (ctypes.c_int, [ctypes.POINTER(csr_t), _P, _P, ctypes.POINTER(params_t), _I64,
                                      ctypes.POINTER(stats_t), ctypes.POINTER(stats_t), _P]),
    "gmres_matrix_features": (ctypes.c_int, [ctypes.POINTER(csr_t), _P, _P]),
    "gmres_mlp_forward": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "gmres_mlp_loss_grad": (ctypes.c_int, [_P, _P, _P, _I32, _P, _P, _P]),
    "gmres_mlp_train": (ctypes.c_int, [_P, _P, _P, _I32, _I32, ctypes.c_float, _P, _P]),
    "gmres_select_params": (ctypes.c_int, [ctypes.POINTER(csr_t), ctypes.POINTER(selector_t),
                                           ctypes.POINTER(params_t), _P, _P, _P]),
    "gmres_plan_set_tolerances": (ctypes.c_int, [_P, _D, _D, _I64]),
    "gmres_plan_spmv_timed": (ctypes.c_int, [_P, _P, _P, _I32, _P, _P]),
    "gmres_ir_solve_batched": (ctypes.c_int, [ctypes.POINTER(csr_batch_t), _P, _P,
                                              ctypes.POINTER(params_t),
                                              ctypes.POINTER(batch_stats_t), _P]),
}
NOALLOC_MAX_N = 1 << 20


def lib() -> ctypes.CDLL:
    """Load libgmres_ir.so (built in-tree by paper_2109_01232_b300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python paper_2109_01232_b300/build.py`")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the GMRES library needs a CUDA device (none is visible)")
    return torch


def _stream(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr())


def _check(code: int, what: str, allowed=(OK,)):
    if code not in allowed:
        detail = ""
        if code in (ERR_CUDA, ERR_OOM) and _lib is not None:
            detail = (_lib.gmres_last_error() or b"").decode(errors="replace")
        raise GmresError(code, what, detail)
    return code


def default_params(**kw) -> params_t:
    p = params_t()
    lib().gmres_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "inner_prec" and isinstance(v, str):
            v = PREC[v]
        if k == "cgs_kernel" and isinstance(v, str):
            v = CGS_KERNEL[v]
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


class DeviceCSR:
    """CSR matrix on the device (int32 indices, FP64 values) backed by torch tensors."""

    def __init__(self, row_ptr, col_idx, vals, n: int | None = None):
        torch = _torch()
        self.row_ptr = torch.as_tensor(row_ptr, dtype=torch.int32, device="cuda").contiguous()
        self.col_idx = torch.as_tensor(col_idx, dtype=torch.int32, device="cuda").contiguous()
        self.vals = torch.as_tensor(vals, dtype=torch.float64, device="cuda").contiguous()
        self.n = int(n if n is not None else self.row_ptr.numel() - 1)
        self.nnz = int(self.vals.numel())

    @classmethod
    def from_problem(cls, p) -> "DeviceCSR":
        return cls(p.row_ptr, p.col_idx, p.vals, p.n)

    def c(self) -> csr_t:
        return csr_t(self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx), _ptr(self.vals))


@dataclass
class SolveResult:
    status: int
    iters: int
    outer: int
    relres: float
    t_solve_ms: float
    t_setup_ms: float
    history: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def status_name(self) -> str:
        return STATUS[self.status]


def _result(code: int, st: stats_t, hist: np.ndarray | None) -> SolveResult:
    _check(code, "solve", (OK, NOT_CONVERGED, BREAKDOWN, NONFINITE))
    h = hist[:st.history_len].copy() if hist is not None else np.zeros(0)
    return SolveResult(code, int(st.iters), int(st.outer_iters), float(st.rel_resid),
                       float(st.t_solve_ms), float(st.t_setup_ms), h)


def _stats(params: params_t):
    st = stats_t()
    hist = None
    if params.record_history:
        hist = np.zeros(max(int(params.max_iters), 1), dtype=np.float64)
        st.history = hist.ctypes.data
        st.history_cap = hist.size
    return st, hist


def _solve(fn_name: str, A: DeviceCSR, b, x, stream=None, **kw) -> SolveResult:
    p = default_params(**kw)
    st, hist = _stats(p)
    c = A.c()
    code = getattr(lib(), fn_name)(ctypes.byref(c), _ptr(b), _ptr(x), ctypes.byref(p),
                                   ctypes.byref(st), _stream(stream))
    return _result(code, st, hist)


def gmres_solve(A: DeviceCSR, b, x, stream=None, **kw) -> SolveResult:
    """FP64 GMRES(m) (Algorithm 1, CGS2).  b, x: float64 CUDA tensors; x is updated."""
    return _solve("gmres_solve", A, b, x, stream, **kw)


def gmres_ir_solve(A: DeviceCSR, b, x, stream=None, **kw) -> SolveResult:
    """GMRES-IR (Algorithm 2) with inner precision kw['inner_prec'] ('fp32' default)."""
    return _solve("gmres_ir_solve", A, b, x, stream, **kw)


def _solve_host(fn_name, row_ptr, col_idx, vals, b, x, stream=None, **kw) -> SolveResult:
    """Host-memory variant: numpy (or pinned torch CPU) arrays; x is updated in place."""
    p = default_params(**kw)
    st, hist = _stats(p)
    def host(a, dtype):  # torch CPU tensors (e.g. pinned) are passed without a copy
        if hasattr(a, "data_ptr"):
            return a, int(a.data_ptr()), int(a.numel())
        a = np.ascontiguousarray(a, dtype)
        return a, a.ctypes.data, a.size

    keep = [host(row_ptr, np.int32), host(col_idx, np.int32), host(vals, np.float64)]
    c = csr_t(keep[0][2] - 1, keep[2][2], keep[0][1], keep[1][1], keep[2][1])
    bp = b.data_ptr() if hasattr(b, "data_ptr") else b.ctypes.data
    xp = x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
    code = getattr(lib(), fn_name)(ctypes.byref(c), bp, xp, ctypes.byref(p), ctypes.byref(st),
                                   _stream(stream))
    return _result(code, st, hist)


def gmres_ir_solve_host(row_ptr, col_idx, vals, b, x, stream=None, **kw) -> SolveResult:
    return _solve_host("gmres_ir_solve_host", row_ptr, col_idx, vals, b, x, stream, **kw)


def gmres_solve_host(row_ptr, col_idx, vals, b, x, stream=None, **kw) -> SolveResult:
    return _solve_host("gmres_solve_host", row_ptr, col_idx, vals, b, x, stream, **kw)


class Plan:
    """Reusable solver workspace + captured cycle graph for one matrix.

    kind: 'gmres' (FP64 GMRES), 'ir' (GMRES-IR with inner_prec) or 'fp32' (GMRES entirely
    in single precision, GMRES-FD's first stage)."""

    def __init__(self, A: DeviceCSR, kind: str = "ir", stream=None, **kw):
        self.A = A
        self.params = default_params(**kw)
        self.kind = {"gmres": 0, "ir": 1, "fp32": 2}[kind]
        self.prec = 0 if self.kind == 0 else (1 if self.kind == 2 else self.params.inner_prec)
        h = ctypes.c_void_p()
        c = A.c()
        _check(lib().gmres_plan_create(ctypes.byref(h), ctypes.byref(c), self.kind,
                                       ctypes.byref(self.params), _stream(stream)), "plan_create")
        self.handle = h

    @property
    def storage_dtype(self):
        torch = _torch()
        return {0: torch.float64, 1: torch.float32, 2: torch.float16, 3: torch.bfloat16}[self.prec]

    @property
    def work_dtype(self):
        torch = _torch()
        return torch.float64 if self.prec == 0 else torch.float32

    def spmv_timed(self, x, reps: int = 1000, stream=None):
        """(y = A x, mean ms per SpMV) with the plan's inner copy of A alone; x in the working
        dtype."""
        torch = _torch()
        y = torch.empty(self.A.n, dtype=self.work_dtype, device="cuda")
        ms = ctypes.c_float(0.0)
        _check(lib().gmres_plan_spmv_timed(self.handle, _ptr(x), _ptr(y), int(reps), ctypes.byref(ms),
                                           _stream(stream)), "spmv_timed")
        return y, float(ms.value)

    def set_tolerances(self, rtol: float, inner_rtol: float, max_iters: int):
        _check(lib().gmres_plan_set_tolerances(self.handle, rtol, inner_rtol, max_iters),
               "plan_set_tolerances")
        self.params.rtol, self.params.inner_rtol, self.params.max_iters = rtol, inner_rtol, max_iters

    def solve(self, b, x, stream=None) -> SolveResult:
        st, hist = _stats(self.params)
        code = lib().gmres_plan_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(st),
                                      _stream(stream))
        return _result(code, st, hist)

    def spmv(self, v, stream=None):
        torch = _torch()
        y = torch.empty(self.A.n, dtype=self.work_dtype, device="cuda")
        _check(lib().gmres_plan_spmv(self.handle, _ptr(v), _ptr(y), _stream(stream)), "spmv")
        return y

    def arnoldi(self, v0, steps: int, stream=None):
        """Returns (V (steps+1, n) tensor in the storage dtype, H numpy (steps+1, steps), k)."""
        torch = _torch()
        V = torch.zeros((steps + 1, self.A.n), dtype=self.storage_dtype, device="cuda")
        H = np.zeros((steps, steps + 1), dtype=np.float64)  # column-major (steps+1) x steps
        k = ctypes.c_int32(0)
        _check(lib().gmres_plan_arnoldi(self.handle, _ptr(v0), steps, _ptr(V), H.ctypes.data,
                                        ctypes.byref(k), _stream(stream)), "arnoldi")
        return V, H.T.copy(), int(k.value)

    def poly_apply(self, v, stream=None):
        """y = p(A) v with the plan's GMRES polynomial (the polynomial's working dtype)."""
        torch = _torch()
        dt = torch.float32 if (self.prec == 0 and self.params.poly_in_fp32) else self.work_dtype
        y = torch.empty(self.A.n, dtype=dt, device="cuda")
        _check(lib().gmres_plan_poly_apply(self.handle, _ptr(v), _ptr(y), _stream(stream)),
               "poly_apply")
        return y

    def bj_apply(self, v, stream=None):
        """y = M^{-1} v with the plan's block-Jacobi factors (working dtype; the plan's
        numbering, i.e. reordered when the plan was created with bj_rcm)."""
        torch = _torch()
        y = torch.empty(self.A.n, dtype=self.work_dtype, device="cuda")
        _check(lib().gmres_plan_bj_apply(self.handle, _ptr(v), _ptr(y), _stream(stream)),
               "bj_apply")
        return y

    def perm(self) -> np.ndarray | None:
        """perm[new] = old of the plan's reverse Cuthill-McKee reordering, or None."""
        out = np.zeros(max(self.A.n, 1), dtype=np.int32)
        flag = ctypes.c_int32(0)
        _check(lib().gmres_plan_perm(self.handle, out.ctypes.data, ctypes.byref(flag)), "perm")
        return out[:self.A.n] if flag.value else None

    def roots(self) -> np.ndarray:
        n = ctypes.c_int32(0)
        _check(lib().gmres_plan_poly_roots(self.handle, None, None, ctypes.byref(n)), "roots")
        re, im = np.zeros(n.value), np.zeros(n.value)
        _check(lib().gmres_plan_poly_roots(self.handle, re.ctypes.data, im.ctypes.data,
                                           ctypes.byref(n)), "roots")
        return re + 1j * im

    def info(self) -> dict:
        out = np.zeros(8, dtype=np.int64)
        _check(lib().gmres_plan_info(self.handle, out.ctypes.data), "plan_info")
        keys = ["n", "nnz", "ld", "m", "prec", "grid_spmv", "grid_vec", "grid_res"]
        return dict(zip(keys, map(int, out)))

    def profile_cycle(self, b, x0, stream=None, graph: bool = False) -> np.ndarray:
        """Per-launch device times (ms) of one cycle, shape (m+1, 3): row j = (SpMV, first CGS
        update, second CGS update) of step j, last row = (least squares, x update, residual);
        -1 where the cycle ended earlier.  graph=False: kernels launched one by one with events
        around each; graph=True: event-record nodes inside a captured graph of the cycle."""
        m = int(self.params.restart_m)
        out = np.zeros(3 * m + 3, dtype=np.float64)
        fn = lib().gmres_plan_profile_cycle_graph if graph else lib().gmres_plan_profile_cycle
        _check(fn(self.handle, _ptr(b), _ptr(x0), out.ctypes.data, _stream(stream)), "profile_cycle")
        return out.reshape(m + 1, 3)

    def time_cycle(self, b, x0, stream=None) -> tuple:
        """(ms, steps) of one cycle run as a captured graph with events only at its two ends
        (no event node between kernels)."""
        out = np.zeros(2, dtype=np.float64)
        _check(lib().gmres_plan_time_cycle_graph(self.handle, _ptr(b), _ptr(x0), out.ctypes.data,
                                                 _stream(stream)), "time_cycle")
        return float(out[0]), int(out[1])

    def close(self):
        if self.handle:
            lib().gmres_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poly_roots(A: DeviceCSR, degree: int, seed: int = 0, v0=None, stream=None) -> np.ndarray:
    """Leja-ordered roots of the GMRES polynomial of the given degree (complex numpy array)."""
    re = np.zeros(degree + 1)
    im = np.zeros(degree + 1)
    nr = ctypes.c_int32(0)
    c = A.c()
    _check(lib().gmres_poly_roots(ctypes.byref(c), degree, seed, _ptr(v0) if v0 is not None else None,
                                  re.ctypes.data, im.ctypes.data, ctypes.byref(nr),
                                  _stream(stream)), "poly_roots")
    return re[:nr.value] + 1j * im[:nr.value]


def rcm(row_ptr, col_idx, n: int | None = None) -> np.ndarray:
    """Reverse Cuthill-McKee permutation (perm[new] = old) of a CSR structure, computed by
    the library on the host (no GPU needed)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    n = int(rp.size - 1 if n is None else n)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().gmres_rcm(n, rp.ctypes.data, ci.ctypes.data, perm.ctypes.data), "rcm")
    return perm[:n]


def splitmix64(n: int, seed: int, stream=None):
    """SplitMix64 vector in [-1, 1) computed on the device."""
    torch = _torch()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(lib().gmres_splitmix64_fill(_ptr(out), n, seed, _stream(stream)), "splitmix64")
    return out


def spmv_fp64_noalloc(A: DeviceCSR, v, y, stream=None) -> None:
    """y = A v in FP64 through gmres_spmv_fp64_noalloc, which allocates no device memory
    (for callers whose GPU memory belongs to another allocator or that must not trigger
    cudaMalloc's implicit synchronisation).  v, y: contiguous float64 CUDA tensors of at
    least n entries on the current device; y may be v (in place).  Synchronous."""
    torch = _torch()
    dev = torch.cuda.current_device()
    for name, t in (("v", v), ("y", y)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise ValueError(f"{name} must be a float64 CUDA tensor")
        if t.device.index != dev or not t.is_contiguous() or t.numel() < A.n:
            raise ValueError(f"{name} must be contiguous, on the current device, with >= n entries")
    c = A.c()
    _check(lib().gmres_spmv_fp64_noalloc(ctypes.byref(c), _ptr(v), _ptr(y), _stream(stream)),
           "spmv_fp64_noalloc")


# ------------------------------------------------------------------ batched ----
BATCH_MAX_M = 32


class DeviceBatch:
    """Many independent CSR systems concatenated for the batched solver: the local row
    pointers of system i start at row_ptr[row_off[i] + i], its column indices are local."""

    def __init__(self, problems):
        import numpy as np
        torch = _torch()
        ns = [int(p.n) for p in problems]
        zs = [int(len(p.vals)) for p in problems]
        self.nsys = len(problems)
        self.row_off = np.zeros(self.nsys + 1, dtype=np.int64)
        self.nnz_off = np.zeros(self.nsys + 1, dtype=np.int64)
        np.cumsum(ns, out=self.row_off[1:])
        np.cumsum(zs, out=self.nnz_off[1:])
        cat = lambda xs, dt: np.concatenate([np.asarray(x, dtype=dt) for x in xs]) if xs else np.zeros(0, dt)
        self.row_ptr = torch.as_tensor(cat([p.row_ptr for p in problems], np.int32), device="cuda")
        self.col_idx = torch.as_tensor(cat([p.col_idx for p in problems], np.int32), device="cuda")
        self.vals = torch.as_tensor(cat([p.vals for p in problems], np.float64), device="cuda")
        self.rows = int(self.row_off[-1])

    def c(self) -> csr_batch_t:
        return csr_batch_t(self.nsys, self.row_off.ctypes.data, self.nnz_off.ctypes.data,
                           _ptr(self.row_ptr), _ptr(self.col_idx), _ptr(self.vals))

    def split(self, v):
        """Per-system views of a concatenated vector."""
        return [v[int(self.row_off[i]):int(self.row_off[i + 1])] for i in range(self.nsys)]


class BatchResult:
    def __init__(self, code, status, iters, outer, relres, ms):
        self.code, self.status, self.iters, self.outer = code, status, iters, outer
        self.rel_resid, self.t_solve_ms = relres, ms


class BatchPlan:
    """Batched GMRES-IR plan: one persistent, graph-captured kernel for all systems."""

    def __init__(self, batch: DeviceBatch, autotune: bool = True, stream=None, **kw):
        self.batch = batch
        kw.setdefault("restart_m", 30)  # the batched kernel keeps at most BATCH_MAX_M columns
        self.params = default_params(**kw)
        h = ctypes.c_void_p()
        c = batch.c()
        _check(lib().gmres_batch_plan_create(ctypes.byref(h), ctypes.byref(c),
                                             ctypes.byref(self.params), int(bool(autotune)),
                                             _stream(stream)), "batch_plan_create")
        self.handle = h

    def info(self) -> dict:
        import numpy as np
        out = np.zeros(7, dtype=np.int64)
        _check(lib().gmres_batch_plan_info(self.handle, out.ctypes.data), "batch_plan_info")
        keys = ("threads", "ctas", "candidates_timed", "max_rows", "ld", "prec", "cluster")
        return dict(zip(keys, map(int, out)))

    def solve(self, b, x, stream=None, allowed=(OK,)) -> BatchResult:
        import numpy as np
        n = self.batch.nsys
        st = np.zeros(n, np.int32); it = np.zeros(n, np.int64)
        ou = np.zeros(n, np.int32); rr = np.zeros(n, np.float64)
        s = batch_stats_t(st.ctypes.data, it.ctypes.data, ou.ctypes.data, rr.ctypes.data, 0.0)
        code = lib().gmres_batch_plan_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(s),
                                            _stream(stream))
        _check(code, "batch_plan_solve", allowed=tuple(allowed) + STATUS_SOLVER)
        return BatchResult(code, st, it, ou, rr, s.t_solve_ms)

    def close(self):
        if getattr(self, "handle", None):
            lib().gmres_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ir_solve_batched(batch: DeviceBatch, b, x, stream=None, **kw) -> BatchResult:
    """One-shot batched GMRES-IR (plan without autotuning, solve, destroy)."""
    import numpy as np
    kw.setdefault("restart_m", 30)
    params = default_params(**kw)
    n = batch.nsys
    st = np.zeros(n, np.int32); it = np.zeros(n, np.int64)
    ou = np.zeros(n, np.int32); rr = np.zeros(n, np.float64)
    s = batch_stats_t(st.ctypes.data, it.ctypes.data, ou.ctypes.data, rr.ctypes.data, 0.0)
    c = batch.c()
    code = lib().gmres_ir_solve_batched(ctypes.byref(c), _ptr(b), _ptr(x), ctypes.byref(params),
                                        ctypes.byref(s), _stream(stream))
    _check(code, "ir_solve_batched", allowed=(OK,) + STATUS_SOLVER)
    return BatchResult(code, st, it, ou, rr, s.t_solve_ms)


# ----------------------------------------------------------------- selector ----
SEL_FEATURES, SEL_CLASSES, SEL_PARAMS = 16, 32, 7328


def _f32(a, n=None):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def matrix_features(A: DeviceCSR, stream=None):
    """The 16 selector features of A (gmres_matrix_features), float32."""
    import numpy as np
    out = np.zeros(SEL_FEATURES, np.float32)
    c = A.c()
    _check(lib().gmres_matrix_features(ctypes.byref(c), out.ctypes.data, _stream(stream)), "features")
    return out


def mlp_forward(params, X, stream=None):
    import numpy as np
    params, X = _f32(params, SEL_PARAMS), _f32(X)
    B = X.size // SEL_FEATURES
    out = np.zeros((B, SEL_CLASSES), np.float32)
    _check(lib().gmres_mlp_forward(params.ctypes.data, X.ctypes.data, B, out.ctypes.data,
                                   _stream(stream)), "mlp_forward")
    return out


def mlp_loss_grad(params, X, labels, stream=None):
    import numpy as np
    params, X = _f32(params, SEL_PARAMS), _f32(X)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    loss = np.zeros(1, np.float32)
    grad = np.zeros(SEL_PARAMS, np.float32)
    _check(lib().gmres_mlp_loss_grad(params.ctypes.data, X.ctypes.data, lab.ctypes.data, lab.size,
                                     loss.ctypes.data, grad.ctypes.data, _stream(stream)), "mlp_loss_grad")
    return float(loss[0]), grad


def mlp_train(params0, X, labels, epochs: int, lr: float, stream=None):
    """Full-batch Adam on the GPU (gmres_mlp_train); returns (params, losses)."""
    import numpy as np
    params = _f32(params0, SEL_PARAMS).copy()
    X = _f32(X)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    losses = np.zeros(max(epochs, 1), np.float32)
    _check(lib().gmres_mlp_train(params.ctypes.data, X.ctypes.data, lab.ctypes.data, lab.size, epochs,
                                 float(lr), losses.ctypes.data, _stream(stream)), "mlp_train")
    return params, losses[:epochs]


class Selector:
    """A trained selector model (arrays as saved by selector.save_model); None = default only."""

    def __init__(self, model: dict | None):
        import numpy as np
        self.model = model
        self._keep = []
        if model is None:
            self.c = None
            return
        arr = lambda k, dt: self._keep.append(np.ascontiguousarray(model[k], dtype=dt)) or self._keep[-1]
        self.c = selector_t(arr("params", np.float32).ctypes.data, arr("feat_mean", np.float32).ctypes.data,
                            arr("feat_scale", np.float32).ctypes.data, arr("class_m", np.int32).ctypes.data,
                            arr("class_degree", np.int32).ctypes.data, arr("class_prec", np.int32).ctypes.data,
                            arr("class_inner_rtol", np.float64).ctypes.data,
                            float(model.get("min_confidence", 0.0)))

    def choose(self, A: DeviceCSR, stream=None, **kw):
        """gmres_params for A: the selector's choice (or the default) on top of kw."""
        p = default_params(**kw)
        cls = ctypes.c_int32(-1)
        conf = ctypes.c_float(0.0)
        c = A.c()
        _check(lib().gmres_select_params(ctypes.byref(c), ctypes.byref(self.c) if self.c else None,
                                         ctypes.byref(p), ctypes.byref(cls), ctypes.byref(conf),
                                         _stream(stream)), "select_params")
        return p, int(cls.value), float(conf.value)


def gmres_fd_solve(A: DeviceCSR, b, x, switch_iters: int, stream=None, **kw):
    """GMRES-FD (Section 3.3): FP32 GMRES for switch_iters iterations (rounded up to whole
    cycles), then FP64 GMRES from that iterate.  Returns (fp32 stage, fp64 stage) results."""
    p = default_params(**kw)
    s32, h32 = _stats(p)
    s64, h64 = _stats(p)
    c = A.c()
    code = lib().gmres_fd_solve(ctypes.byref(c), _ptr(b), _ptr(x), ctypes.byref(p), int(switch_iters),
                                ctypes.byref(s32), ctypes.byref(s64), _stream(stream))
    r64 = _result(code, s64, h64)
    r32 = SolveResult(int(s32.status), int(s32.iters), int(s32.outer_iters), float(s32.rel_resid),
                      float(s32.t_solve_ms), float(s32.t_setup_ms))
    return r32, r64
