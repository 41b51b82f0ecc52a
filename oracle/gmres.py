"""Plain CPU reference ("oracle") for GMRES(m), GMRES-IR and GMRES-FD.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg import this module.  It shares no code with the
CUDA library and imports nothing from it.  Everything here is FP64 numpy,
written for readability: one Arnoldi step at a time, library matmuls for the
dot products, no blocking or fusion.

Method (Loe, Glusa, Yamazaki, Boman, Rajamanickam, "A Study of Mixed Precision
Strategies for GMRES on GPUs", arXiv 2109.01232):

* Algorithm 1, GMRES(m): r0 = b - A x0, gamma = ||r0||, v1 = r0/gamma; for
  j = 1..m: w = A v_j, H[:, j] = V_j^T w, w -= V_j H[:, j], h_{j+1,j} = ||w||,
  v_{j+1} = w / h_{j+1,j}; then y = argmin ||gamma e1 - Hbar y||, x += V y and
  restart from the explicit residual.
* Section 3.1: orthogonalisation is CGS2, i.e. the two lines "H = V^T w;
  w -= V H" are executed twice and the two coefficient vectors are summed.
* Algorithm 2, GMRES-IR: r = b - A x in FP64, GMRES(m) solves A u = r in low
  precision, x += u in FP64, repeat until ||b - A x|| / ||b|| <= tol.  The
  outer test happens only at a restart (Section 3.2).
* Section 3.3, GMRES-FD: FP32 GMRES(m) up to a restart, then FP64 GMRES(m)
  continuing from that x.
* Section 3.4: right preconditioning A M^{-1} (M x) = b with M^{-1} = p(A)
  (see oracle/poly.py), or any M^{-1} given as a function (`right_prec`: block
  Jacobi, see oracle/precond.py), whose result is rounded to the working precision.

Readings where the paper is silent:
* Convergence is measured by the explicit ||b - A x||_2 / ||b||_2 (Section
  3.1's definition).  FP64 GMRES ends a cycle early when the implicit residual
  |g_{j+1}| (Givens) reaches rtol*||b||, then confirms with the explicit one.
* The least-squares right-hand side is e1 (unit) and the cycle's correction is
  gamma * V y, with gamma applied in FP64; this is the same y scaled by 1/gamma.
* Givens rotations: rho = hypot(a, b), c = a/rho, s = b/rho; (c, s) = (1, 0)
  when b == 0.  g_{j+1} = -s g_j, g_j = c g_j.
* Lucky breakdown: h_{j+1,j} <= 16 u ||A v_j|| with u the unit roundoff of the
  working precision; the cycle then ends with j columns.
* A singular triangular factor (|R_kk| <= 16 u max|R|) drops the last column
  and reports BREAKDOWN.
* IR inner cycle: one cycle per refinement step.  inner_rtol = 0 runs the full
  m steps (the paper's behaviour: IR iteration counts are multiples of m);
  inner_rtol > 0 ends the cycle when |g_{j+1}| <= inner_rtol.
* Low-precision storage (IR): the copy of A is stored as round(A / s_A) and
  basis vectors as round(s_v v) / s_v, with s_A = max|a_ij| and s_v the largest
  power of two with s_v^2 <= 2n (within a factor sqrt(2) of sqrt(n): the entries of
  a unit vector, ~1/sqrt(n), are held near 1) for FP16 and s_A = s_v = 1 otherwise;
  products accumulate in FP32.  Scaling by a power of two adds no rounding.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .lowprec import round_to, unit_roundoff

OK, NOT_CONVERGED, BREAKDOWN, NONFINITE, INVALID = 0, 1, 2, 3, 4


# --------------------------------------------------------------------------
# Sparse matrix-vector product (Algorithm 1, "w_j = A v_j")
# --------------------------------------------------------------------------

def spmv(A, x: np.ndarray, vals: np.ndarray | None = None) -> np.ndarray:
    """y_i = sum over the CSR entries p of row i of vals[p] * x[col[p]], summed in FP64 in
    CSR order.  `A` has attributes n, row_ptr, col_idx, vals; `vals` overrides the values."""
    v = A.vals if vals is None else vals
    x = np.asarray(x, dtype=np.float64)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return np.bincount(rows, weights=v * x[A.col_idx], minlength=A.n)


def dense(A) -> np.ndarray:
    """Dense copy of a CSR matrix (small cases only)."""
    M = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    np.add.at(M, (rows, A.col_idx), A.vals)
    return M


# --------------------------------------------------------------------------
# Precision model of the inner solver
# --------------------------------------------------------------------------

def vector_scale(n: int) -> float:
    """FP16 basis scale: the largest power of two s with s^2 <= 2n (exact integers)."""
    k = ((2 * max(int(n), 1)).bit_length() - 1) // 2
    return float(2 ** k)



@dataclass
class Precision:
    """Storage format of the Krylov basis and of the low-precision copy of A, plus the
    precision that vector-operation results are rounded to ('work')."""

    storage: str = "fp64"  # fp64 | fp32 | fp16 | bf16
    work: str = "fp64"  # fp64 | fp32
    n: int = 1
    s_A: float = 1.0
    s_v: float = 1.0

    @staticmethod
    def for_inner(storage: str, A, arith: str = "fp32") -> "Precision":
        """IR inner precision.  arith='fp32' rounds every vector result to FP32 (FP32
        accumulation); arith='fp64' keeps FP64 arithmetic and rounds only stored values."""
        work = "fp64" if storage == "fp64" else ("fp32" if arith == "fp32" else "fp64")
        s_A, s_v = 1.0, 1.0
        if storage == "fp16":
            s_A = float(np.max(np.abs(A.vals))) if A.vals.size else 1.0
            s_v = vector_scale(A.n)
        return Precision(storage, work, A.n, s_A, s_v)

    def store_vector(self, v: np.ndarray) -> np.ndarray:
        if self.storage == "fp64":
            return np.asarray(v, dtype=np.float64).copy()
        return round_to(np.asarray(v) * self.s_v, self.storage) / self.s_v

    def matrix_values(self, vals: np.ndarray) -> np.ndarray:
        """Stored (scaled, rounded) values of the low-precision copy of A."""
        if self.storage == "fp64":
            return np.asarray(vals, dtype=np.float64).copy()
        return round_to(np.asarray(vals) / self.s_A, self.storage)

    def rw(self, x):
        """Round a vector-operation result to the working precision."""
        return round_to(x, self.work) if self.work != "fp64" else np.asarray(x, dtype=np.float64)

    @property
    def u_work(self) -> float:
        return unit_roundoff(self.work)


FP64 = None  # sentinel: plain double precision everywhere


def _fp64(n: int) -> Precision:
    return Precision("fp64", "fp64", n)


# --------------------------------------------------------------------------
# Arnoldi with CGS2 and Givens least squares (Algorithm 1 steps 4-12)
# --------------------------------------------------------------------------

def cgs2(Vj: np.ndarray, w: np.ndarray, prec: Precision) -> tuple[np.ndarray, np.ndarray]:
    """Section 3.1: two classical Gram-Schmidt passes of w against the columns of Vj.
    Each pass is h = Vj^T w (transposed GEMV) then w = w - Vj h (plain GEMV).
    Returns (h1 + h2, w)."""
    h1 = prec.rw(Vj.T @ w)
    w = prec.rw(w - Vj @ h1)
    h2 = prec.rw(Vj.T @ w)
    w = prec.rw(w - Vj @ h2)
    return h1 + h2, w


def givens(a: float, b: float) -> tuple[float, float]:
    """Rotation (c, s) with [c s; -s c] [a; b] = [rho; 0], rho = hypot(a, b) >= 0."""
    if b == 0.0:
        return 1.0, 0.0
    rho = float(np.hypot(a, b))
    return a / rho, b / rho


def back_substitute(R: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Solve the upper-triangular R y = g from the last row up."""
    k = len(g)
    y = np.zeros(k)
    for i in reversed(range(k)):
        y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:k]) / R[i, i]
    return y


@dataclass
class Cycle:
    V: np.ndarray  # n x (k+1) basis actually built (last column zero after a breakdown)
    Hbar: np.ndarray  # (k+1) x k Hessenberg matrix before rotation
    R: np.ndarray  # k x k triangular factor after the rotations
    g: np.ndarray  # rotated right-hand side (length k+1), g[0] started at 1
    y: np.ndarray  # least-squares solution (length k, or k-1 after a singular factor)
    k: int  # Arnoldi steps taken
    gamma: float  # ||r|| of the cycle's right-hand side
    hist: list = field(default_factory=list)  # |g_{j+1}| after each step (relative to gamma)
    breakdown: bool = False
    singular: bool = False


def gmres_cycle(op, r: np.ndarray, m: int, stop_rel: float, prec: Precision) -> Cycle:
    """One restart cycle of GMRES(m) for op(u) = r, with the least-squares right-hand side
    e1 (so the correction is gamma * V y).  Ends after m steps, at a lucky breakdown, or when
    the implicit relative residual |g_{j+1}| <= stop_rel."""
    n = r.shape[0]
    gamma = float(np.linalg.norm(r))
    V = np.zeros((n, m + 1))
    Hbar = np.zeros((m + 1, m))
    R = np.zeros((m + 1, m))
    cs, sn = np.zeros(m), np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = 1.0
    V[:, 0] = prec.store_vector(r / gamma)
    hist, k, breakdown = [], 0, False
    for j in range(m):
        w = prec.rw(op(V[:, j]))
        wnorm = float(np.linalg.norm(w))
        h, w = cgs2(V[:, :j + 1], w, prec)
        hn = float(prec.rw(np.linalg.norm(w)))
        Hbar[:j + 1, j] = h
        Hbar[j + 1, j] = hn
        col = Hbar[:j + 2, j].copy()
        for i in range(j):  # previous rotations
            t = cs[i] * col[i] + sn[i] * col[i + 1]
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
            col[i] = t
        c, s = givens(col[j], col[j + 1])
        col[j] = c * col[j] + s * col[j + 1]
        col[j + 1] = 0.0
        cs[j], sn[j] = c, s
        R[:j + 2, j] = col
        g[j + 1] = -s * g[j]
        g[j] = c * g[j]
        k = j + 1
        hist.append(abs(g[j + 1]))
        if hn <= 16.0 * prec.u_work * wnorm:
            breakdown = True
            break
        V[:, j + 1] = prec.store_vector(w / hn)
        if abs(g[j + 1]) <= stop_rel:
            break
    Rk = R[:k, :k]
    kk, singular = k, False
    rmax = float(np.max(np.abs(Rk))) if k else 0.0
    while kk > 0 and abs(Rk[kk - 1, kk - 1]) <= 16.0 * prec.u_work * rmax:
        kk -= 1
        singular = True
    y = back_substitute(Rk[:kk, :kk], g[:kk]) if kk else np.zeros(0)
    return Cycle(V=V[:, :k + 1], Hbar=Hbar[:k + 1, :k], R=Rk, g=g[:k + 1], y=y, k=k,
                 gamma=gamma, hist=hist, breakdown=breakdown, singular=singular)


def arnoldi(op, v0: np.ndarray, steps: int, prec: Precision | None = None):
    """`steps` Arnoldi steps (CGS2) from v0 / ||v0||.  Returns (V, Hbar, k) with k <= steps
    the number of steps taken (fewer after a lucky breakdown)."""
    prec = prec or _fp64(v0.shape[0])
    cyc = gmres_cycle(op, v0, steps, -1.0, prec)
    return cyc.V, cyc.Hbar, cyc.k


# --------------------------------------------------------------------------
# Solvers
# --------------------------------------------------------------------------

@dataclass
class Info:
    status: int
    iters: int
    outer: int
    relres: float
    history: list = field(default_factory=list)  # explicit relres after each restart
    inner_hist: list = field(default_factory=list)  # implicit residual per iteration


def _check_inputs(A, b):
    if not (np.all(np.isfinite(A.vals)) and np.all(np.isfinite(b))):
        return NONFINITE
    return OK


def gmres(A, b, x0=None, m: int = 50, rtol: float = 1e-10, max_iters: int = 100000,
          poly_roots=None, precision: str = "fp64", right_prec=None) -> tuple[np.ndarray, Info]:
    """Restarted GMRES(m) (Algorithm 1, CGS2, right polynomial preconditioner optional).

    precision='fp64' is the plain double-precision solver.  precision='fp32' runs the whole
    solver in single precision (A, x, r, V and every vector result rounded to FP32), the
    first stage of GMRES-FD and the paper's "fp32 GMRES" curve (Section 5.2)."""
    n = A.n
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    if _check_inputs(A, b) != OK:
        return x, Info(NONFINITE, 0, 0, float("nan"))
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), Info(OK, 0, 0, 0.0)
    if precision == "fp64":
        prec = _fp64(n)
        vals = A.vals
        rw = prec.rw
    else:
        prec = Precision("fp32", "fp32", n)
        vals = round_to(A.vals, "fp32")
        b = round_to(b, "fp32")
        x = round_to(x, "fp32")
        rw = prec.rw

    def opA(v):
        return rw(spmv(A, v, vals))

    op = opA
    if poly_roots is not None and len(poly_roots):
        from .poly import poly_apply

        def op(v):
            return opA(poly_apply(opA, poly_roots, v, rw))
    elif right_prec is not None:
        def op(v):
            return opA(rw(right_prec(v)))

    r = rw(b - opA(x))
    gamma = float(np.linalg.norm(r))
    info = Info(OK, 0, 0, gamma / bnorm, [gamma / bnorm])
    while True:
        if not np.isfinite(gamma):
            info.status = NONFINITE
            break
        if gamma <= rtol * bnorm:
            break
        if info.iters >= max_iters:
            info.status = NOT_CONVERGED
            break
        cyc = gmres_cycle(op, r, min(m, max_iters - info.iters), rtol * bnorm / gamma, prec)
        info.iters += cyc.k
        info.outer += 1
        info.inner_hist += [h * gamma / bnorm for h in cyc.hist]
        u = rw(cyc.V[:, :len(cyc.y)] @ cyc.y)
        if poly_roots is not None and len(poly_roots):
            from .poly import poly_apply
            u = poly_apply(opA, poly_roots, u, rw)
        elif right_prec is not None:
            u = rw(right_prec(u))
        x = rw(x + gamma * u)
        r = rw(b - opA(x))
        gamma = float(np.linalg.norm(r))
        info.relres = gamma / bnorm
        info.history.append(info.relres)
        if cyc.singular:
            info.status = BREAKDOWN if gamma > rtol * bnorm else OK
            break
    info.relres = gamma / bnorm
    return x, info


# GMRES-IR gives up (NOT_CONVERGED) after this many refinement steps in a row that do not
# lower the explicit relative residual by 0.1%: with an inner precision too coarse for the
# problem the refinement stalls or diverges (the paper does not say when to stop then).
IR_STALL_LIMIT = 20


def gmres_ir(A, b, x0=None, m: int = 50, rtol: float = 1e-10, inner: str = "fp32",
             inner_rtol: float = 0.0, max_iters: int = 100000, poly_roots=None,
             arith: str = "fp32", right_prec=None) -> tuple[np.ndarray, Info]:
    """GMRES-IR (Algorithm 2): FP64 residual and update around a low-precision GMRES(m)
    cycle.  `inner` is the storage precision of A's copy and of the basis (fp32, fp16, bf16;
    fp64 reproduces plain restarted GMRES with an explicit residual test at each restart)."""
    n = A.n
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    if _check_inputs(A, b) != OK:
        return x, Info(NONFINITE, 0, 0, float("nan"))
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), Info(OK, 0, 0, 0.0)
    prec = Precision.for_inner(inner, A, arith)
    low_vals = prec.matrix_values(A.vals)

    def op_low(v):  # SpMV with the low-precision copy, result in working precision
        return prec.rw(prec.s_A * spmv(A, v, low_vals))

    op = op_low
    if poly_roots is not None and len(poly_roots):
        from .poly import poly_apply

        def op(v):
            return op_low(poly_apply(op_low, poly_roots, v, prec.rw))
    elif right_prec is not None:
        def op(v):
            return op_low(prec.rw(right_prec(v)))

    r = b - spmv(A, x)  # [double]
    gamma = float(np.linalg.norm(r))
    info = Info(OK, 0, 0, gamma / bnorm, [gamma / bnorm])
    best, stall = gamma / bnorm, 0  # stall test (reading: no 0.1% progress in 20 steps)
    while True:
        if not np.isfinite(gamma):
            info.status = NONFINITE
            break
        if gamma <= rtol * bnorm:
            break
        if info.iters >= max_iters or stall >= IR_STALL_LIMIT:
            info.status = NOT_CONVERGED
            break
        cyc = gmres_cycle(op, r, min(m, max_iters - info.iters), inner_rtol, prec)  # [single]
        info.iters += cyc.k
        info.outer += 1
        info.inner_hist += [h for h in cyc.hist]
        u = prec.rw(cyc.V[:, :len(cyc.y)] @ cyc.y)
        if poly_roots is not None and len(poly_roots):
            from .poly import poly_apply
            u = poly_apply(op_low, poly_roots, u, prec.rw)
        elif right_prec is not None:
            u = prec.rw(right_prec(u))
        x = x + gamma * u  # [double]
        r = b - spmv(A, x)  # [double]
        gamma = float(np.linalg.norm(r))
        info.relres = gamma / bnorm
        info.history.append(info.relres)
        if info.relres < best * (1.0 - 1e-3):
            best, stall = info.relres, 0
        else:
            stall += 1
        if cyc.singular:
            info.status = BREAKDOWN if gamma > rtol * bnorm else OK
            break
    info.relres = gamma / bnorm
    return x, info


def gmres_fd(A, b, switch_iter: int, m: int = 50, rtol: float = 1e-10,
             max_iters: int = 100000) -> tuple[np.ndarray, Info, Info]:
    """GMRES-FD (Section 3.3): FP32 GMRES(m) for `switch_iter` iterations (a multiple of m:
    the switch happens at a restart), then FP64 GMRES(m) from that solution."""
    x32, info32 = gmres(A, b, None, m, rtol, max_iters=switch_iter, precision="fp32")
    x, info64 = gmres(A, b, x32, m, rtol, max_iters=max_iters)
    return x, info32, info64
