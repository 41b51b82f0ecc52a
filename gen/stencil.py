"""Finite-difference convection-diffusion test matrices and right-hand sides.

The paper's test problems (Section 5) are Galeri stencils (BentPipe2D, UniFlow2D,
Laplace3D, Stretched2D) and SuiteSparse matrices, none of which ship here.  The
stand-ins built below have the same shape: 5-point (2D) and 7-point (3D)
operators, 5 and 7 nonzeros per interior row, nonsymmetric when the wind is
nonzero, CSR with int32 indices and FP64 values (the paper's storage, Section
5.5).

Operator: -div(K grad u) + beta . grad u on the unit square/cube with zero
Dirichlet boundary, grid spacing h = 1/(side+1), K = diag(1, eps, 1) (eps =
1/anisotropy on the second axis), beta = Pe * unit wind, first-order upwind
convection.  Every row is multiplied by h^2, so for axis k

    coefficient of u[i - e_k] = -K_k - h * max(beta_k, 0)
    coefficient of u[i + e_k] = -K_k - h * max(-beta_k, 0)
    diagonal                  = sum_k (2 K_k + h |beta_k|)

which is a weakly diagonally dominant M-matrix.  Unknowns are numbered
lexicographically with the first axis fastest, and the columns of each row come
out sorted.

Random numbers come from numpy's PCG64 generator seeded per call.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """A CSR matrix plus descriptive metadata (no right-hand side)."""

    name: str
    n: int
    row_ptr: np.ndarray  # int32, n+1
    col_idx: np.ndarray  # int32, nnz
    vals: np.ndarray  # float64, nnz
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.vals, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _conv_diff(dims: tuple[int, ...], kdiag: tuple[float, ...], beta: tuple[float, ...],
               name: str, meta: dict) -> Problem:
    d = len(dims)
    side = dims[0]
    if any(s != side for s in dims):
        raise ValueError("only cubic grids are generated")
    n = int(np.prod(dims))
    if n >= 2**31 - 1:
        raise ValueError("int32 CSR indices overflow")
    h = 1.0 / (side + 1)
    strides = [int(np.prod(dims[:k])) for k in range(d)]
    i = np.arange(n, dtype=np.int64)
    coord = [(i // strides[k]) % dims[k] for k in range(d)]

    # Column slots in increasing column order: -e_{d-1}, ..., -e_0, diag, +e_0, ..., +e_{d-1}.
    slots = 2 * d + 1
    cols = np.empty((n, slots), dtype=np.int64)
    vals = np.empty((n, slots), dtype=np.float64)
    mask = np.ones((n, slots), dtype=bool)
    diag = sum(2.0 * kdiag[k] + h * abs(beta[k]) for k in range(d))
    for s, k in enumerate(reversed(range(d))):
        cols[:, s] = i - strides[k]
        vals[:, s] = -kdiag[k] - h * max(beta[k], 0.0)
        mask[:, s] = coord[k] > 0
    cols[:, d] = i
    vals[:, d] = diag
    for k in range(d):
        s = d + 1 + k
        cols[:, s] = i + strides[k]
        vals[:, s] = -kdiag[k] - h * max(-beta[k], 0.0)
        mask[:, s] = coord[k] < dims[k] - 1

    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = cols[mask].astype(np.int32)
    v = vals[mask]
    meta = dict(meta)
    meta.update(dims=list(dims), h=h, K=list(kdiag), beta=list(beta),
                cell_peclet=float(max(abs(b) for b in beta) * h / 2.0))
    return Problem(name=name, n=n, row_ptr=row_ptr.astype(np.int32), col_idx=col_idx,
                   vals=v, meta=meta)


def conv_diff_2d(side: int, peclet: float = 0.0, wind=(1.0, 0.0), anisotropy: float = 1.0,
                 name: str | None = None) -> Problem:
    """5-point upwind convection-diffusion on a side x side grid."""
    w = np.asarray(wind, dtype=np.float64)
    w = w / np.linalg.norm(w) if np.linalg.norm(w) > 0 else w
    beta = tuple(float(peclet * c) for c in w)
    kd = (1.0, 1.0 / anisotropy)
    nm = name or f"convdiff2d_{side}"
    return _conv_diff((side, side), kd, beta, nm,
                      dict(peclet=peclet, wind=list(map(float, w)), anisotropy=anisotropy))


def conv_diff_3d(side: int, peclet: float = 0.0, wind=(1.0, 0.0, 0.0), anisotropy: float = 1.0,
                 name: str | None = None) -> Problem:
    """7-point upwind convection-diffusion on a side^3 grid."""
    w = np.asarray(wind, dtype=np.float64)
    w = w / np.linalg.norm(w) if np.linalg.norm(w) > 0 else w
    beta = tuple(float(peclet * c) for c in w)
    kd = (1.0, 1.0 / anisotropy, 1.0)
    nm = name or f"convdiff3d_{side}"
    return _conv_diff((side, side, side), kd, beta, nm,
                      dict(peclet=peclet, wind=list(map(float, w)), anisotropy=anisotropy))


def random_wind(seed: int, dim: int) -> np.ndarray:
    """Unit wind direction: angle ~ U(0, 2pi) in 2D, uniform on the sphere in 3D."""
    g = _rng(seed)
    if dim == 2:
        phi = g.uniform(0.0, 2.0 * np.pi)
        return np.array([np.cos(phi), np.sin(phi)])
    v = g.standard_normal(3)
    return v / np.linalg.norm(v)


def rhs_manufactured(p: Problem, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """x_true ~ U(-1, 1) from the seed and b = A x_true (FP64)."""
    x_true = _rng(seed).uniform(-1.0, 1.0, p.n)
    return p.scipy() @ x_true, x_true


def rhs_ones(p: Problem) -> np.ndarray:
    return np.ones(p.n)


def rhs_ones_plus_noise(p: Problem, seed: int, sigma: float = 1e-3) -> np.ndarray:
    """b = A * ones + sigma * N(0, 1)."""
    return p.scipy() @ np.ones(p.n) + sigma * _rng(seed).standard_normal(p.n)


# --------------------------------------------------------------------------
# Workload recipes (sizes and seeds of the five workloads).
# --------------------------------------------------------------------------

def config_small_2d(side: int = 64):
    """64x64 5-point convection-diffusion, Pe 10, random wind (seed 101), manufactured
    solution x_true ~ U(-1,1) (seed 102)."""
    p = conv_diff_2d(side, 10.0, random_wind(101, 2), name=f"convdiff2d_{side}_pe10")
    b, x_true = rhs_manufactured(p, 102)
    return p, b, x_true


def config_3d(peclet: float = 10.0, side: int = 100):
    """100^3 7-point convection-diffusion; Pe in {1, 10, 50} picks wind seed 201/202/203 and
    noise seed 211/212/213; b = A*1 + 1e-3 N(0,1)."""
    table = {1.0: (201, 211), 10.0: (202, 212), 50.0: (203, 213)}
    ws, rs = table.get(float(peclet), (200 + int(peclet), 210 + int(peclet)))
    p = conv_diff_3d(side, peclet, random_wind(ws, 3), name=f"convdiff3d_{side}_pe{peclet:g}")
    return p, rhs_ones_plus_noise(p, rs)


def config_aniso_2d(side: int = 2000, anisotropy: float = 100.0, peclet: float = 100.0):
    """2000^2 anisotropic 5-point convection-diffusion, eps = 1e-2, Pe 100, wind (1,1)/sqrt(2),
    b = ones."""
    p = conv_diff_2d(side, peclet, (1.0, 1.0), anisotropy,
                     name=f"aniso2d_{side}_a{anisotropy:g}_pe{peclet:g}")
    return p, rhs_ones(p)


def batched_systems(count: int = 512, seed0: int = 5000, side_lo: int = 32, side_hi: int = 256):
    """Uneven batch: system s uses seed seed0+s; side ~ U{side_lo..side_hi}, Pe ~ U(0.1, 50),
    wind angle ~ U(0, 2pi), x_true ~ U(-1, 1), b = A x_true."""
    out = []
    for s in range(count):
        g = _rng(seed0 + s)
        side = int(g.integers(side_lo, side_hi + 1))
        pe = float(g.uniform(0.1, 50.0))
        phi = float(g.uniform(0.0, 2.0 * np.pi))
        p = conv_diff_2d(side, pe, (np.cos(phi), np.sin(phi)), name=f"batch{s}_{side}")
        x_true = g.uniform(-1.0, 1.0, p.n)
        out.append((p, p.scipy() @ x_true, x_true))
    return out


def selector_matrices(count: int = 400, seed0: int = 4000, n_lo: float = 1e4, n_hi: float = 4e6):
    """Parameter-selector corpus descriptors (built lazily: large ones are up to 4M unknowns).

    Matrix s uses seed seed0+s: dim 2 or 3 (50:50), Pe log-uniform [0.1, 100], anisotropy
    log-uniform [1, 1e3], N log-uniform [n_lo, n_hi], side = round(N^(1/dim)), wind random.
    Returns a list of dicts; build one with `build_selector_matrix`."""
    out = []
    for s in range(count):
        g = _rng(seed0 + s)
        dim = 2 if g.uniform() < 0.5 else 3
        pe = float(10 ** g.uniform(-1.0, 2.0))
        an = float(10 ** g.uniform(0.0, 3.0))
        nn = float(10 ** g.uniform(np.log10(n_lo), np.log10(n_hi)))
        side = max(4, int(round(nn ** (1.0 / dim))))
        if dim == 2:
            phi = float(g.uniform(0.0, 2.0 * np.pi))
            wind = [np.cos(phi), np.sin(phi)]
        else:
            v = g.standard_normal(3)
            wind = list(v / np.linalg.norm(v))
        out.append(dict(index=s, seed=seed0 + s, dim=dim, peclet=pe, anisotropy=an,
                        side=side, wind=wind))
    return out


def build_selector_matrix(desc: dict) -> Problem:
    if desc["dim"] == 2:
        return conv_diff_2d(desc["side"], desc["peclet"], desc["wind"], desc["anisotropy"],
                            name=f"sel{desc['index']}")
    return conv_diff_3d(desc["side"], desc["peclet"], desc["wind"], desc["anisotropy"],
                        name=f"sel{desc['index']}")


# Shape of the selector network (16 features -> 64 -> 64 -> 32 classes), needed to draw its
# initial weights; the network's arithmetic lives in the library and in the oracle.
MLP_SHAPES = ((16, 64), (64,), (64, 64), (64,), (64, 32), (32,))


def mlp_init(seed: int = 4242) -> np.ndarray:
    """Initial selector weights, flat float32 in the layout W1, b1, W2, b2, W3, b3 (W row-major
    [in][out]): W ~ U(-a, a) with a = sqrt(6 / (fan_in + fan_out)) from PCG64(seed), b = 0."""
    g = _rng(seed)
    out = []
    for s in MLP_SHAPES:
        if len(s) == 2:
            a = np.sqrt(6.0 / (s[0] + s[1]))
            out.append(g.uniform(-a, a, s).astype(np.float32).ravel())
        else:
            out.append(np.zeros(s, np.float32))
    return np.concatenate(out)


def stencil_matrix(dims: tuple[int, ...], offsets, name: str) -> Problem:
    """Constant-coefficient stencil on a grid with zero Dirichlet boundary: -1 for every
    in-grid neighbour at the given offsets and the stencil's neighbour count on the diagonal
    (a Galeri-style Laplacian of any stencil shape).  Rows in lexicographic order, x fastest."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n)
    coords = np.unravel_index(idx, dims[::-1])[::-1]  # coords[0] = x (fastest)
    strides = [int(np.prod(dims[:k])) for k in range(len(dims))]
    rows, cols, vals = [idx], [idx], [np.zeros(n)]
    for off in offsets:
        ok = np.ones(n, bool)
        shift = 0
        for k, o in enumerate(off):
            c = coords[k] + o
            ok &= (c >= 0) & (c < dims[k])
            shift += o * strides[k]
        r = idx[ok]
        rows.append(r)
        cols.append(r + shift)
        vals.append(-np.ones(len(r)))
    vals[0] = np.full(n, float(len(offsets)))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sort_indices()
    return Problem(name, n, A.indptr.astype(np.int32), A.indices.astype(np.int32),
                   A.data.astype(np.float64), dict(dims=list(dims), stencil=len(offsets) + 1))


def laplace_2d(side: int) -> Problem:
    """5-point Laplacian (Galeri Laplace2D-like)."""
    return stencil_matrix((side, side), [(1, 0), (-1, 0), (0, 1), (0, -1)], f"laplace2d_{side}")


def laplace_3d(side: int) -> Problem:
    """7-point Laplacian (Galeri Laplace3D-like)."""
    offs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    return stencil_matrix((side, side, side), offs, f"laplace3d_{side}")


def uniflow_2d(side: int) -> Problem:
    """UniFlow2D-like stand-in (Galeri's matrix is absent): 5-point upwind
    convection-diffusion with a uniform diagonal wind, Peclet 100."""
    return conv_diff_2d(side, 100.0, (1.0, 1.0), name=f"uniflow2d_{side}")


def bentpipe_2d(side: int) -> Problem:
    """BentPipe2D-like stand-in: convection at an angle, Peclet 50."""
    return conv_diff_2d(side, 50.0, (0.8, -0.6), name=f"bentpipe2d_{side}")


def box_2d(side: int) -> Problem:
    """9-point box stencil (Galeri Star2D / Cross-like 3x3 neighbourhood)."""
    offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]
    return stencil_matrix((side, side), offs, f"box2d_{side}")


def star_3d(side: int) -> Problem:
    """13-point fourth-order star: two neighbours along each axis direction in 3D."""
    offs = [tuple(s * r if k == a else 0 for k in range(3)) for a in range(3) for s in (1, -1)
            for r in (1, 2)]
    return stencil_matrix((side, side, side), offs, f"star3d_{side}")


def box_3d(side: int) -> Problem:
    """27-point box stencil in 3D (SPD; a stand-in for 3D finite-element matrices with about
    27 entries per row)."""
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dx, dy, dz) != (0, 0, 0)]
    return stencil_matrix((side, side, side), offs, f"box3d_{side}")


def shuffled(p: Problem, seed: int) -> Problem:
    """The same matrix with its unknowns relabelled by a seeded random permutation q
    (row/column i of the result is row/column q[i] of p): an arbitrary numbering like a
    matrix collection's, for the reordering to undo."""
    q = _rng(seed).permutation(p.n)
    A = sp.csr_matrix((p.vals, p.col_idx, p.row_ptr), shape=(p.n, p.n))[q][:, q].tocsr()
    A.sort_indices()
    meta = dict(p.meta, shuffle_seed=int(seed))
    return Problem(p.name + f"_shuf{seed}", p.n, A.indptr.astype(np.int32),
                   A.indices.astype(np.int32), A.data.astype(np.float64), meta)


def scaled(p: Problem, sigma: float, seed: int) -> Problem:
    """S A S with S = diag(exp(sigma z)), z ~ N(0, 1) seeded: the badly scaled unknowns of
    assembled engineering matrices (an SPD A stays SPD), which Jacobi-type preconditioners
    undo."""
    d = np.exp(sigma * _rng(seed).standard_normal(p.n))
    A = sp.csr_matrix((p.vals, p.col_idx, p.row_ptr), shape=(p.n, p.n))
    A = (sp.diags(d) @ A @ sp.diags(d)).tocsr()
    A.sort_indices()
    meta = dict(p.meta, scale_sigma=float(sigma), scale_seed=int(seed))
    return Problem(p.name + f"_scaled{sigma:g}", p.n, A.indptr.astype(np.int32),
                   A.indices.astype(np.int32), A.data.astype(np.float64), meta)


def config_bj() -> list[tuple[Problem, int]]:
    """The block-Jacobi workloads (Section 5.8's "J k" rows, whose SuiteSparse matrices are
    absent): synthetic stand-ins, badly scaled (sigma = 1) and in a shuffled numbering,
    each with its block size.
      * SPD 3D, 27-point box stencil on 60^3 (n = 216,000, ~27 entries per row), k = 42
        (for the SPD finite-element row, "J 42");
      * nonsymmetric 3D upwind convection-diffusion, 48^3 (n = 110,592, 7 per row), Pe 50,
        k = 1 (for the nonsymmetric row, "J 1")."""
    return [(shuffled(scaled(box_3d(60), 1.0, 13), 11), 42),
            (shuffled(scaled(conv_diff_3d(48, 50.0, (0.6, 0.8, 0.0)), 1.0, 14), 12), 1)]

