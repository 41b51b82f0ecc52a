"""Oracle of the block-Jacobi preconditioner with reverse Cuthill-McKee ordering.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): imported by tests/ and the
benchmark's CPU legs, never by the CUDA library, and it imports nothing from it.

Method (Section 5.8 and its table of SuiteSparse runs; Section 3.4 for a single-precision
preconditioner inside GMRES-IR): the matrix is reordered with a reverse Cuthill-McKee
(RCM) ordering, then preconditioned with block Jacobi of block size k (the table's
"J k"; k = 1 and k = 42 there), inside GMRES and GMRES-IR.  The paper gives no further
detail, so the following readings are ours:

* RCM works on the structure of A + A^T without the diagonal.  deg(i) is the number of
  distinct neighbours of i.  Vertices are ranked by (deg, index).  Components are taken
  in the order of their lowest-ranked vertex s; each starts from the pseudo-peripheral
  vertex of the George-Liu iteration from s (root r = s; repeat: x = lowest-ranked
  vertex of the last BFS level of r; if the level structure of x is deeper than r's,
  r = x and repeat, else stop; the start vertex is x).  The Cuthill-McKee BFS appends
  the unvisited neighbours of each dequeued vertex in rank order; the concatenated order
  is reversed.  perm[new] = old.
* The reordered system is B x' = b' with B = P A P^T (B[i, j] = A[perm[i], perm[j]]),
  b' = b[perm], and x[perm[i]] = x'[i].
* Block Jacobi: M = blockdiag(B[s:e, s:e]) over the contiguous blocks [s, e) =
  [q k, min((q + 1) k, n)), the last one ragged; entries absent from the CSR are zero.
  It is a right preconditioner, like the polynomial (A M^{-1} y = r, u = M^{-1} y).
  Here M^{-1} v solves each block exactly in FP64 (library LU with partial pivoting);
  the solvers round the result to their working precision.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def adjacency(n: int, row_ptr, col_idx) -> list[list[int]]:
    """Sorted neighbour lists of the structure of A + A^T without self-loops."""
    nb = [set() for _ in range(n)]
    for i in range(n):
        for p in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            j = int(col_idx[p])
            if j != i:
                nb[i].add(j)
                nb[j].add(i)
    return [sorted(s) for s in nb]


def _levels(adj, root: int) -> list[list[int]]:
    """BFS level structure rooted at `root` (its component only)."""
    seen = {root}
    levels = [[root]]
    while True:
        nxt = []
        for u in levels[-1]:
            for v in adj[u]:
                if v not in seen:
                    seen.add(v)
                    nxt.append(v)
        if not nxt:
            return levels
        levels.append(nxt)


def pseudo_peripheral(adj, deg, seed: int) -> int:
    """George-Liu: the start vertex of the component of `seed` (module docstring)."""
    r = seed
    lr = _levels(adj, r)
    while True:
        x = min(lr[-1], key=lambda v: (deg[v], v))
        lx = _levels(adj, x)
        if len(lx) > len(lr):
            r, lr = x, lx
        else:
            return x


def rcm(n: int, row_ptr, col_idx) -> np.ndarray:
    """Reverse Cuthill-McKee permutation (perm[new] = old) of the CSR structure."""
    adj = adjacency(n, row_ptr, col_idx)
    deg = [len(a) for a in adj]
    visited = [False] * n
    order = []
    for s in sorted(range(n), key=lambda v: (deg[v], v)):
        if visited[s]:
            continue
        start = pseudo_peripheral(adj, deg, s)
        visited[start] = True
        q = deque([start])
        while q:
            u = q.popleft()
            order.append(u)
            for v in sorted((v for v in adj[u] if not visited[v]), key=lambda v: (deg[v], v)):
                visited[v] = True
                q.append(v)
    return np.array(order[::-1], dtype=np.int64)


def bandwidth(n: int, row_ptr, col_idx) -> int:
    """max |i - j| over the stored entries."""
    bw = 0
    for i in range(n):
        for p in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            bw = max(bw, abs(i - int(col_idx[p])))
    return bw


def permute(A, perm):
    """P A P^T as a new CSR problem (columns sorted in each row)."""
    from gen import Problem

    n = A.n
    perm = np.asarray(perm, dtype=np.int64)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        o = perm[i]
        s, e = int(A.row_ptr[o]), int(A.row_ptr[o + 1])
        c = iperm[A.col_idx[s:e]]
        k = np.argsort(c, kind="stable")
        cols.append(c[k])
        vals.append(A.vals[s:e][k])
        rp.append(rp[-1] + (e - s))
    ci = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    va = np.concatenate(vals) if vals else np.zeros(0)
    return Problem(A.name + "_perm", n, np.array(rp, dtype=np.int32), ci.astype(np.int32), va,
                   dict(A.meta))


class BlockJacobi:
    """M^{-1} v for M = blockdiag of the k x k diagonal blocks of A (module docstring)."""

    def __init__(self, A, k: int):
        if k < 1:
            raise ValueError("block size must be positive")
        self.n, self.k = A.n, k
        self.blocks = []
        for s in range(0, A.n, k):
            e = min(s + k, A.n)
            D = np.zeros((e - s, e - s))
            for i in range(s, e):
                for p in range(int(A.row_ptr[i]), int(A.row_ptr[i + 1])):
                    j = int(A.col_idx[p])
                    if s <= j < e:
                        D[i - s, j - s] += A.vals[p]
            self.blocks.append((s, e, D))

    def apply(self, v: np.ndarray) -> np.ndarray:
        v = np.asarray(v, dtype=np.float64)
        z = np.empty_like(v)
        for s, e, D in self.blocks:
            z[s:e] = np.linalg.solve(D, v[s:e])
        return z
