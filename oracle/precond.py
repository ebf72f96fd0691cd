"""Outer preconditioning for the SPD (graph Laplacian) form (Sec. 4.4.2, Sec. 5.1),
and inner preconditioning for the normal form (Sec. 4.4.1).

TEST INFRASTRUCTURE ONLY, like the rest of this package.

The paper replaces B = A + eps D by B_R = P_R^-1 A P_R^-T + eps D, with P_R the
incomplete Cholesky factor of A (Matlab ichol, threshold dropping, diagonal
compensation 0.1), and maps the result back by V <- P_R^-T V (Sec. 4.4.2).  The
preconditioner built here is the fixed-pattern form of the same factorization:

  1. the graph of A (its off-diagonal pattern) is coloured by the Jones-Plassmann
     rule: vertex v gets the smallest colour not used by its neighbours of higher
     priority, priorities being uniform draws (Philox stream PRIORITY_STREAM, ties
     by index).  That is greedy colouring in descending priority order;
  2. the vertices are renumbered colour by colour (stable in the index), giving a
     permutation Pi and A~ = Pi^T A Pi;
  3. L is the incomplete Cholesky factor with zero fill, IC(0), of
     A~ + alpha diag(A~): lower triangular on the pattern of tril(A~), with
     (L L^T)_ij = (A~ + alpha diag A~)_ij on that pattern;
  4. P_R = Pi L, so B_R = L^-1 A~ L^-T + eps D in the renumbered space, and
     null(A) = Pi L^-T null(B_R - eps D).

Within one colour no two vertices are adjacent, so every row of L (and of L^T)
depends only on rows of other colours: the factorization and both triangular
solves proceed colour by colour.  This differs from the paper's threshold
factorization (which fills in and orders the work sequentially) in the pattern;
the operator and the post-processing are the paper's.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .philox import uniform01

PRIORITY_STREAM = 0x7FFFFFFF  # Philox stream of the colouring priorities
DIAGCOMP = 0.1                # Matlab ichol 'diagcomp' of Eq. (defichol)


def greedy_coloring_by_priority(A: sp.csr_matrix, prio: np.ndarray) -> np.ndarray:
    """Plain definition: visit vertices by descending (priority, index); each takes
    the smallest colour that no already coloured neighbour has."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    order = sorted(range(n), key=lambda v: (prio[v], v), reverse=True)
    color = np.full(n, -1, dtype=np.int64)
    for v in order:
        nb = A.indices[A.indptr[v]:A.indptr[v + 1]]
        used = {int(color[u]) for u in nb if u != v and color[u] >= 0}
        c = 0
        while c in used:
            c += 1
        color[v] = c
    return color


def jp_coloring(A: sp.csr_matrix, seed: int) -> np.ndarray:
    """Jones-Plassmann rounds: every uncoloured vertex whose (priority, index) beats
    all its uncoloured neighbours takes the smallest colour absent among its
    coloured neighbours.  Returns the colour of every vertex."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    prio = uniform01(seed, PRIORITY_STREAM, n)
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    cols = A.indices.astype(np.int64)
    off = rows != cols
    rows, cols = rows[off], cols[off]
    color = np.full(n, -1, dtype=np.int64)
    while (color < 0).any():
        unc = color < 0
        # edge (v, u) with both uncoloured and u ahead of v: v is not a local maximum
        beats = unc[rows] & unc[cols] & ((prio[cols] > prio[rows]) | ((prio[cols] == prio[rows]) & (cols > rows)))
        blocked = np.zeros(n, dtype=bool)
        blocked[rows[beats]] = True
        winners = np.nonzero(unc & ~blocked)[0]
        for v in winners:
            nb = A.indices[A.indptr[v]:A.indptr[v + 1]]
            used = {int(color[u]) for u in nb if u != v and color[u] >= 0}
            c = 0
            while c in used:
                c += 1
            color[v] = c
    return color


def color_permutation(color: np.ndarray) -> np.ndarray:
    """perm[new] = old: vertices ordered by colour, then by index."""
    return np.lexsort((np.arange(color.size), color)).astype(np.int64)


def permute(A: sp.csr_matrix, perm: np.ndarray) -> sp.csr_matrix:
    """A~ = Pi^T A Pi with (Pi^T A Pi)[i, j] = A[perm[i], perm[j]]."""
    A = sp.csr_matrix(A)
    At = A[perm][:, perm].tocsr()
    At.sort_indices()
    return At


def ic0(At: sp.csr_matrix, alpha: float = DIAGCOMP) -> sp.csr_matrix:
    """IC(0) of At + alpha diag(At): for each row i in order, each kept entry (i, j),
    j < i, is (a_ij - sum_k l_ik l_jk) / l_jj over the columns k < j kept in both
    rows, then l_ii = sqrt(a_ii (1 + alpha) - sum_j l_ij^2).  Raises on a
    non-positive pivot."""
    At = sp.csr_matrix(At)
    n = At.shape[0]
    Lr = [None] * n  # per row: (cols ascending, values), diagonal last
    for i in range(n):
        cols = At.indices[At.indptr[i]:At.indptr[i + 1]]
        vals = At.data[At.indptr[i]:At.indptr[i + 1]]
        keep = cols < i
        lc = cols[keep].astype(np.int64)
        lv = vals[keep].astype(np.float64).copy()
        order = np.argsort(lc, kind="stable")
        lc, lv = lc[order], lv[order]
        dpos = np.nonzero(cols == i)[0]
        aii = float(vals[dpos[0]]) if dpos.size else 0.0
        row = dict()
        for p, j in enumerate(lc):
            jc, jv = Lr[j]
            s = lv[p]
            # common columns k < j of row i (entries before p) and row j (off-diagonal part)
            for q in range(p):
                k = lc[q]
                hit = np.searchsorted(jc[:-1], k)
                if hit < jc.size - 1 and jc[hit] == k:
                    s -= lv[q] * jv[hit]
            lv[p] = s / jv[-1]
        piv = aii * (1.0 + alpha) - float(np.dot(lv, lv))
        if not piv > 0.0:
            raise np.linalg.LinAlgError(f"IC(0) breakdown at row {i}")
        Lr[i] = (np.concatenate([lc, [i]]), np.concatenate([lv, [np.sqrt(piv)]]))
        del row
    indptr = np.zeros(n + 1, dtype=np.int64)
    indptr[1:] = np.cumsum([c.size for c, _ in Lr])
    ind = np.concatenate([c for c, _ in Lr]) if n else np.zeros(0, np.int64)
    dat = np.concatenate([v for _, v in Lr]) if n else np.zeros(0)
    return sp.csr_matrix((dat, ind, indptr), shape=(n, n))


class Preconditioner:
    """P_R = Pi L for an SPD A (graph Laplacian)."""

    def __init__(self, A: sp.csr_matrix, seed: int, alpha: float = DIAGCOMP):
        A = sp.csr_matrix(A, dtype=np.float64)
        self.color = jp_coloring(A, seed)
        self.perm = color_permutation(self.color)
        self.At = permute(A, self.perm)
        self.L = ic0(self.At, alpha)
        self.LT = self.L.T.tocsr()
        self.alpha = alpha

    def solve_L(self, Y):
        return spla.spsolve_triangular(self.L, Y, lower=True)

    def solve_LT(self, Y):
        return spla.spsolve_triangular(self.LT, Y, lower=False)

    def unpermute(self, V):
        """Rows back to the original numbering: out[perm[i]] = V[i]."""
        out = np.empty_like(V)
        out[self.perm] = V
        return out


class PrecondOperator:
    """B_R X = L^-1 A~ L^-T X + eps D X in the renumbered space (Sec. 4.4.2)."""

    def __init__(self, pc: Preconditioner, eps: float, Dvec: np.ndarray):
        self.pc = pc
        self.eps = float(eps)
        self.D = np.asarray(Dvec, dtype=np.float64)
        self.n = pc.At.shape[0]
        self.mode = "spd"

    def apply(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        Y = self.pc.solve_L(self.pc.At @ self.pc.solve_LT(X))
        return Y.reshape(X.shape) + self.eps * self.D[:, None] * X

    def norm_bound(self) -> float:
        """Reading P2: the first cycle takes ||A||_inf + eps as its bound on ||B_R||."""
        ninf = float(abs(self.pc.At).sum(axis=1).max()) if self.pc.At.nnz else 0.0
        return ninf + self.eps


def effective_condition(M: np.ndarray, nullity: int) -> float:
    """Largest over smallest nonzero eigenvalue of a symmetric PSD matrix with a known
    nullity (dense; small matrices only)."""
    w = np.linalg.eigvalsh(0.5 * (M + M.T))
    return float(w[-1] / w[nullity])


def inner_scaled(A: sp.csr_matrix) -> sp.csr_matrix:
    """Inner preconditioning (Sec. 4.4.1) with P_L = diag(A A^T): A^T P_L^-1 A equals
    (S A)^T (S A) with S = diag(1 / ||a_i||_2) (0 for a zero row, the pseudo-inverse).
    null(S A) = null(A) because S is invertible on the nonzero rows."""
    A = sp.csr_matrix(A, dtype=np.float64)
    q = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    s = np.where(q > 0, 1.0 / np.sqrt(np.where(q > 0, q, 1.0)), 0.0)
    return sp.csr_matrix(sp.diags(s) @ A)
