"""Reference quantities for checking any computed null-space basis.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).
"""

import numpy as np
import scipy.sparse as sp


def components(A) -> tuple[int, np.ndarray]:
    """Connected components of the graph whose edges are the off-diagonal nonzeros
    of a Laplacian (or the two endpoints of every incidence-matrix row).  The null
    space of a graph Laplacian is spanned by the component indicators (Sec. 5.1)."""
    A = sp.csr_matrix(A)
    if A.shape[0] == A.shape[1]:
        G = A
    else:  # incidence matrix: columns sharing a row are adjacent
        G = (abs(A).T @ abs(A)).tocsr()
    return sp.csgraph.connected_components(G, directed=False)


def indicator_basis(labels: np.ndarray) -> np.ndarray:
    """Orthonormal basis of span{indicator of each component}: closed-form null space."""
    labels = np.asarray(labels)
    k = int(labels.max()) + 1
    n = labels.size
    U = np.zeros((n, k))
    U[np.arange(n), labels] = 1.0
    return U / np.sqrt(U.sum(axis=0))[None, :]


def copy_pair_basis(n: int, pairs: np.ndarray) -> np.ndarray:
    """Orthonormal basis {(e_src + e_copy)/sqrt 2} of the planted null space."""
    U = np.zeros((n, len(pairs)))
    for j, (s, c) in enumerate(pairs):
        U[s, j] = U[c, j] = 1.0 / np.sqrt(2.0)
    return U


def principal_sine(U: np.ndarray, X: np.ndarray) -> float:
    """Sine of the largest principal angle between span(U) and span(X) (Def. defPA).

    Both bases are orthonormalized first; for equal dimensions this equals
    ||U U^T - X X^T||_2 (Sec. 2.3).  For unequal dimensions the result is 1.
    """
    if U.shape[1] != X.shape[1]:
        return 1.0
    if U.shape[1] == 0:
        return 0.0
    Qu, _ = np.linalg.qr(U)
    Qx, _ = np.linalg.qr(X)
    s = np.linalg.svd(Qu.T @ Qx, compute_uv=False)
    c = float(np.clip(s.min(), 0.0, 1.0))
    # sin from the residual for accuracy at small angles
    resid = Qx - Qu @ (Qu.T @ Qx)
    return float(np.linalg.norm(resid, 2)) if c > 0.7 else float(np.sqrt(max(0.0, 1 - c * c)))
