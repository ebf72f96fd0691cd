"""Pins of the oracle's outer preconditioning (Sec. 4.4.2, Eq. defichol).

Each check compares the oracle with a fact fixed by the mathematics, not with its
own formulas: the colouring against its sequential definition, the IC(0) factor
against its defining property and against a library Cholesky where no fill can
occur, the preconditioned operator's null space against the closed form
L^T Pi^T (component indicators), and the effect (a smaller effective condition
number and fewer B applications) on badly conditioned grid Laplacians.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lanczos_nullspace, principal_sine, indicator_basis
from oracle.philox import uniform01
from oracle.precond import (PRIORITY_STREAM, Preconditioner, PrecondOperator, color_permutation,
                            effective_condition, greedy_coloring_by_priority, ic0, jp_coloring, permute)
from workloads import laplacian_grid_components, laplacian_er_components, laplacian_cycle_components


@pytest.mark.parametrize("make", [lambda: laplacian_grid_components(3, 6, 8, 16),
                                  lambda: laplacian_er_components(4, 5, 60, 0.08),
                                  lambda: laplacian_cycle_components(5, 3000, 7, 8, "powerlaw", 50)])
def test_jones_plassmann_is_greedy_colouring_in_priority_order(make):
    w = make()
    A = w.A.to_scipy()
    seed = 11
    col = jp_coloring(A, seed)
    ref = greedy_coloring_by_priority(A, uniform01(seed, PRIORITY_STREAM, A.shape[0]))
    assert np.array_equal(col, ref)
    Ac = sp.coo_matrix(A)
    off = Ac.row != Ac.col
    assert not np.any(col[Ac.row[off]] == col[Ac.col[off]]), "not a proper colouring"
    assert col.max() + 1 <= int(np.diff(A.indptr).max())  # at most max degree + 1 colours


def test_renumbering_is_by_colour_then_index():
    col = np.array([2, 0, 1, 0, 2, 1, 0])
    perm = color_permutation(col)
    assert perm.tolist() == [1, 3, 6, 2, 5, 0, 4]
    A = sp.random(7, 7, density=0.5, random_state=1, format="csr")
    At = permute(A, perm)
    D, P = A.toarray(), At.toarray()
    for i in range(7):
        for j in range(7):
            assert P[i, j] == D[perm[i], perm[j]]


@pytest.mark.parametrize("alpha", [0.1, 0.0, 1.0])
def test_ic0_defining_property(alpha):
    """L lower triangular with a positive diagonal, and (L L^T)_ij equals
    (A~ + alpha diag A~)_ij on the pattern of tril(A~)."""
    w = laplacian_grid_components(7, 4, 6, 12)
    A = w.A.to_scipy()
    pc = Preconditioner(A, 5, alpha if alpha > 0 else 1e-12)
    L = pc.L
    assert sp.triu(L, 1).nnz == 0
    assert np.all(L.diagonal() > 0)
    At = pc.At
    M = (At + pc.alpha * sp.diags(At.diagonal())).tocsr()
    pat = sp.tril(At).tocsr()
    pat.data[:] = 1.0
    R = (L @ L.T - M).multiply(pat)
    assert abs(R).max() <= 1e-13 * abs(M).max()
    # L keeps exactly the pattern of tril(A~)
    assert (abs(sp.tril(At)).astype(bool) != abs(L).astype(bool)).nnz == 0


def test_ic0_is_exact_cholesky_without_fill():
    """A matching (disjoint edges) has no fill in any order: IC(0) is the Cholesky
    factor of the shifted matrix."""
    n = 40
    rows, cols = np.arange(0, n, 2), np.arange(1, n, 2)
    Adj = sp.coo_matrix((np.ones(n // 2), (rows, cols)), shape=(n, n))
    Adj = Adj + Adj.T
    rng = np.random.default_rng(3)
    Lap = sp.diags(np.asarray(Adj.sum(axis=1)).ravel() + rng.random(n)) - Adj
    At = permute(sp.csr_matrix(Lap), rng.permutation(n))
    L = ic0(At, 0.1)
    M = At.toarray() + 0.1 * np.diag(At.diagonal())
    assert np.allclose(L.toarray(), np.linalg.cholesky(M), rtol=0, atol=1e-14)


def test_ic0_breakdown_is_reported():
    """A symmetric matrix that is not positive definite fails at its pivot."""
    A = sp.csr_matrix(np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(np.linalg.LinAlgError):
        ic0(A, 0.0)


def test_preconditioned_null_space_closed_form():
    """null(L^-1 A~ L^-T) = L^T null(A~): with U the component indicators of A,
    B_R (L^T Pi^T U) = eps D L^T Pi^T U exactly (up to rounding)."""
    w = laplacian_grid_components(9, 5, 6, 14)
    A = w.A.to_scipy()
    pc = Preconditioner(A, 2)
    U = indicator_basis(w.labels)[pc.perm]  # renumbered rows
    V = pc.LT @ U
    op = PrecondOperator(pc, 0.0, np.zeros(A.shape[0]))
    BV = op.apply(V)
    assert np.abs(BV).max() <= 1e-12 * np.abs(V).max() * abs(A).sum(axis=1).max()


def test_preconditioning_reduces_the_condition_number():
    """On 2-D grid components (kappa ~ side^2) IC(0) shrinks the effective condition
    number: kappa(L^-1 A~ L^-T) < kappa(A) / 3 (dense eigenvalues, small case)."""
    w = laplacian_grid_components(3, 6, 8, 16)
    A = w.A.to_scipy()
    pc = Preconditioner(A, 7)
    Ad = pc.At.toarray()
    Li = np.linalg.inv(pc.L.toarray())
    k0 = effective_condition(Ad, w.nullity)
    k1 = effective_condition(Li @ Ad @ Li.T, w.nullity)
    assert k1 < k0 / 3, (k0, k1)


def test_preconditioned_solve_finds_the_components():
    """The preconditioned method (Sec. 4.4.2) finds every component of a grid
    Laplacian, maps the basis back to null(A), and needs fewer B applications."""
    w = laplacian_grid_components(3, 6, 8, 16)
    A = w.A.to_scipy()
    U = indicator_basis(w.labels)
    plain = lanczos_nullspace(A, "spd", 1, 60, tol=1e-10, seed=7)
    pre = lanczos_nullspace(A, "spd", 1, 60, tol=1e-10, seed=7, precond=0.1)
    assert plain.N == pre.N == w.nullity
    assert principal_sine(pre.X, U) <= 1e-8
    assert np.abs(pre.X.T @ pre.X - np.eye(pre.N)).max() <= 1e-12
    assert np.linalg.norm(A @ pre.X) <= 1e-9 * abs(A).sum(axis=1).max()
    assert pre.stats["matvecs"] < plain.stats["matvecs"]


# ---------------------------------------------------------- inner (Sec. 4.4.1) ---

def test_inner_scaling_keeps_the_null_space_and_balances_rows():
    """S A has unit rows (P_L = diag(A A^T)), the planted copy-pair null space of the
    badly scaled matrix is exactly its null space, and the effective condition of
    the normal matrix drops."""
    from oracle import copy_pair_basis
    from oracle.precond import inner_scaled
    from workloads import rectangular_copies_scaled
    w = rectangular_copies_scaled(5, 600, 400, 4, 3.0)
    A = w.A.to_scipy()
    As = inner_scaled(A)
    rn = np.sqrt(np.asarray(As.multiply(As).sum(axis=1)).ravel())
    assert np.allclose(rn[rn > 0], 1.0, rtol=1e-14)
    U = copy_pair_basis(400, w.copy_pairs)
    assert np.abs(As @ U).max() <= 1e-14
    assert np.abs(A @ U).max() <= 1e-12 * abs(A).max()
    Gd, Gs = (A.T @ A).toarray(), (As.T @ As).toarray()
    assert effective_condition(Gs, w.nullity) < effective_condition(Gd, w.nullity) / 10


def test_inner_preconditioned_solve_on_badly_scaled_rows():
    """Rows scaled over 3 decades: the plain method does not find the null space within
    its budget, the inner-preconditioned one finds all of it."""
    from oracle import copy_pair_basis
    from workloads import rectangular_copies_scaled
    w = rectangular_copies_scaled(23, 4500, 3000, 6, 3.0)
    A = w.A.to_scipy()
    pre = lanczos_nullspace(A, "normal", 2, 60, tol=1e-10, seed=9, inner=True)
    assert pre.N == 6
    assert principal_sine(pre.X, copy_pair_basis(3000, w.copy_pairs)) <= 1e-8
    plain = lanczos_nullspace(A, "normal", 2, 60, tol=1e-10, seed=9, max_matvec=10 * pre.stats["matvecs"])
    assert plain.N < 6


@pytest.mark.parametrize("variant", ["outer", "inner"])
def test_omega_bounds_hold_for_the_preconditioned_operators(variant):
    """Sec. 4.2's W recurrence bounds the true ||Q_k^T Q_{l+1}|| for any symmetric
    operator it is run on: every W entry of the (partially reorthogonalized) run still
    dominates the true inner products, locked rows included, for B_R (outer, reading P2's
    first-cycle bound) and for B_L (inner)."""
    from workloads import rectangular_copies_scaled
    worst = [0.0]
    seen = [0]

    def probe(j, Z, X, col, colX, dd):
        Qn = Z[:, (j + 1) * dd:(j + 2) * dd]
        for b in range(j + 1):
            true = np.linalg.norm(Z[:, b * dd:(b + 1) * dd].T @ Qn, 2)
            if col[b] < 1e-3:
                worst[0] = max(worst[0], true / col[b])
        if X.shape[1]:
            worst[0] = max(worst[0], float(np.max(np.abs(X.T @ Qn).max(axis=1) / colX)))
            seen[0] += 1

    if variant == "outer":
        w = laplacian_grid_components(3, 6, 8, 16)
        r = lanczos_nullspace(w.A.to_scipy(), "spd", 1, 30, seed=9, probe=probe, refine=False, precond=0.1)
    else:
        w = rectangular_copies_scaled(5, 900, 600, 4, 3.0)
        r = lanczos_nullspace(w.A.to_scipy(), "normal", 2, 60, seed=9, probe=probe, refine=False, inner=True)
    assert r.N == w.nullity
    assert seen[0] > 0
    assert worst[0] <= 1.0, worst[0]
