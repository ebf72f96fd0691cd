"""Outer (Sec. 4.4.2) and inner (Sec. 4.4.1) preconditioning on the GPU against the oracle.

Colouring and renumbering are integer work: bit-exact.  The IC(0) factor: the
same pattern exactly, values within 1e-13 relative (the same operations in the same
order; FMA contraction may round differently).  The preconditioned operator: FP64
within 1e-12 of max |Y|, FP32 within 1e-4.  Solves: nullity equal to the oracle's,
bases within the principal-angle bars of the other parity tests.
"""

import numpy as np
import pytest

from oracle import lanczos_nullspace, principal_sine, indicator_basis
from oracle.precond import Preconditioner, PrecondOperator, jp_coloring
from workloads import (laplacian_grid_components, laplacian_er_components, laplacian_cycle_components,
                       rectangular_copies)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ns(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2407_04634_gb300 import nullspace
    return nullspace


def handle(ns, w, seed):
    A = w.A
    return ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, seed, w.mode)


TWINS = {
    "grid": lambda: laplacian_grid_components(41, 12, 10, 30),
    "er_config1": lambda: laplacian_er_components(42, 20, 100, 0.05),
    "cycles_config2": lambda: laplacian_cycle_components(43, 30000, 15, 8, "powerlaw", 50),
}


@pytest.mark.parametrize("name", sorted(TWINS))
def test_colouring_renumbering_and_factor_match_the_oracle(ns, name):
    w = TWINS[name]()
    seed = 77
    h = handle(ns, w, seed)
    info = h.precond_build(0.1)
    ref = Preconditioner(w.A.to_scipy(), seed, 0.1)
    assert np.array_equal(info["color"], ref.color)
    assert np.array_equal(info["perm"], ref.perm)
    assert info["ncolors"] == ref.color.max() + 1
    rp, ci, va = h.precond_factor(info["nnz_L"])
    L = ref.L
    assert np.array_equal(rp, L.indptr) and np.array_equal(ci, L.indices)
    assert np.abs(va - L.data).max() <= 1e-13 * np.abs(L.data).max()


@pytest.mark.parametrize("precision,d,tol", [("fp64", 1, 1e-12), ("fp64", 4, 1e-12), ("mixed", 2, 1e-4),
                                              ("mixed", 8, 1e-4)])
def test_preconditioned_operator_matches_the_oracle(ns, precision, d, tol):
    w = TWINS["grid"]()
    h = handle(ns, w, 5)
    h.precond_build(0.1)
    ref = Preconditioner(w.A.to_scipy(), 5, 0.1)
    D = h.perturbation()
    X = np.random.default_rng(d).standard_normal((w.A.n, d))
    Y = h.apply_precond(X, 1e-3, precision)
    Yr = PrecondOperator(ref, 1e-3, D).apply(X)
    assert np.abs(Y - Yr).max() <= tol * np.abs(Yr).max()


def test_shift_refactors_and_breakdown_is_reported(ns):
    w = TWINS["er_config1"]()
    h = handle(ns, w, 3)
    a = h.precond_build(0.1)
    rp, ci, va1 = h.precond_factor(a["nnz_L"])
    h.precond_build(0.5)
    _, _, va5 = h.precond_factor(a["nnz_L"])
    diag = rp[1:] - 1
    assert np.all(va5[diag] > va1[diag])
    # a symmetric matrix that is not positive definite: the second pivot is 1 - 4 < 0
    rp2 = np.array([0, 2, 4], dtype=np.int64)
    ci2 = np.array([0, 1, 0, 1], dtype=np.int32)
    h2 = ns.Handle(rp2, ci2, np.array([1.0, 2.0, 2.0, 1.0]), 2, 2, 1, "spd")
    with pytest.raises(ns.NullspaceError) as e:
        h2.precond_build(0.0)
    assert e.value.status == ns.NS_ERR_NUMERICAL


@pytest.mark.parametrize("name,precision,d", [("grid", "fp64", 1), ("grid", "mixed", 1), ("grid", "fp64", 4),
                                              ("er_config1", "fp64", 1), ("cycles_config2", "fp64", 1),
                                              ("cycles_config2", "mixed", 4)])
def test_preconditioned_solve_matches_the_oracle(ns, name, precision, d):
    w = TWINS[name]()
    seed = 123
    R = 60 if w.A.n < 5000 else 120
    ref = lanczos_nullspace(w.A.to_scipy(), "spd", d, R, tol=1e-10, seed=seed, precond=0.1)
    h = handle(ns, w, seed)
    r = h.solve(d, R, 1e-10, precision=precision, precond=1)
    assert r.nullity == ref.N == w.nullity
    X = h.basis()
    U = indicator_basis(w.labels)
    bar = 1e-6 if precision == "fp64" else 1e-5
    assert principal_sine(X, U) <= bar
    assert principal_sine(X, ref.X) <= bar
    A = w.A.to_scipy()
    assert np.linalg.norm(A @ X) / abs(A).sum(axis=1).max() <= 1e-8
    assert np.abs(X.T @ X - np.eye(r.nullity)).max() <= 1e-12


def test_preconditioning_cuts_matvecs_on_grids(ns):
    w = TWINS["grid"]()
    h = handle(ns, w, 9)
    plain = h.solve(1, 60, 1e-10)
    pre = h.solve(1, 60, 1e-10, precond=1)
    assert plain.nullity == pre.nullity == w.nullity
    assert pre.stats["matvecs"] < plain.stats["matvecs"]


def test_precond_options_are_checked(ns):
    w = rectangular_copies(23, 900, 600, 3)
    h = handle(ns, w, 1)
    assert h.solve(2, 20, 1e-10, check=False, precond=1).status == ns.NS_ERR_INVALID_ARG  # normal mode
    g = TWINS["grid"]()
    hg = handle(ns, g, 1)
    assert hg.solve(1, 60, 1e-10, check=False, precond=2).status == ns.NS_ERR_INVALID_ARG
    assert hg.solve(1, 60, 1e-10, check=False, precond=1, precond_shift=-1.0).status == ns.NS_ERR_INVALID_ARG


def test_preconditioned_resume_is_bit_identical(ns, tmp_path):
    w = TWINS["grid"]()
    h0 = handle(ns, w, 21)
    r0 = h0.solve(1, 60, 1e-10, precond=1, spmm_schedule=4)
    X0 = h0.basis().copy()
    path = str(tmp_path / "pc.ckpt")
    h1 = handle(ns, w, 21)
    r1 = h1.solve(1, 60, 1e-10, check=False, precond=1, spmm_schedule=4, max_matvec=r0.stats["matvecs"] // 2,
                  checkpoint_every=1, checkpoint_path=path)
    assert r1.status == ns.NS_ERR_NOT_CONVERGED
    assert ns.read_checkpoint(path)["precond"] == 0.1
    h2 = handle(ns, w, 21)
    assert h2.solve(1, 60, 1e-10, check=False, resume=1, checkpoint_path=path).status == ns.NS_ERR_INVALID_ARG
    r2 = h2.solve(1, 60, 1e-10, precond=1, resume=1, checkpoint_path=path)
    assert r2.stats["matvecs"] == r0.stats["matvecs"]
    assert np.array_equal(h2.basis(), X0)


# ------------------------------------------------------ inner (Sec. 4.4.1) ---

def test_inner_scaling_and_operator_match_the_oracle(ns):
    from oracle import Operator
    from oracle.precond import inner_scaled
    from workloads import rectangular_copies_scaled
    w = rectangular_copies_scaled(51, 3000, 2000, 5, 3.0)
    A = w.A.to_scipy()
    h = handle(ns, w, 4)
    s = h.inner_precond()
    q = np.asarray(A.multiply(A).sum(axis=1)).ravel()
    assert np.abs(s - 1.0 / np.sqrt(q)).max() <= 1e-15 * np.abs(s).max()
    D = h.perturbation()
    ref = Operator(inner_scaled(A), "normal", 1e-3, D)
    for precision, d, tol in (("fp64", 2, 1e-13), ("mixed", 4, 1e-5)):
        X = np.random.default_rng(d).standard_normal((w.A.n, d))
        Y = h.apply_precond(X, 1e-3, precision)
        Yr = ref.apply(X)
        assert np.abs(Y - Yr).max() <= tol * np.abs(Yr).max(), precision


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_inner_preconditioned_solve_matches_the_oracle(ns, precision):
    from oracle import copy_pair_basis
    from workloads import rectangular_copies_scaled
    w = rectangular_copies_scaled(23, 4500, 3000, 6, 3.0)
    ref = lanczos_nullspace(w.A.to_scipy(), "normal", 2, 60, tol=1e-10, seed=9, inner=True)
    h = handle(ns, w, 9)
    r = h.solve(2, 60, 1e-10, precision=precision, precond=2)
    assert r.nullity == ref.N == 6
    X = h.basis()
    bar = 1e-6 if precision == "fp64" else 1e-5
    assert principal_sine(X, copy_pair_basis(3000, w.copy_pairs)) <= bar
    assert principal_sine(X, ref.X) <= bar
    plain = h.solve(2, 60, 1e-10, check=False, precision=precision, max_matvec=10 * r.stats["matvecs"])
    assert plain.nullity < 6  # the badly scaled rows stall the plain method within that budget


def test_inner_precond_options_are_checked(ns):
    g = TWINS["grid"]()
    hg = handle(ns, g, 1)
    assert hg.solve(1, 60, 1e-10, check=False, precond=2).status == ns.NS_ERR_INVALID_ARG  # SPD handle
    with pytest.raises(ns.NullspaceError):
        hg.inner_precond()
