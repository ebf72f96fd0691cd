"""The large-block variant (Sec. 5.3.2, Table tabCHLB): no perturbation (eps = 0) and a
block size at least the nullity, against the oracle (reading L1 for the null test)."""

import numpy as np
import pytest

from oracle import lanczos_nullspace, principal_sine, copy_pair_basis, indicator_basis
from workloads import rectangular_copies, laplacian_er_components

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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_block_unperturbed_finds_every_copy(ns, precision):
    w = rectangular_copies(23, 4500, 3000, 6)
    ref = lanczos_nullspace(w.A.to_scipy(), "normal", 8, 64, tol=1e-10, seed=9, eps=0.0)
    h = handle(ns, w, 9)
    r = h.solve(8, 64, 1e-10, precision=precision, eps=0.0)
    assert r.nullity == ref.N == 6
    bar = 1e-6 if precision == "fp64" else 1e-5
    X = h.basis()
    assert principal_sine(X, copy_pair_basis(3000, w.copy_pairs)) <= bar
    assert principal_sine(X, ref.X) <= bar


def test_unperturbed_small_block_misses_null_vectors(ns):
    """d < N without the perturbation: the block Krylov space holds at most d vectors of
    the N-fold null eigenspace (the reason for eps D)."""
    w = rectangular_copies(23, 4500, 3000, 6)
    h = handle(ns, w, 9)
    r = h.solve(2, 16, 1e-10, check=False, eps=0.0)
    assert r.nullity < 6
    assert h.solve(2, 16, 1e-10, eps=1e-3).nullity == 6


def test_large_block_on_a_laplacian(ns):
    w = laplacian_er_components(3, 5, 80, 0.06)
    ref = lanczos_nullspace(w.A.to_scipy(), "spd", 8, 64, tol=1e-10, seed=9, eps=0.0)
    h = handle(ns, w, 9)
    r = h.solve(8, 64, 1e-10, eps=0.0)
    assert r.nullity == ref.N == 5
    assert principal_sine(h.basis(), indicator_basis(w.labels)) <= 1e-6
