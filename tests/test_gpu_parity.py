"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Inputs are seeded synthetic matrices from `workloads`; expected values come
from the oracle or from closed forms (component indicators, planted copies).
Tolerances:
  * integer / index work (transpose, nullity): bit-exact;
  * FP64 products: |y_gpu - y_ref| <= 1e-13 (|B| |X|)_i elementwise (a few
    roundings per inner product of at most ~40 terms);
  * FP32 products: 1e-5 (|B| |X|)_i;
  * null-space bases: largest principal-angle sine <= 1e-6 (FP64 path) and
    <= 1e-5 (mixed path, after FP64 refinement) against the oracle's basis, and
    ||A X||_F / ||A||_2 <= 1e-8.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import (lanczos_nullspace, principal_sine, indicator_basis, copy_pair_basis, perturbation_diagonal,
                    start_block, Operator, norm2_A)
from workloads import (make_config, laplacian_cycle_components, incidence_cycle_components, rectangular_copies,
                       laplacian_er_components)

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


def abs_bound(w, X, eps, D):
    A = abs(w.A.to_scipy())
    Xa = np.abs(X)
    if w.mode == "normal":
        return A.T @ (A @ Xa) + eps * D[:, None] * Xa
    return A @ Xa + eps * D[:, None] * Xa


# ------------------------------------------------------------------ kernels ---

def test_perturbation_and_start_block_match_philox_streams(ns):
    w = laplacian_cycle_components(5, 3001, 3, 6, "uniform", 100, 2000)
    h = handle(ns, w, 12345)
    np.testing.assert_array_equal(h.perturbation(), perturbation_diagonal(12345, 3001))
    for d in (1, 3, 8):
        np.testing.assert_allclose(h.start_block(d), start_block(12345, 3001, d), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("make", ["incidence", "copies"])
def test_transpose_bit_exact(ns, make):
    if make == "incidence":
        w = incidence_cycle_components(7, 20011, 9, 8, 100, 4000)
    else:
        w = rectangular_copies(7, 30011, 20011, 13)
    h = handle(ns, w, 1)
    rp, ci, va = h.transpose(w.A.nnz)
    At = w.A.to_scipy().T.tocsr()
    At.sort_indices()
    np.testing.assert_array_equal(rp, At.indptr)
    np.testing.assert_array_equal(ci, At.indices)
    np.testing.assert_array_equal(va, At.data)


@pytest.mark.parametrize("mode", ["spd", "normal"])
@pytest.mark.parametrize("d", [1, 2, 4, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_apply_B_matches_oracle(ns, mode, d, precision):
    if mode == "spd":
        w = laplacian_cycle_components(9, 40009, 7, 8, "powerlaw", 50)
    else:
        w = rectangular_copies(9, 30007, 20011, 5)
    h = handle(ns, w, 77)
    rng = np.random.default_rng(d)
    X = rng.standard_normal((w.A.n, d))
    if precision == "mixed":
        X = X.astype(np.float32).astype(np.float64)
    eps = 1e-3
    D = h.perturbation()
    ref = Operator(w.A.to_scipy(), mode, eps, D).apply(X)
    Y = h.apply_B(X, eps, precision)
    bound = abs_bound(w, X, eps, D)
    tol = 1e-13 if precision == "fp64" else 1e-5
    assert np.all(np.abs(Y - ref) <= tol * bound + 1e-300)


def _balanced_matrix(seed, m, n, symmetric):
    """Sparse m x n matrix whose rows and columns hold nearly the same number of entries
    (so both A and A^T fit the sliced layout), with empty rows and m not a multiple of
    the 32-row slice."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(m):
        if i % 97 == 5:
            continue  # an empty row
        k = 11 + (i % 2)
        rows.append(np.full(k, i))
        cols.append((7 * i + 257 * np.arange(k) + 1) % n)
    M = sp.csr_matrix((rng.standard_normal(sum(len(r) for r in rows)), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m, n))
    if symmetric:
        M = (M + M.T).tocsr()
    return M


def _skewed_matrix(seed, m, n):
    """Sparse m x n matrix with empty rows (one whole 256-row tile among them), short
    rows, and a few rows of 600-3000 entries (tiles too long to stage in shared
    memory), m not a multiple of 256."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 12, size=m)
    lens[rng.choice(m, 5, replace=False)] = rng.integers(600, 3000, size=5)
    lens[rng.choice(m, 40, replace=False)] = 0
    lens[256:512] = 0
    rows = np.repeat(np.arange(m), lens)
    cols = np.concatenate([rng.choice(n, size=k, replace=False) for k in lens])
    vals = rng.standard_normal(rows.size)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, n))


@pytest.mark.parametrize("mode", ["spd", "normal"])
@pytest.mark.parametrize("d,precision", [(1, "fp64"), (1, "mixed"), (2, "fp64"), (4, "mixed"), (8, "fp64")])
@pytest.mark.parametrize("schedule", [64, 1, 4, 32, 128])
def test_apply_B_every_schedule(ns, mode, d, precision, schedule):
    """Every SpMM schedule (TMA-staged, 1/4/32 threads per row, sliced ELLPACK) against
    the oracle's operator, on rows from empty to 3000 entries and a ragged last tile;
    the sliced layout on a matrix of nearly uniform rows and columns (0-24 entries) with
    a ragged last slice, since long rows would exceed its padding limit."""
    from workloads.graphs import CSR, Workload
    if schedule == 128:
        M = _balanced_matrix(100 + d, 4099, 4099 if mode == "spd" else 3001, mode == "spd")
    else:
        M = _skewed_matrix(100 + d, 4099, 4099 if mode == "spd" else 3001)
    w = Workload("skewed", CSR.from_scipy(M), mode, 0)
    h = handle(ns, w, 5)
    rng = np.random.default_rng(schedule + 7)
    X = rng.standard_normal((w.A.n, d))
    if precision == "mixed":
        X = X.astype(np.float32).astype(np.float64)
    D = h.perturbation()
    ref = Operator(w.A.to_scipy(), mode, 1e-3, D).apply(X)
    Y = h.apply_B(X, 1e-3, precision, schedule)
    # first-order bound of a recursive sum of k terms: (k + 3) u sum |a x| per stage
    # (the +3 covers the eps D x term and the rounding of A to FP32); the normal form
    # adds the row length of its A^T stage
    k = int(np.diff(M.indptr).max()) + (int(np.diff(M.tocsc().indptr).max()) if mode == "normal" else 0)
    u = 2.0**-53 if precision == "fp64" else 2.0**-24
    assert np.all(np.abs(Y - ref) <= (k + 3) * u * abs_bound(w, X, 1e-3, D) + 1e-300)


def test_apply_B_rejects_unknown_schedule(ns):
    w = laplacian_cycle_components(3, 3001, 3, 6, "uniform", 100, 2000)
    h = handle(ns, w, 1)
    with pytest.raises(ns.NullspaceError):
        h.apply_B(np.ones((w.A.n, 1)), 1e-3, "fp64", 3)


@pytest.mark.parametrize("k", [3, 17, 64, 120, 160])
def test_syev_matches_dense_eigensolver(ns, k):
    rng = np.random.default_rng(k)
    M = rng.standard_normal((k, k))
    T = M + M.T
    if k >= 64:  # a cluster of tiny eigenvalues, as in the projected null-space problem
        Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
        ev = np.concatenate([1e-3 * (0.5 + 1e-6 * rng.random(k // 3)), 1 + 10 * rng.random(k - k // 3)])
        T = (Q * ev) @ Q.T
        T = 0.5 * (T + T.T)
    th, V = ns.syev(T)
    ref = np.linalg.eigvalsh(T)
    nrm = np.linalg.norm(T, 2)
    assert np.all(np.diff(th) >= 0)
    np.testing.assert_allclose(th, ref, atol=1e-12 * nrm)
    assert np.linalg.norm(T @ V - V * th) <= 1e-12 * nrm * k
    assert np.linalg.norm(V.T @ V - np.eye(k)) <= 1e-13 * k


@pytest.mark.parametrize("w", [1, 2, 4, 8])
@pytest.mark.parametrize("precision", ["fp64", "fp64_pairs", "mixed"])
def test_cgs2_projection(ns, w, precision):
    """CGS2 against a dense reference; fp64_pairs (FP64 data, compensated FP32-pair
    products, the FP64 path's default) meets the same bars as FP64 FMA."""
    rng = np.random.default_rng(w)
    n, K = 70001, 37
    V, _ = np.linalg.qr(rng.standard_normal((n, K)))
    W = rng.standard_normal((n, w)) + V[:, :w] * 3.0
    Wp, Cc = ns.project(V, W, precision)
    f64 = precision != "mixed"
    tol = 1e-13 if f64 else 2e-6
    assert np.abs(V.T @ Wp).max() <= tol * np.sqrt(n)
    ref = W - V @ (V.T @ W)
    assert np.abs(Wp - ref).max() <= (1e-12 if f64 else 1e-4)
    np.testing.assert_allclose(Cc, V.T @ W, atol=1e-11 if f64 else 1e-3)


@pytest.mark.parametrize("w", [2, 8])
def test_pair_products_are_as_accurate_as_fp64(ns, w):
    """Nearly orthogonal inputs (the partial-reorthogonalization case: |V^T W| ~ 1e-8
    from terms of size 1/n): the coefficients from compensated FP32 pairs are at least
    as close to an exactly rounded reference (computed in extended precision from the
    FP64 inputs) as those of FP64 FMA, and within 1e-15."""
    rng = np.random.default_rng(40 + w)
    n, K = 100003, 16
    V, _ = np.linalg.qr(rng.standard_normal((n, K)))
    W = rng.standard_normal((n, w))
    W -= V @ (V.T @ W)
    W /= np.linalg.norm(W, axis=0)
    W += 1e-8 * V[:, :w]
    Vl, Wl = V.astype(np.longdouble), W.astype(np.longdouble)
    ref = (Vl.T @ Wl).astype(np.float64)  # first pass of CGS2: C1 = V^T W
    _, C64 = ns.project(V, W, "fp64")
    _, Cdf = ns.project(V, W, "fp64_pairs")
    # C sums both passes; the second pass adds V^T (W - V C1) ~ rounding level
    e64 = np.abs(C64 - ref).max()
    edf = np.abs(Cdf - ref).max()
    assert edf <= 1e-15 and edf <= 4 * e64 + 1e-16


# ------------------------------------------------------------------- solves ---

def check_solution(w, X, N_expect, U_ref, sine_tol, normA=None):
    A = w.A.to_scipy()
    assert X.shape[1] == N_expect
    assert principal_sine(U_ref, X) <= sine_tol
    normA = normA or norm2_A(A, w.mode)
    assert np.linalg.norm(A @ X) / normA <= 1e-8
    assert np.linalg.norm(X.T @ X - np.eye(X.shape[1])) <= max(1e-12, A.shape[1] * X.shape[1] * 2.0**-52)


def test_config1_fp64_matches_oracle(ns):
    w, p = make_config(1)
    ref = lanczos_nullspace(w.A.to_scipy(), w.mode, p["d"], p["restart"], tol=p["tol"], seed=1000)
    h = handle(ns, w, 1000)
    r = h.solve(p["d"], p["restart"], p["tol"])
    assert r.status == ns.NS_OK
    assert r.nullity == ref.N == 20
    X = h.basis()
    check_solution(w, X, ref.N, ref.X, 1e-6)
    assert principal_sine(indicator_basis(w.labels), X) <= 1e-6


@pytest.mark.parametrize("d", [1, 2, 4, 8])
def test_cycle_laplacian_twin_fp64(ns, d):
    w = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50)
    ref = lanczos_nullspace(w.A.to_scipy(), "spd", d, 120, tol=1e-10, seed=1001)
    h = handle(ns, w, 1001)
    r = h.solve(d, 120, 1e-10)
    assert r.nullity == ref.N == 15
    check_solution(w, h.basis(), 15, ref.X, 1e-6)


def test_incidence_twin_fp64(ns):
    w = incidence_cycle_components(22, 8000, 8, 8, 100, 3900 // 4)
    ref = lanczos_nullspace(w.A.to_scipy(), "normal", 4, 80, tol=1e-10, seed=1002)
    h = handle(ns, w, 1002)
    r = h.solve(4, 80, 1e-10)
    assert r.nullity == ref.N == 8
    check_solution(w, h.basis(), 8, ref.X, 1e-6)


def test_copies_twin_fp64(ns):
    w = rectangular_copies(23, 4500, 3000, 6)
    ref = lanczos_nullspace(w.A.to_scipy(), "normal", 2, 60, tol=1e-10, seed=1003)
    h = handle(ns, w, 1003)
    r = h.solve(2, 60, 1e-10)
    assert r.nullity == ref.N == 6
    check_solution(w, h.basis(), 6, ref.X, 1e-6)


@pytest.mark.parametrize("case", ["laplacian", "incidence", "copies"])
def test_mixed_precision_twins(ns, case):
    if case == "laplacian":
        w = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50)
        d, R, U = 1, 120, indicator_basis(w.labels)
    elif case == "incidence":
        w = incidence_cycle_components(22, 8000, 8, 8, 100, 3900 // 4)
        d, R, U = 4, 80, indicator_basis(w.labels)
    else:
        w = rectangular_copies(23, 4500, 3000, 6)
        d, R, U = 2, 60, copy_pair_basis(3000, w.copy_pairs)
    h = handle(ns, w, 2000)
    r = h.solve(d, R, 1e-10, precision="mixed")
    assert r.nullity == w.nullity
    check_solution(w, h.basis(), w.nullity, U, 1e-5)


def test_long_restart_fp64(ns):
    """restart_len 448 in FP64: the restart products take the chunked kernel (the row-tile
    FP64 kernel stages all R basis columns and serves R <= 400)."""
    w = laplacian_cycle_components(24, 20000, 9, 8, "powerlaw", 50)
    h = handle(ns, w, 2002)
    r = h.solve(1, 448, 1e-10)
    assert r.nullity == 9
    check_solution(w, h.basis(), 9, indicator_basis(w.labels), 1e-6)


def test_block_size_8_mixed(ns):
    """d = 8: the merged partial-reorthogonalization panel is 16 columns wide."""
    w = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50)
    h = handle(ns, w, 2001)
    r = h.solve(8, 120, 1e-10, precision="mixed")
    assert r.nullity == 15
    check_solution(w, h.basis(), 15, indicator_basis(w.labels), 1e-5)


def test_full_rank_matrix_has_empty_null_space(ns):
    w = laplacian_er_components(3, 1, 400, 0.05)  # one connected component: nullity 1
    h = handle(ns, w, 5)
    r = h.solve(1, 40, 1e-10)
    assert r.nullity == 1
    # shift away the null space: A + I is nonsingular
    A = (w.A.to_scipy() + sp.identity(w.A.n)).tocsr()
    h2 = ns.Handle(A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, A.shape[0], A.shape[1], 5, "spd")
    r2 = h2.solve(1, 40, 1e-10)
    assert r2.nullity == 0


def test_max_matvec_reports_not_converged(ns):
    w = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50)
    h = handle(ns, w, 1001)
    r = h.solve(1, 120, 1e-10, check=False, max_matvec=200)
    assert r.status == ns.NS_ERR_NOT_CONVERGED


def test_calls_out_of_order_and_bad_sizes(ns):
    w = laplacian_cycle_components(21, 3000, 3, 8, "powerlaw", 50)
    h = handle(ns, w, 1)
    import ctypes
    N = ctypes.c_int64()
    assert h.lib.ns_nullity(h.h, ctypes.byref(N)) == ns.NS_ERR_STATE
    assert h.lib.ns_solve(h.h, 3, 30, 1e-10, None) == ns.NS_ERR_INVALID_ARG
    assert h.lib.ns_solve(h.h, 2, 31, 1e-10, None) == ns.NS_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config2_full_size_closed_form(ns, precision):
    """n = 1e6, 500 components: nullity and the indicator basis (closed form, any size)."""
    w, p = make_config(2)
    h = handle(ns, w, 1001)
    r = h.solve(1, 120, 1e-10, precision=precision)
    assert r.nullity == 500
    X = h.basis()
    U = indicator_basis(w.labels)
    assert principal_sine(U, X) <= (1e-6 if precision == "fp64" else 1e-5)
    A = w.A.to_scipy()
    assert np.linalg.norm(A @ X) / r.stats["normA"] <= 1e-8


# ------------------------------------------------ W recurrence (Sec. 4.2) ---

@pytest.mark.parametrize("d", [1, 2])
def test_omega_columns_match_oracle(ns, d):
    """Every W column of the first cycle (configuration 1, n = 2000, restart 60), as the
    CUDA recurrence produced it, against the oracle's recorded columns element by
    element.  The cycle triggers partial reorthogonalization several times, so the
    columns after each reset to u_d are covered too."""
    w, _ = make_config(1)
    R = 60
    ref = lanczos_nullspace(w.A.to_scipy(), w.mode, d, R, tol=1e-10, seed=1000, restart=False, record=True)
    h = handle(ns, w, 1000)
    Wg = h.trace_omega(d, R)
    nb = R // d
    assert Wg.shape == (nb + 1, nb + 1)
    rec = ref["Wrec"]
    assert len(rec) == nb - 1
    triggers = 0
    for col, newcol, newX in rec:
        np.testing.assert_allclose(Wg[:col, col], newcol[:col], rtol=1e-9, atol=0)
        assert np.all(Wg[col:, col] == 0)
        triggers += bool((newcol[:col] > ref.u_ro).any())
    assert np.all(Wg[:, :2] == 0)
    assert triggers >= 3


# ------------------------------------------------------ FP32 value input ----

@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fp32_values_give_the_same_solve(ns, precision):
    """ns_create with vals_is_fp32 = 1 on the configuration-4 twin (whose values are FP32
    numbers): the device holds the same FP32 and FP64 values as for the FP64 input (the
    copy and the widening are exact; checked on the transpose), and the solve gives the
    same nullity and the same null space.  The bases need not be bit-identical: each
    handle autotunes its SpMM schedule by timing, which may change summation orders."""
    w = rectangular_copies(23, 4500, 3000, 6)
    A = w.A
    h64 = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, 2000, w.mode)
    h32 = ns.Handle(A.rowptr, A.colind, A.vals.astype(np.float32), A.m, A.n, 2000, w.mode)
    r64 = h64.solve(2, 60, 1e-10, precision=precision)
    r32 = h32.solve(2, 60, 1e-10, precision=precision)
    assert r64.nullity == r32.nullity == w.nullity
    X64, X32 = h64.basis(), h32.basis()
    bar = 1e-5 if precision == "mixed" else 1e-6
    U = copy_pair_basis(3000, w.copy_pairs)
    assert principal_sine(U, X32) <= bar and principal_sine(U, X64) <= bar
    assert principal_sine(X64, X32) <= bar
    check_solution(w, X32, w.nullity, U, bar)
    rp, ci, va = h32.transpose(A.nnz)
    At = A.to_scipy().T.tocsr()
    At.sort_indices()
    np.testing.assert_array_equal(va, At.data)


def test_fp32_values_from_device_memory(ns):
    """FP32 values handed over in device memory (inputs_on_device = 1)."""
    import torch
    w = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50)
    A = w.A
    rp = torch.as_tensor(A.rowptr, device="cuda")
    ci = torch.as_tensor(A.colind, device="cuda")
    va = torch.as_tensor(A.vals.astype(np.float32), device="cuda")
    h = ns.Handle(rp, ci, va, A.m, A.n, 1001, w.mode)
    r = h.solve(1, 120, 1e-10, precision="mixed")
    assert r.nullity == 15
    check_solution(w, h.basis(), 15, indicator_basis(w.labels), 1e-5)
