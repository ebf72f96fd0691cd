"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed block) makes at least one of them fail.
"""

import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import (lanczos_nullspace, refine_null, principal_sine, indicator_basis,
                    copy_pair_basis, components, philox4x32_10, uniform01, gaussian,
                    perturbation_diagonal, start_block, Operator)
from workloads import (make_config, laplacian_cycle_components, incidence_cycle_components,
                       rectangular_copies, diag_example, tiny_planted)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox -----

def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(*v[:4], *v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_and_gaussian_streams():
    u = uniform01(7, 0, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = gaussian(7, 1, 200001)
    assert z.size == 200001 and np.isfinite(z).all()
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1.5e-2
    # independent streams and seeds
    assert not np.allclose(uniform01(7, 0, 16), uniform01(8, 0, 16))
    assert not np.allclose(uniform01(7, 0, 16), uniform01(7, 2, 16))
    # row-major layout of the start block: element e of the n x d block is z[e]
    Om = start_block(7, 5, 3)
    np.testing.assert_array_equal(Om.ravel(), gaussian(7, 1, 15))
    np.testing.assert_array_equal(perturbation_diagonal(7, 9), uniform01(7, 0, 9))


# -------------------------------------------------------- Lanczos relations ---

def _lanczos_relation_residual(op, Z, T, Qn, G):
    R = Z.shape[1]
    d = Qn.shape[1]
    E = np.zeros((d, R))
    E[:, R - d:] = np.eye(d)
    return np.linalg.norm(op.apply(Z) - Z @ T - Qn @ G @ E)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_alg1_block_lanczos_relation(d):
    """Alg. 1 with full reorthogonalization: B Z = Z T + Q_{l+1} Gamma_l E_l^T to rounding,
    Z orthonormal, T = Z^T B Z (pins reading R1 and the block placement of T)."""
    w = laplacian_cycle_components(11, 600, 3, 6, "uniform", 100, 300)
    A = w.A.to_scipy()
    R = 30 * d
    r = lanczos_nullspace(A, "spd", d, R, seed=5, restart=False, reorth="full")
    op = Operator(A, "spd", 1e-3, r.D)
    Z, T = r.Z, r.T
    assert np.linalg.norm(Z.T @ Z - np.eye(R)) < 1e-12
    assert _lanczos_relation_residual(op, Z, T, r.Qnext, r.Gamma_last) < 1e-12 * r.normB
    np.testing.assert_allclose(T, Z.T @ op.apply(Z), atol=1e-12 * r.normB)
    if d > 1:  # a transposed Gamma block would break the relation
        Tbad = T.copy()
        for b in range(R // d - 1):
            blk = Tbad[(b + 1) * d:(b + 2) * d, b * d:(b + 1) * d].copy()
            Tbad[(b + 1) * d:(b + 2) * d, b * d:(b + 1) * d] = blk.T
            Tbad[b * d:(b + 1) * d, (b + 1) * d:(b + 2) * d] = blk
        assert _lanczos_relation_residual(op, Z, Tbad, r.Qnext, r.Gamma_last) > 1e-3


@pytest.mark.parametrize("d", [1, 2])
def test_restarted_krylov_schur_relation(d):
    """After thick restarts (Sec. 4.1) the arrow-plus-block-tridiagonal T of Eq. (defT),
    with Theta, F = R Gamma V_Z(last, kept) (reading R8), still satisfies
    B Z = Z T + Q_{l+1} Gamma E^T.  Locking drops the residuals rho_k of the locked
    Ritz pairs (their directions are projected out of later blocks), so the relation
    holds up to ||rho||_2 plus rounding."""
    w = laplacian_cycle_components(12, 800, 4, 6, "uniform", 100, 300)
    A = w.A.to_scipy()
    r = lanczos_nullspace(A, "spd", d, 24 * d, seed=3, reorth="full", refine=False, record=True,
                          max_matvec=400 * d)
    op = Operator(A, "spd", 1e-3, r.D)
    cycles = r.stats["cycles"]
    assert len(cycles) >= 3 and any(c["k0"] > 0 for c in cycles)
    for c in cycles:
        tol = 1e-12 * r.normB + 1.01 * np.linalg.norm(c["x_rho"])
        assert _lanczos_relation_residual(op, c["Z"], c["T"], c["Qnext"], c["Gamma_last"]) < tol
        np.testing.assert_allclose(c["T"], c["Z"].T @ op.apply(c["Z"]), atol=tol)
    assert max(np.linalg.norm(c["x_rho"]) for c in cycles) > 0  # locking happened


@pytest.mark.parametrize("d", [1, 2])
def test_omega_recurrence_bounds_true_orthogonality(d):
    """Sec. 4.2: every W entry bounds the true ||Q_k^T Q_{l+1}|| (also the rows of the
    retained Ritz blocks, of Q_{l0+1} and of the locked vectors, readings R2-R5)."""
    w = laplacian_cycle_components(13, 900, 6, 6, "uniform", 80, 250)
    A = w.A.to_scipy()
    worst = [0.0]
    seen = {"ritz": 0, "locked": 0}

    def probe(j, Z, X, col, colX, dd):
        Qn = Z[:, (j + 1) * dd:(j + 2) * dd]
        for b in range(j + 1):
            true = np.linalg.norm(Z[:, b * dd:(b + 1) * dd].T @ Qn, 2)
            if col[b] < 1e-3:
                worst[0] = max(worst[0], true / col[b])
        if X.shape[1]:
            true = np.abs(X.T @ Qn).max(axis=1)
            worst[0] = max(worst[0], float(np.max(true / colX)))
            seen["locked"] += 1
        seen["ritz"] += 1

    r = lanczos_nullspace(A, "spd", d, 30 * d, seed=9, probe=probe, refine=False)
    assert r.N == 6
    assert seen["locked"] > 10
    assert worst[0] <= 1.0, worst[0]


# ------------------------------------------------------ closed-form null spaces

def test_config1_laplacian_closed_form():
    w, p = make_config(1)
    A = w.A.to_scipy()
    ncc, lab = components(A)
    assert ncc == 20
    r = lanczos_nullspace(A, "spd", p["d"], p["restart"], tol=p["tol"], seed=1000)
    assert r.converged and r.N == 20
    U = indicator_basis(w.labels)
    assert principal_sine(U, r.X) <= 1e-9
    assert np.linalg.norm(A @ r.X) / r.normA <= 1e-8
    # orthonormality criterion of Sec. 5.3.1: ||V^T V - I||_F <= n N u
    assert np.linalg.norm(r.X.T @ r.X - np.eye(r.N)) <= A.shape[1] * r.N * 2.0**-52


@pytest.mark.parametrize("d", [1, 4])
def test_cycle_laplacian_twin_of_config2(d):
    w = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50)
    A = w.A.to_scipy()
    r = lanczos_nullspace(A, "spd", d, 120, tol=1e-10, seed=1001)
    assert r.converged and r.N == 15
    assert principal_sine(indicator_basis(w.labels), r.X) <= 1e-9
    assert np.linalg.norm(A @ r.X) / r.normA <= 1e-8


def test_incidence_twin_of_config3():
    w = incidence_cycle_components(22, 8000, 8, 8, 100, 3900 // 4)
    A = w.A.to_scipy()
    assert components(A)[0] == 8
    r = lanczos_nullspace(A, "normal", 4, 80, tol=1e-10, seed=1002)
    assert r.converged and r.N == 8
    assert principal_sine(indicator_basis(w.labels), r.X) <= 1e-9
    assert np.linalg.norm(A @ r.X) / r.normA <= 1e-8


def test_copied_columns_twin_of_config4():
    w = rectangular_copies(23, 4500, 3000, 6)
    A = w.A.to_scipy()
    r = lanczos_nullspace(A, "normal", 2, 60, tol=1e-10, seed=1003)
    assert r.converged and r.N == 6
    # distance to null(A) <= ||A x|| / sigma_min; here sigma_min ~ 0.3 and the refinement
    # stops at ||A x|| <= 1e-10 ||A||, hence a 1e-8 bound on the sine
    assert principal_sine(copy_pair_basis(3000, w.copy_pairs), r.X) <= 1e-8
    assert np.linalg.norm(A @ r.X) / r.normA <= 1e-8


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_planted_against_dense_svd(seed):
    """Brute force: nullity and null space from a dense SVD (rank threshold 1e-10 ||A||)."""
    w = tiny_planted(seed, 150, 120, 7)
    A = w.A.to_scipy()
    Ad = A.toarray()
    U, s, Vt = np.linalg.svd(Ad)
    rank = int((s > 1e-10 * s[0]).sum())
    N = Ad.shape[1] - rank
    assert N == 7
    Vnull = Vt[rank:].T
    r = lanczos_nullspace(A, "normal", 1, 30, tol=1e-10, eps=1e-3 * min(1.0, (s[rank - 1] ** 2)), seed=seed)
    assert r.N == N
    # every refined column has ||A x|| <= 1e-10 ||A||, hence distance to null(A)
    # <= 1e-10 ||A|| / sigma_min and a sine <= sqrt(N) times that
    assert principal_sine(Vnull, r.X) <= 1.01 * np.sqrt(N) * 1e-10 * s[0] / s[rank - 1]


# ----------------------------------------------------- the diagonal example ---

@pytest.mark.slow
def test_diag_example_perturbed_finds_all_64():
    """Sec. 1, eq. (matrixA): with the random perturbation, d = 1 recovers all 64."""
    w = diag_example()
    A = w.A.to_scipy()
    r = lanczos_nullspace(A, "spd", 1, 128, tol=1e-10, seed=64)
    assert r.N == 64
    E = np.zeros((A.shape[0], 64))
    E[np.arange(64), np.arange(64)] = 1.0
    assert principal_sine(E, r.X) <= 1e-9


@pytest.mark.slow
@pytest.mark.parametrize("d,expect_full", [(1, False), (2, False), (4, False), (64, True)])
def test_diag_example_unperturbed_block_lanczos(d, expect_full):
    """Table tabintro: eps = 0, full reorthogonalization, 1024 matvecs, threshold 1e-4.
    Small blocks report more than d but fewer than 64 zeros; d = 64 finds all 64."""
    w = diag_example()
    A = w.A.to_scipy()
    r = lanczos_nullspace(A, "spd", d, 1024, eps=0.0, seed=d, restart=False, reorth="full")
    count = int((r.theta < 1e-4).sum())
    if expect_full:
        assert count == 64
    else:
        assert d < count < 64


# ------------------------------------------------------- theory invariants ---

def test_unrefined_output_bounds_spd():
    """Thm thmVANg (SPD form, Sec. 5.2): ||V^T A V|| <= eps^2 / (sigma^2 - eps) for the
    invariant subspace of B; the locked Ritz vectors meet it up to their residual."""
    w = laplacian_cycle_components(31, 600, 4, 6, "uniform", 100, 200)
    A = w.A.to_scipy()
    ev = np.linalg.eigvalsh(A.toarray())
    sig2 = ev[4]  # smallest nonzero eigenvalue plays the role of sigma^2
    eps = 1e-3
    r = lanczos_nullspace(A, "spd", 1, 40, tol=1e-10, eps=eps, seed=4, refine=False)
    V = r.X_lanczos
    assert r.N == 4
    assert np.linalg.norm(V.T @ (A @ V), 2) <= 1.01 * eps**2 / (sig2 - eps) + 1e-12
    assert np.all(r.x_theta < 3 * eps)  # Remark cormain
    assert np.linalg.norm(V.T @ V - np.eye(4)) <= 600 * 4 * 2.0**-52


def test_unrefined_output_bounds_normal():
    """Thm thmVANg: ||A V_N|| <= eps (sigma^2 - eps)^{-1/2}; Remark cormain:
    ||A V||^2 <= 161 eps^2 / (30 sigma^2)."""
    w = rectangular_copies(32, 900, 600, 4)
    A = w.A.to_scipy()
    s = np.linalg.svd(A.toarray(), compute_uv=False)
    sig2 = s[-5] ** 2
    eps = 1e-3
    assert eps < sig2 / 3
    r = lanczos_nullspace(A, "normal", 1, 40, tol=1e-10, eps=eps, seed=5, refine=False)
    V = r.X_lanczos
    assert r.N == 4
    nAV = np.linalg.norm(A @ V, 2)
    assert nAV <= 1.01 * eps / np.sqrt(sig2 - eps)
    assert nAV**2 <= 1.01 * 161 * eps**2 / (30 * sig2)


def test_single_vector_scaling_with_eps():
    """Table tabConNull: lambda_N(T) = O(eps), ||AV|| = O(eps), ||V^T A V|| = O(eps^2)
    (Alg. 1, d = 1, full reorthogonalization, SPD form B = A + eps D)."""
    w = laplacian_cycle_components(33, 400, 4, 6, "uniform", 80, 120)
    A = w.A.to_scipy()
    N = 4
    epss = 4.0 ** -np.arange(4, 8)
    lam, av, vav = [], [], []
    for eps in epss:
        r = lanczos_nullspace(A, "spd", 1, 300, eps=eps, seed=6, restart=False, reorth="full")
        V = r.Z @ r.VZ[:, :N]
        lam.append(r.theta[N - 1])
        av.append(np.linalg.norm(A @ V, 2))
        vav.append(np.linalg.norm(V.T @ (A @ V), 2))
    sl = lambda y: np.polyfit(np.log(epss), np.log(y), 1)[0]  # noqa: E731
    assert abs(sl(lam) - 1) < 0.2
    assert abs(sl(av) - 1) < 0.2
    assert abs(sl(vav) - 2) < 0.3


# ------------------------------------------------------------- refinement ---

@pytest.mark.parametrize("mode", ["spd", "normal"])
def test_refinement_is_orthogonal_projection(mode):
    """CG (spd) / CGLS (normal) from delta = 0 converges to x - P_range x = P_null x."""
    if mode == "spd":
        w = laplacian_cycle_components(41, 300, 3, 6, "uniform", 80, 120)
    else:
        w = rectangular_copies(41, 450, 300, 3)
    A = w.A.to_scipy()
    Ad = A.toarray()
    rng = np.random.default_rng(0)
    Xin = rng.standard_normal((A.shape[1], 5))
    _, s, Vt = np.linalg.svd(Ad)
    rank = int((s > 1e-10 * s[0]).sum())
    P = Vt[rank:].T @ Vt[rank:]
    Xr, info = refine_null(A, mode, Xin, 1e-12 * s[0], 2000)
    assert info["failed"] == 0
    np.testing.assert_allclose(Xr, P @ Xin, atol=1e-9)


# ------------------------------------------------------------ generators ---

def test_generators_match_planted_structure():
    w, _ = make_config(1)
    assert w.A.n == 2000 and components(w.A.to_scipy())[0] == 20
    w = laplacian_cycle_components(3, 5000, 7)
    assert components(w.A.to_scipy())[0] == 7
    assert np.allclose(w.A.to_scipy() @ indicator_basis(w.labels), 0)
    w = incidence_cycle_components(3, 4000, 5, 8, 100, 1500)
    assert w.A.m == 4 * 4000 and w.A.nnz == 2 * w.A.m
    assert np.allclose(w.A.to_scipy() @ indicator_basis(w.labels), 0)
    w = rectangular_copies(3, 3000, 2000, 5)
    assert np.abs(w.A.to_scipy() @ copy_pair_basis(2000, w.copy_pairs)).max() == 0.0
    cols = np.bincount(w.A.colind, minlength=2000)
    assert cols.min() >= 8


@pytest.mark.parametrize("theta", [1e-9, 1e-6, 1e-3, 0.3, 1.2])
def test_principal_sine_of_a_known_rotation(theta):
    """Principal angles (Def. defPA): rotating one basis vector of span(U) by theta
    towards a vector orthogonal to span(U) gives a largest principal angle of exactly
    theta, so principal_sine must return sin(theta) (both branches: the residual norm
    at small angles, the cosine at large ones), independently of the basis chosen for
    span(X) and of the other, unrotated columns."""
    from oracle import principal_sine
    rng = np.random.default_rng(7)
    n, k = 500, 6
    Q, _ = np.linalg.qr(rng.standard_normal((n, k + 1)))
    U, v = Q[:, :k], Q[:, k]
    X = U.copy()
    X[:, 2] = np.cos(theta) * U[:, 2] + np.sin(theta) * v
    M = rng.standard_normal((k, k))  # any other basis of the same span
    s = principal_sine(U, X @ M)
    assert abs(s - np.sin(theta)) <= 1e-12 + 1e-9 * np.sin(theta)
    assert principal_sine(U, U @ M) <= 1e-14
    assert principal_sine(U, X[:, :k - 1]) == 1.0  # unequal dimensions


@pytest.mark.parametrize("d", [1, 2])
def test_omega_bounds_with_ritz_norm_estimate(d):
    """Reading M4 (u_d from 1.1 x the largest Ritz value once a cycle has run) on a
    matrix whose cheap norm bound R9 is loose (N(0,1) values, normal form): u_d drops
    well below its R9 value, and every W entry still bounds the true ||Q_k^T Q_{l+1}||
    of the (partially reorthogonalized) run, locked rows included."""
    from workloads import rectangular_copies
    w = rectangular_copies(31, 900, 600, 4)
    A = w.A.to_scipy()
    worst = [0.0]

    def probe(j, Z, X, col, colX, dd):
        Qn = Z[:, (j + 1) * dd:(j + 2) * dd]
        for b in range(j + 1):
            true = np.linalg.norm(Z[:, b * dd:(b + 1) * dd].T @ Qn, 2)
            if col[b] < 1e-3:
                worst[0] = max(worst[0], true / col[b])
        if X.shape[1]:
            worst[0] = max(worst[0], float(np.max(np.abs(X.T @ Qn).max(axis=1) / colX)))

    r = lanczos_nullspace(A, "normal", d, 30 * d, seed=5, probe=probe, refine=False)
    ref = lanczos_nullspace(A, "normal", d, 30 * d, seed=5, refine=False, ud_rule="bound")
    assert r.N == ref.N == 4
    assert r.u_d < 0.5 * ref.u_d  # the Ritz estimate is much tighter than R9 here
    assert worst[0] <= 1.0, worst[0]


def test_slow_start_waits_for_the_first_lock():
    """d = dim K / 8 (d = 8, dim K = 64): the first cycles converge nothing, so there is
    no speed estimate yet; the termination test of Sec. 4.3 must not stop the iteration
    before the smallest Ritz value has settled, and the planted nullity is found for
    every block size of the sweep (Sec. 5.3.1), with more B applications for larger d."""
    w = rectangular_copies(35, 6000, 4000, 10)
    mv = {}
    for d in (8, 2):
        r = lanczos_nullspace(w.A.to_scipy(), "normal", d, 64, tol=1e-10, seed=11)
        assert r.N == 10, d
        assert principal_sine(r.X, copy_pair_basis(4000, w.copy_pairs)) <= 1e-8
        mv[d] = r.stats["matvecs"]
    assert mv[8] > mv[2]


def test_unperturbed_block_lanczos_needs_block_size_at_least_the_nullity():
    """Sec. 5.3.2: without the perturbation (eps = 0) the null eigenvalue is N-fold and a
    block Krylov space holds at most d vectors of its eigenspace, so d < N misses null
    vectors while the large-block variant d >= N finds them all (reading L1 counts the
    rounding-level Ritz values as null)."""
    w = rectangular_copies(23, 4500, 3000, 6)
    A = w.A.to_scipy()
    big = lanczos_nullspace(A, "normal", 8, 64, tol=1e-10, seed=9, eps=0.0)
    assert big.N == 6
    assert principal_sine(big.X, copy_pair_basis(3000, w.copy_pairs)) <= 1e-8
    for d in (1, 2):
        small = lanczos_nullspace(A, "normal", d, 16 if d == 2 else 60, tol=1e-10, seed=9, eps=0.0)
        assert small.N < 6, d
    pert = lanczos_nullspace(A, "normal", 2, 16, tol=1e-10, seed=9, eps=1e-3)
    assert pert.N == 6
