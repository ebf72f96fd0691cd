"""Host-side helpers of bench.py, checked on the CPU.

closed_form_sine() is the basis check of the bench line: the largest principal-angle
sine between a computed basis and the workload's known null space, computed as
||(I - U U^T) X||_2 from an N x N Gram matrix.  It must agree with the oracle's
principal_sine (an SVD of U^T X) and react to a perturbed basis.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from oracle import lanczos_nullspace, principal_sine, indicator_basis, copy_pair_basis  # noqa: E402
from workloads import laplacian_cycle_components, rectangular_copies  # noqa: E402


def test_closed_form_sine_indicators():
    w = laplacian_cycle_components(21, 3000, 5, 8, "powerlaw", 50)
    r = lanczos_nullspace(w.A.to_scipy(), "spd", 1, 40, tol=1e-10, seed=3)
    U = indicator_basis(w.labels)
    assert bench.closed_form_sine(w, torch.as_tensor(r.X)) == pytest.approx(principal_sine(U, r.X), rel=1e-6)
    Xp = r.X.copy()
    Xp[:, 0] += 1e-3 * np.random.default_rng(0).standard_normal(Xp.shape[0])
    Xp, _ = np.linalg.qr(Xp)
    s = bench.closed_form_sine(w, torch.as_tensor(Xp))
    assert s == pytest.approx(principal_sine(U, Xp), rel=1e-9) and s > 1e-2


def test_closed_form_sine_copy_pairs():
    w = rectangular_copies(23, 4500, 3000, 6)
    r = lanczos_nullspace(w.A.to_scipy(), "normal", 2, 60, tol=1e-10, seed=3)
    U = copy_pair_basis(3000, w.copy_pairs)
    assert bench.closed_form_sine(w, torch.as_tensor(r.X)) == pytest.approx(principal_sine(U, r.X), rel=1e-6)


def test_independent_residual_and_norm_estimate():
    """The bench's residual check (sparse product + power-iteration ||A||_2), on CPU
    tensors: ||A||_2 from 150 power steps never exceeds the dense 2-norm and lies
    within 1e-3 of it (an underestimate only makes the residual ratio larger) for a small Laplacian and a rectangular matrix, and ||A X||_F / ||A||_2
    matches the dense computation."""
    import scipy.sparse as sp
    for w in (laplacian_cycle_components(21, 400, 3, 8, "powerlaw", 50), rectangular_copies(23, 450, 300, 4)):
        A = w.A.to_scipy()
        Ad = bench.device_csr(A, device="cpu")
        AdT = bench.device_csr(A.T.tocsr(), device="cpu") if w.mode == "normal" else None
        ref = float(np.linalg.norm(A.toarray(), 2))
        est = bench.norm2_power(Ad, AdT)
        assert ref * (1 - 1e-3) <= est <= ref * (1 + 1e-12)
        X = np.random.default_rng(0).standard_normal((A.shape[1], 5))
        r = bench.residual_ratio(Ad, torch.from_numpy(X), ref, chunk=2)
        assert abs(r - np.linalg.norm(A @ X) / ref) <= 1e-12 * r
