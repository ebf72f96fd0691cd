"""Full-size parity of configurations 2 (d = 4), 3 and 4, through the C ABI.

The oracle cannot run at these sizes, so the result is checked against what the
problem fixes at any size:
  * nullity: bit-exact against the component count (incidence matrix: one null
    vector per connected component) or the 300 planted column copies;
  * basis: largest principal-angle sine against the closed form (normalised
    component indicators; (e_src + e_copy)/sqrt(2) for the copies), <= 1e-6 on
    the FP64 path and <= 1e-5 on the mixed path after FP64 refinement;
  * residual ||A X||_F / ||A||_2 <= 1e-8, recomputed here with PyTorch's sparse
    product and a power-iteration ||A||_2 (not read from the library's stats);
  * orthonormality: ||X^T X - I||_F <= n N u (the paper's level for a computed
    orthonormal basis, Sec. 5) and max |X^T X - I| <= 32 sqrt(n) u (a few times the
    rounding error of one FP64 inner product of length n).
The launch configuration is the one bench.py times for these workloads.
"""

import numpy as np
import pytest

from gpu_checks import device_csr, norm2_power, residual_ratio, indicator_sine, copy_pair_sine, orthonormality
from workloads import make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ns(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2407_04634_gb300 import nullspace
    return nullspace


def solve_and_check(ns, w, seed, d, R, precision, sine_bar):
    import torch
    A = w.A
    h = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, seed, w.mode)
    r = h.solve(d, R, 1e-10, precision=precision)
    assert r.status == ns.NS_OK
    assert r.nullity == w.nullity
    X = torch.empty((r.nullity, A.n), dtype=torch.float64, device="cuda")
    h.basis(out=X)
    h.close()
    X = X.T
    As = A.to_scipy()
    Ad = device_csr(As)
    AdT = device_csr(As.T.tocsr()) if w.mode == "normal" else None
    normA = norm2_power(Ad, AdT)
    res = residual_ratio(Ad, X, normA)
    if w.labels is not None:
        sine = indicator_sine(w.labels, X)
    else:
        sine = copy_pair_sine(w.copy_pairs, A.n, X)
    orth = orthonormality(X)
    del X, Ad, AdT
    torch.cuda.empty_cache()
    assert sine <= sine_bar, sine
    assert res <= 1e-8, res
    n, N = A.n, w.nullity
    u = 2.0**-52
    assert orth[1] <= n * N * u, orth
    assert orth[0] <= 32.0 * np.sqrt(n) * u, orth
    return r


@pytest.fixture(scope="module")
def incidence():
    w, _ = make_config(3)
    return w


@pytest.fixture(scope="module")
def copies():
    w, _ = make_config(4)
    return w


def test_config2_full_size_d4(ns):
    """Laplacian n = 1e6, 500 components, d = 4, restart 120, FP64."""
    w, _ = make_config(2)
    solve_and_check(ns, w, 1001, 4, 120, "fp64", 1e-6)


@pytest.mark.parametrize("precision,bar", [("mixed", 1e-5), ("fp64", 1e-6)])
def test_config3_incidence_full_size(ns, incidence, precision, bar):
    """Incidence matrix 8e6 x 2e6, 1000 components: nullity 1000, d = 4, restart 160."""
    assert incidence.A.m == 8_000_000 and incidence.A.n == 2_000_000 and incidence.nullity == 1000
    solve_and_check(ns, incidence, 1002, 4, 160, precision, bar)


def test_config4_copies_full_size(ns, copies):
    """3e6 x 2e6, 12 N(0,1) entries per row, 300 planted sign-flipped copies: nullity 300,
    d = 2, restart 150, mixed path with FP64 refinement, FP32 values given as FP32."""
    assert copies.A.m == 3_000_000 and copies.A.n == 2_000_000 and copies.nullity == 300
    w = copies
    import copy
    w32 = copy.copy(w)
    w32.A = copy.copy(w.A)
    w32.A.vals = w.A.vals.astype(np.float32)  # exact: the values are FP32 numbers
    solve_and_check(ns, w32, 1003, 2, 150, "mixed", 1e-5)
