"""The thick-restart product Z V_Z(:, sel) (Alg. 2, Sec. 4.1) through ns_restart_product.

Every kernel is compared element by element with the FP64 product of the same
operands (numpy), within the first-order error bound of its arithmetic, on tiles
with a ragged last row tile, K = R not a multiple of the 64-column chunk, panel
widths d = 1..8, up to 256 output columns, and both output layouts (the
locked-candidate panel and the next basis blocks):
  * FP64 CUDA-core kernel: |out - ref| <= (R + 2) u64 (|Z| |V|);
  * FP32 CUDA-core kernel: against Z rounded to FP32, (R + 2) u32 (|Z32| |V|);
  * tensor cores, 3 bf16 slices (6 products): (R + 8) u32 (|Z32| |V|) -- the
    dropped slice products are below 3 u32 relative to the operands;
  * tensor cores, 2 bf16 slices (3 products, "3xBF16"): 3 * 2^-16 (|Z32| |V|) plus
    the FP32 accumulation -- each operand is carried to 16 bits;
  * tensor cores, exact FP64 slicing (8 integer slices, R <= 208): the FP64 bound
    plus R 2^-49 max_j |z_ij| max_j |v_jc| for the truncated slice tails and the
    dropped slice pairs (p + q >= 8).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U32, U64 = 2.0**-24, 2.0**-53


@pytest.fixture(scope="module")
def ns(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2407_04634_gb300 import nullspace
    return nullspace


def operands(n, R, nsel, seed):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, R)) / np.sqrt(n)
    V, _ = np.linalg.qr(rng.standard_normal((R, R)))
    sel = rng.permutation(R)[:nsel].astype(np.int32)
    return Z, V, sel


CASES = [  # n, d, R, nsel, nl
    (1000, 1, 120, 60, 0),
    (20011, 8, 208, 104, 8),
    (70001, 1, 120, 60, 0),
    (70001, 2, 150, 76, 0),
    (33333, 4, 160, 80, 16),
    (5000, 8, 448, 256, 0),
    (4097, 1, 60, 17, 17),
    (12345, 2, 40, 18, 6),
]


@pytest.mark.parametrize("n,d,R,nsel,nl", CASES)
@pytest.mark.parametrize("kind", ["fp64", "fp32", "tc3", "tc2", "tc_exact"])
def test_restart_product_matches_fp64(ns, n, d, R, nsel, nl, kind):
    if kind == "tc_exact" and R > 208:
        pytest.skip("the exact slicing serves R <= 208")
    Z, V, sel = operands(n, R, nsel, seed=n + R + nsel)
    if kind == "tc_exact":  # rows and columns of very different scales
        rng = np.random.default_rng(n)
        Z *= 2.0 ** rng.integers(-30, 4, size=(n, 1))
        V = V * 2.0 ** rng.integers(-20, 2, size=(1, R))
    prec = "fp64" if kind in ("fp64", "tc_exact") else "mixed"
    gemm = {"fp64": "cuda_cores", "fp32": "cuda_cores", "tc3": "tc3", "tc2": "tc2", "tc_exact": "tc_exact"}[kind]
    out = ns.restart_product(Z, V, sel, nl, d, prec, gemm)
    Zr = Z if prec == "fp64" else Z.astype(np.float32).astype(np.float64)
    ref = Zr @ V[:, sel]
    mag = np.abs(Zr) @ np.abs(V[:, sel])
    if kind == "fp64":
        bound = (R + 2) * U64 * mag
    elif kind == "tc_exact":
        scale = np.abs(Zr).max(axis=1)[:, None] * np.abs(V[:, sel]).max(axis=0)[None, :]
        bound = (R + 2) * U64 * mag + R * 2.0**-49 * scale
    elif kind == "fp32":
        bound = (R + 2) * U32 * mag + U32 * mag  # + the rounding of V to FP32
    elif kind == "tc3":
        bound = (R + 8) * U32 * mag
    else:
        bound = 3 * 2.0**-16 * mag + (R + 2) * U32 * mag
    err = np.abs(out - ref)
    assert np.all(err <= bound), (float((err / np.maximum(mag, 1e-300)).max()), float(err.max()))


def test_restart_product_tensor_cores_need_mixed_and_at_most_256_columns(ns):
    Z, V, sel = operands(100, 40, 20, 1)
    with pytest.raises(ns.NullspaceError):
        ns.restart_product(Z, V, sel, 0, 1, "fp64", "tc3")
    with pytest.raises(ns.NullspaceError):
        ns.restart_product(Z, V, sel, 0, 1, "mixed", "tc_exact")
    Z, V, sel = operands(100, 216, 20, 3)
    with pytest.raises(ns.NullspaceError):
        ns.restart_product(Z, V, sel, 0, 1, "fp64", "tc_exact")  # R > 208
    Z, V, sel = operands(300, 300, 272, 2)
    with pytest.raises(ns.NullspaceError):
        ns.restart_product(Z, V, sel, 0, 1, "mixed", "tc3")


@pytest.mark.parametrize("gemm", ["cuda_cores", "tc2", "tc3"])
@pytest.mark.parametrize("case", ["laplacian", "incidence"])
def test_mixed_solve_with_each_restart_kernel(ns, gemm, case):
    """A whole mixed-precision solve with each restart-product kernel: exact nullity,
    principal-angle sine <= 1e-5 against the closed form, residual <= 1e-8."""
    from oracle import principal_sine, indicator_basis, norm2_A
    from workloads import laplacian_cycle_components, incidence_cycle_components
    if case == "laplacian":
        w, d, R = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50), 1, 120
    else:
        w, d, R = incidence_cycle_components(22, 8000, 8, 8, 100, 3900 // 4), 4, 80
    A = w.A
    h = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, 2000, w.mode)
    r = h.solve(d, R, 1e-10, precision="mixed", gemm=gemm)
    assert r.status == ns.NS_OK and r.nullity == w.nullity
    X = h.basis()
    As = A.to_scipy()
    assert principal_sine(indicator_basis(w.labels), X) <= 1e-5
    assert np.linalg.norm(As @ X) / norm2_A(As, w.mode) <= 1e-8


@pytest.mark.parametrize("gemm", ["cuda_cores", "tc_exact"])
def test_fp64_solve_with_each_restart_kernel(ns, gemm):
    """A whole FP64 solve with the CUDA-core and the exact tensor-core restart product:
    exact nullity, sine <= 1e-6 against the indicators, residual <= 1e-8."""
    from oracle import principal_sine, indicator_basis, norm2_A
    from workloads import laplacian_cycle_components
    w = laplacian_cycle_components(21, 30000, 15, 8, "powerlaw", 50)
    A = w.A
    h = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, 1001, w.mode)
    r = h.solve(1, 120, 1e-10, gemm=gemm)
    assert r.status == ns.NS_OK and r.nullity == 15
    X = h.basis()
    As = A.to_scipy()
    assert principal_sine(indicator_basis(w.labels), X) <= 1e-6
    assert np.linalg.norm(As @ X) / norm2_A(As, "spd") <= 1e-8


@pytest.mark.parametrize("products", [0, 1])
def test_fp64_solve_with_each_product_arithmetic(ns, products):
    """FP64 solves with the Gram-Schmidt products in compensated FP32 pairs (0, the
    default) and in FP64 FMA (1): exact nullity, sine <= 1e-6, residual <= 1e-8."""
    from oracle import principal_sine, indicator_basis, norm2_A, lanczos_nullspace
    from workloads import incidence_cycle_components
    w = incidence_cycle_components(22, 8000, 8, 8, 100, 3900 // 4)
    A = w.A
    h = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, 1002, w.mode)
    r = h.solve(4, 80, 1e-10, fp64_products=products)
    assert r.status == ns.NS_OK and r.nullity == 8
    X = h.basis()
    As = A.to_scipy()
    ref = lanczos_nullspace(As, "normal", 4, 80, tol=1e-10, seed=1002)
    assert principal_sine(ref.X, X) <= 1e-6
    assert principal_sine(indicator_basis(w.labels), X) <= 1e-6
    assert np.linalg.norm(As @ X) / norm2_A(As, "normal") <= 1e-8
