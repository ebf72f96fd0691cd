"""Parity of the batched persistent form (ns_batch_*) with the CPU oracle.

Every instance is an independent SPD problem B_i = A_i + eps D_i (Sec. 5.1
form, d = 1) with Philox key seed + i, so instance i is compared with the
oracle's solve of A_i under the same key.  Bars:
  * nullity: bit-exact against the oracle and against the planted component
    count (Laplacian nullity = number of connected components);
  * basis: largest principal-angle sine <= 1e-5 (FP32 Lanczos vectors, FP64
    refinement) against the oracle's basis and against the component
    indicators; ||A X||_F / ||A||_2 <= 1e-8; |X^T X - I| <= 1e-12;
  * replays of the captured graph and a direct launch give bit-identical bases
    (per-instance arithmetic does not depend on which CTA ran it).
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lanczos_nullspace, principal_sine, indicator_basis, norm2_A
from workloads import batched_laplacians, config_seed, make_config

pytestmark = pytest.mark.gpu

R, TOL, EPS = 40, 1e-5, 1e-3


@pytest.fixture(scope="module")
def ns(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2407_04634_gb300 import nullspace
    return nullspace


def check_instance(ns, b, i, w, oracle_seed=None):
    A = w.A.to_scipy()
    X = b.basis(i)
    N = X.shape[1]
    assert N == w.nullity
    assert np.abs(X.T @ X - np.eye(N)).max() <= 1e-12
    assert np.linalg.norm(A @ X) / norm2_A(A, "spd") <= 1e-8
    assert principal_sine(indicator_basis(w.labels), X) <= 1e-5
    if oracle_seed is not None:
        r = lanczos_nullspace(A, "spd", 1, R, TOL, EPS, oracle_seed)
        assert r["N"] == N
        assert principal_sine(r["X"], X) <= 1e-5


def test_small_batch_matches_oracle(ns):
    seed = 777
    ws = batched_laplacians(config_seed(5) + 11, 6, n_min=200, n_max=900)
    b = ns.Batch([w.A for w in ws], seed)
    b.solve(R, TOL, eps=EPS)
    N, S, I = b.results()
    assert list(S) == [0] * len(ws)
    assert list(N) == [w.nullity for w in ws]
    assert (I[:, 0] > 0).all()
    st = b.stats()
    assert st["graph"] == 1 and st["lanes"] in (1, 2, 4) and st["total_nullity"] == sum(w.nullity for w in ws)
    for i, w in enumerate(ws):
        check_instance(ns, b, i, w, oracle_seed=seed + i)


def test_graph_replay_and_direct_launch_bit_identical(ns):
    ws = batched_laplacians(config_seed(5) + 12, 9, n_min=150, n_max=600)
    b = ns.Batch([w.A for w in ws], 4242)
    b.solve(R, TOL, eps=EPS)
    first = [b.basis(i) for i in range(len(ws))]
    b.solve(R, TOL, eps=EPS)  # replay of the same graph
    assert b.stats()["graph"] == 1
    b.solve(R, TOL, eps=EPS, use_graphs=-1)
    assert b.stats()["graph"] == 0
    for i in range(len(ws)):
        np.testing.assert_array_equal(b.basis(i), first[i])


def test_queue_longer_than_grid(ns):
    """More instances than resident CTAs: every one is taken from the queue exactly once."""
    ws = batched_laplacians(config_seed(5) + 13, 700, n_min=80, n_max=400)
    seed = 99
    b = ns.Batch([w.A for w in ws], seed)
    b.solve(R, TOL, eps=EPS)
    N, S, I = b.results()
    assert b.stats()["grid"] < len(ws)
    assert (S == 0).all()
    assert list(N) == [w.nullity for w in ws]
    assert (I[:, 0] > 0).all() and (I[:, 4] > 0).all()
    for i in (0, 350, 699):
        check_instance(ns, b, i, ws[i], oracle_seed=seed + i if i != 350 else None)


def test_instance_equals_batch_of_one(ns):
    """An instance's result does not depend on the rest of the batch (seed + i keying):
    bit-identical when both batches ran the same kernel variant (the autotuner picks
    the SpMV lanes per batch, and lanes change the FP32 summation order), the same
    null space otherwise."""
    ws = batched_laplacians(config_seed(5) + 14, 4, n_min=200, n_max=500)
    b = ns.Batch([w.A for w in ws], 5000)
    b.solve(R, TOL, eps=EPS)
    one = ns.Batch([ws[2].A], 5002)
    one.solve(R, TOL, eps=EPS)
    X1, X4 = one.basis(0), b.basis(2)
    assert X1.shape == X4.shape
    if (one.stats()["lanes"], one.stats()["block"]) == (b.stats()["lanes"], b.stats()["block"]):
        np.testing.assert_array_equal(X1, X4)
    assert principal_sine(X1, X4) <= 1e-5


def test_invalid_arguments(ns):
    ws = batched_laplacians(config_seed(5) + 15, 2, n_min=90, n_max=90)
    b = ns.Batch([w.A for w in ws], 1)
    for kw in (dict(d=2), dict(R=70), dict(R=7), dict(tol=0.0)):
        st = b.lib.ns_batch_solve(b.h, kw.get("d", 1), kw.get("R", R), kw.get("tol", TOL), None)
        assert st == ns.NS_ERR_INVALID_ARG
    st = b.lib.ns_batch_solve(b.h, 1, 64, TOL, None)  # n = 90 < 64 + 34
    assert st == ns.NS_ERR_INVALID_ARG
    assert b.lib.ns_batch_results(b.h, None, None, None) == ns.NS_ERR_STATE
    A = ws[0].A
    bad = A.colind.copy()
    bad[3] = A.n  # column out of range
    with pytest.raises(ns.NullspaceError):
        ns.Batch([(A.rowptr, bad, A.vals)], 1)


def test_packed_basis_and_device_entry_checks(ns):
    """ns_batch_basis_packed returns every instance's basis back to back, identical to
    the per-instance calls; a non-finite value is rejected by the device-side checks."""
    ws = batched_laplacians(config_seed(5) + 17, 5, n_min=150, n_max=700)
    b = ns.Batch([w.A for w in ws], 321)
    b.solve(R, TOL, eps=EPS)
    P = b.basis_packed()
    ref = np.concatenate([b.basis(i).ravel(order="F") for i in range(len(ws))])
    np.testing.assert_array_equal(P, ref)
    import torch
    Pd = torch.empty(P.size, dtype=torch.float64, device="cuda")
    b.basis_packed(Pd)
    np.testing.assert_array_equal(Pd.cpu().numpy(), ref)
    A = ws[1].A
    bad = A.vals.copy()
    bad[7] = np.nan
    with pytest.raises(ns.NullspaceError):
        ns.Batch([ws[0].A, (A.rowptr, A.colind, bad)], 1)


def test_empty_rows_and_isolated_vertices(ns):
    """Isolated vertices (empty rows) are components of size one: e_k is a null vector."""
    ws = batched_laplacians(config_seed(5) + 16, 1, n_min=300, n_max=300)
    A = ws[0].A.to_scipy().tolil()
    n = A.shape[0]
    A2 = sp.block_diag([A, sp.csr_matrix((3, 3))]).tocsr()
    from workloads.graphs import CSR
    C = CSR.from_scipy(A2)
    b = ns.Batch([C], 31)
    b.solve(R, TOL, eps=EPS)
    N, S, _ = b.results()
    assert S[0] == 0 and N[0] == ws[0].nullity + 3
    X = b.basis(0)
    labels = np.concatenate([ws[0].labels, ws[0].labels.max() + 1 + np.arange(3)])
    assert principal_sine(indicator_basis(labels), X) <= 1e-5
    assert np.linalg.norm(A2 @ X) / norm2_A(A2, "spd") <= 1e-8
    assert n + 3 == X.shape[0]


@pytest.mark.slow
def test_full_size_4096_laplacians(ns):
    """4,096 Laplacians, n log-uniform in [200, 20000], 1-8 components: nullity exact
    everywhere (component counts), oracle parity on sampled instances."""
    ws, _ = make_config(5)  # the 4,096-instance workload the benchmark times
    seed = 1004
    b = ns.Batch([w.A for w in ws], seed)
    b.solve(R, TOL, eps=EPS)
    N, S, I = b.results()
    assert (S == 0).all()
    assert list(N) == [w.nullity for w in ws]
    sizes = np.array([w.A.n for w in ws])
    for i in (int(np.argmax(sizes)), int(np.argmin(sizes)), 2048):
        check_instance(ns, b, i, ws[i], oracle_seed=seed + i)
    for i in range(0, 4096, 97):
        w = ws[i]
        X = b.basis(i)
        assert np.linalg.norm(w.A.to_scipy() @ X) / norm2_A(w.A.to_scipy(), "spd") <= 1e-8


def test_fp32_values_give_bit_identical_batch(ns):
    """ns_batch_create with vals_is_fp32 = 1 (the Laplacians' values are FP32 numbers):
    the same per-instance results and bit-identical bases as the FP64 input, since the
    batched form's FP32 copy and FP64 widening are both exact."""
    ws = batched_laplacians(config_seed(5) + 18, 5, n_min=200, n_max=800)
    b64 = ns.Batch([w.A for w in ws], 606)
    b32 = ns.Batch([(w.A.rowptr, w.A.colind, w.A.vals.astype(np.float32)) for w in ws], 606)
    b64.solve(R, TOL, eps=EPS)
    b32.solve(R, TOL, eps=EPS)
    N64, S64, _ = b64.results()
    N32, S32, _ = b32.results()
    assert list(S32) == [0] * len(ws) and list(N32) == list(N64) == [w.nullity for w in ws]
    if (b64.stats()["lanes"], b64.stats()["block"]) == (b32.stats()["lanes"], b32.stats()["block"]):
        np.testing.assert_array_equal(b32.basis_packed(), b64.basis_packed())
    for i, w in enumerate(ws):
        check_instance(ns, b32, i, w)
