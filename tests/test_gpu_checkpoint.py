"""Checkpoint / resume at thick restarts, and the block-size rule d = dim K / 16.

At a thick restart (Alg. 2, Sec. 4.1) the state of the iteration is small and
complete: the retained Ritz vectors with the next block, the arrow part of the
projected matrix, the W rows, the locked vectors and the counters.  A solve
resumed from a checkpoint must therefore continue exactly as the solve that ran
straight through: same nullity, same counters, and a bit-identical basis when
both use the same SpMM schedule (schedules sum a row in different orders).
"""

import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import indicator_basis, copy_pair_basis, principal_sine, lanczos_nullspace
from workloads import laplacian_cycle_components, rectangular_copies

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


CASES = {
    # name: (workload, d, restart_len, precision, fixed schedule)
    "laplacian_fp64_d1": (lambda: laplacian_cycle_components(31, 20000, 12, 8, "powerlaw", 50), 1, 60, "fp64", 8),
    "laplacian_mixed_d4": (lambda: laplacian_cycle_components(31, 20000, 12, 8, "powerlaw", 50), 4, 64, "mixed",
                           128),
    "copies_fp64_d2": (lambda: rectangular_copies(33, 4500, 3000, 6), 2, 40, "fp64", 4),
    "copies_mixed_d2": (lambda: rectangular_copies(33, 4500, 3000, 6), 2, 40, "mixed", 64),
}
SEED = 4242
COUNTERS = ("nullity", "matvecs", "restarts", "reorth_X", "reorth_Z", "breakdowns", "lock_events", "ghosts", "d")


def known_basis(w):
    return indicator_basis(w.labels) if w.mode == "spd" else copy_pair_basis(w.A.n, w.copy_pairs)


@pytest.fixture(scope="module")
def straight(ns):
    """Each case solved straight through with a fixed SpMM schedule."""
    out = {}
    for name, (mk, d, R, prec, sched) in CASES.items():
        w = mk()
        h = handle(ns, w, SEED)
        r = h.solve(d, R, 1e-10, precision=prec, spmm_schedule=sched)
        assert r.nullity == w.nullity
        assert r.stats["restarts"] >= 3, "the case must restart a few times to be interrupted"
        out[name] = (w, h.basis().copy(), r.stats)
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_resume_is_bit_identical_to_the_straight_solve(ns, straight, tmp_path, name):
    _, d, R, prec, sched = CASES[name]
    w, X_ref, st_ref = straight[name]
    path = str(tmp_path / "state.ckpt")
    budget = st_ref["matvecs"] // 2
    h1 = handle(ns, w, SEED)
    r1 = h1.solve(d, R, 1e-10, check=False, precision=prec, spmm_schedule=sched, max_matvec=budget,
                  checkpoint_every=1, checkpoint_path=path)
    assert r1.status == ns.NS_ERR_NOT_CONVERGED
    info = ns.read_checkpoint(path)
    assert info["matvecs"] == r1.stats["matvecs"] >= budget
    assert info["restarts"] == r1.stats["restarts"] and info["nullity"] == r1.nullity
    assert info["d"] == d and info["restart_len"] == R and info["n"] == w.A.n
    assert info["spmm_A"] in (sched, 8)  # 128 becomes 8 where no sliced ELLPACK was built
    assert not os.path.exists(path + ".tmp")
    # a new handle (as a new process would make) continues from the file
    h2 = handle(ns, w, SEED)
    r2 = h2.solve(d, R, 1e-10, precision=prec, resume=1, checkpoint_path=path)
    assert r2.stats["resumed_at"] == info["restarts"]
    for k in COUNTERS:
        assert r2.stats[k] == st_ref[k], k
    assert np.array_equal(h2.basis(), X_ref)
    assert st_ref["resumed_at"] == -1


def test_checkpoints_do_not_change_the_solve(ns, straight, tmp_path):
    """Writing a checkpoint after every restart leaves the iteration untouched, and
    the last file written describes the last restart before the stop."""
    name = "laplacian_fp64_d1"
    _, d, R, prec, sched = CASES[name]
    w, X_ref, st_ref = straight[name]
    path = str(tmp_path / "every.ckpt")
    h = handle(ns, w, SEED)
    r = h.solve(d, R, 1e-10, precision=prec, spmm_schedule=sched, checkpoint_every=1, checkpoint_path=path)
    assert np.array_equal(h.basis(), X_ref)
    for k in COUNTERS:
        assert r.stats[k] == st_ref[k], k
    info = ns.read_checkpoint(path)
    assert info["restarts"] == st_ref["restarts"] - 1  # the final restart stops; it is not saved


def test_resume_in_a_new_process(ns, straight, tmp_path):
    """The interrupted solve runs in a child process that exits; this process resumes."""
    name = "copies_fp64_d2"
    _, d, R, prec, sched = CASES[name]
    w, X_ref, st_ref = straight[name]
    path = str(tmp_path / "child.ckpt")
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from workloads import rectangular_copies\n"
        "from paper_2407_04634_gb300 import nullspace as ns\n"
        "w = rectangular_copies(33, 4500, 3000, 6); A = w.A\n"
        "h = ns.Handle(A.rowptr, A.colind, A.vals, A.m, A.n, %d, w.mode)\n"
        "r = h.solve(%d, %d, 1e-10, check=False, precision=%r, spmm_schedule=%d, max_matvec=%d,"
        " checkpoint_every=2, checkpoint_path=%r)\n"
        "sys.exit(0 if r.status == ns.NS_ERR_NOT_CONVERGED else 3)\n"
    ) % (ROOT, SEED, d, R, prec, sched, st_ref["matvecs"] // 3, path)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    h = handle(ns, w, SEED)
    r = h.solve(d, R, 1e-10, precision=prec, resume=1, checkpoint_path=path)
    assert r.stats["resumed_at"] == ns.read_checkpoint(path)["restarts"]
    assert r.stats["matvecs"] == st_ref["matvecs"]
    assert np.array_equal(h.basis(), X_ref)


def test_resume_rejects_other_problems_and_bad_files(ns, straight, tmp_path):
    name = "laplacian_fp64_d1"
    _, d, R, prec, sched = CASES[name]
    w, _, st_ref = straight[name]
    path = str(tmp_path / "r.ckpt")
    h = handle(ns, w, SEED)
    h.solve(d, R, 1e-10, check=False, precision=prec, spmm_schedule=sched, max_matvec=st_ref["matvecs"] // 2,
            checkpoint_every=1, checkpoint_path=path)
    # other d, restart length, tolerance, precision, perturbation, seed, matrix
    for kw in (dict(d=2), dict(R=R + 4), dict(tol=1e-9), dict(precision="mixed"), dict(eps=2e-3)):
        dd, RR, tt = kw.pop("d", d), kw.pop("R", R), kw.pop("tol", 1e-10)
        opts = dict(precision=prec)
        opts.update(kw)
        r = h.solve(dd, RR, tt, check=False, resume=1, checkpoint_path=path, **opts)
        assert r.status == ns.NS_ERR_INVALID_ARG, (dd, RR, tt, opts)
    h_seed = handle(ns, w, SEED + 1)
    assert h_seed.solve(d, R, 1e-10, check=False, precision=prec, resume=1,
                        checkpoint_path=path).status == ns.NS_ERR_INVALID_ARG
    w2 = laplacian_cycle_components(32, 20000, 12, 8, "powerlaw", 50)
    assert handle(ns, w2, SEED).solve(d, R, 1e-10, check=False, precision=prec, resume=1,
                                      checkpoint_path=path).status == ns.NS_ERR_INVALID_ARG
    # missing, truncated and corrupt files
    assert h.solve(d, R, 1e-10, check=False, resume=1,
                   checkpoint_path=str(tmp_path / "none.ckpt")).status == ns.NS_ERR_IO
    raw = open(path, "rb").read()
    cut = tmp_path / "cut.ckpt"
    cut.write_bytes(raw[: len(raw) // 2])
    assert h.solve(d, R, 1e-10, check=False, resume=1, checkpoint_path=str(cut)).status == ns.NS_ERR_IO
    flip = bytearray(raw)
    flip[len(raw) // 2] ^= 0x10
    bad = tmp_path / "flip.ckpt"
    bad.write_bytes(bytes(flip))
    assert h.solve(d, R, 1e-10, check=False, resume=1, checkpoint_path=str(bad)).status == ns.NS_ERR_IO
    # option checks
    assert h.solve(d, R, 1e-10, check=False, resume=1).status == ns.NS_ERR_INVALID_ARG
    assert h.solve(d, R, 1e-10, check=False, checkpoint_every=1).status == ns.NS_ERR_INVALID_ARG
    assert h.solve(d, R, 1e-10, check=False, spmm_schedule=3).status == ns.NS_ERR_INVALID_ARG
    # the handle still solves after the rejections
    r = h.solve(d, R, 1e-10, precision=prec, spmm_schedule=sched)
    assert r.nullity == w.nullity


@pytest.mark.parametrize("R,d_expect", [(128, 8), (120, 4), (64, 4), (60, 2), (150, 2), (40, 2), (20, 1)])
def test_block_size_rule(ns, R, d_expect):
    """d = 0 takes dim K / 16 (Sec. 5.3.1), rounded down to a supported d dividing dim K."""
    w = laplacian_cycle_components(34, 6000, 5, 8, "powerlaw", 50)
    h = handle(ns, w, 7)
    r = h.solve(0, R, 1e-10)
    assert r.stats["d"] == d_expect
    assert r.nullity == 5


def test_block_size_sweep_finds_the_same_null_space(ns):
    """The sweep of Table tabCH (block size at a fixed dim K): every d finds the planted
    null space, as the oracle does; the basis agrees with the known one to the FP64 bar.
    d = 8 at dim K = 64 converges nothing in its first cycles (the slow start the
    termination test must wait out)."""
    w = rectangular_copies(35, 6000, 4000, 10)
    U = known_basis(w)
    for d in (1, 2, 4, 8):
        ref = lanczos_nullspace(w.A.to_scipy(), "normal", d, 64, tol=1e-10, seed=11)
        h = handle(ns, w, 11)
        r = h.solve(d, 64, 1e-10)
        assert r.nullity == ref.N == 10, d
        assert principal_sine(h.basis(), U) <= 1e-6, d
