"""ns_project_noalloc, the projection entry point that allocates no device memory.

It is meant for callers that cannot allocate while they run (inside a CUDA graph
capture, inside an allocator callback, hosts that only hand over pre-allocated
buffers).  Its output must match the allocating ns_project on the same inputs,
within the projection tolerance used by the other parity tests, on two calls in
a row of different sizes (so stale scratch contents from the first call would
show up in the second).  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_project_noalloc_matches_project(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2407_04634_gb300 import nullspace as ns
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, K, w, seed in [(70001, 37, 4, 1), (50000, 12, 8, 2)]:
        rng = np.random.default_rng(seed)
        V, _ = np.linalg.qr(rng.standard_normal((n, K)))
        W = rng.standard_normal((n, w)) + 3.0 * V[:, :w]
        W_ref, C_ref = ns.project(V, W, "fp64")
        Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()  # column-major n x K
        Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()  # row-major n x w
        Cd = torch.zeros((K, w), dtype=torch.float64, device="cuda")
        st = lib.ns_project_noalloc(n, K, w, ctypes.c_void_p(Vd.data_ptr()), ctypes.c_void_p(Wd.data_ptr()),
                                    ctypes.c_void_p(Cd.data_ptr()), stream)
        torch.cuda.synchronize()
        assert st == ns.NS_OK
        assert np.abs(Wd.cpu().numpy() - W_ref).max() <= 1e-12
        assert np.abs(Cd.cpu().numpy() - C_ref).max() <= 1e-11
        assert np.abs(V.T @ Wd.cpu().numpy()).max() <= 1e-13 * np.sqrt(n)


def test_project_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_2407_04634_gb300 import nullspace as ns
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert lib.ns_project_noalloc(2_000_000, 4000, 8, dummy, dummy, dummy, None) == ns.NS_ERR_INVALID_ARG
    assert lib.ns_project_noalloc(1000, 10, 3, dummy, dummy, dummy, None) == ns.NS_ERR_INVALID_ARG
