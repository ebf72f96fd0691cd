"""ns_project_noalloc, the projection entry point that allocates no device memory.

It exists for callers that cannot allocate while they run: code recorded into a
CUDA graph (stream capture refuses cudaMalloc), an allocator's own callback, or a
host that only hands over buffers it allocated up front.  Its output must match
the allocating ns_project on the same inputs, within the projection tolerance of
the other parity tests, on calls in a row of different sizes (so stale scratch
contents from one call would show up in the next), the largest size it accepts
included, and from inside a stream capture.  This file is collected last on
purpose; each test works both alone in a fresh process and after the others.
"""

import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ns(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2407_04634_gb300 import nullspace
    return nullspace


def _blocked_orthonormal(n, K, seed):
    """n x K orthonormal columns with disjoint supports (cheap at large K)."""
    rng = np.random.default_rng(seed)
    V = np.zeros((n, K))
    rows = rng.permutation(n)
    for k, idx in enumerate(np.array_split(rows, K)):
        v = rng.standard_normal(idx.size)
        V[idx, k] = v / np.linalg.norm(v)
    return V


def _call(lib, V_d, W_d, C_d, n, K, w, stream):
    return lib.ns_project_noalloc(n, K, w, ctypes.c_void_p(V_d.data_ptr()), ctypes.c_void_p(W_d.data_ptr()),
                                  ctypes.c_void_p(C_d.data_ptr()), stream)


def _check(ns, V, W, Wd, Cd):
    W_ref, C_ref = ns.project(V, W, "fp64")
    Wo, Co = Wd.cpu().numpy(), Cd.cpu().numpy()
    assert np.abs(Wo - W_ref).max() <= 1e-12
    assert np.abs(Co - C_ref).max() <= 1e-11
    assert np.abs(V.T @ Wo).max() <= 1e-13 * np.sqrt(V.shape[0])


def test_project_noalloc_matches_project(lib, ns):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the last case is at the entry's limits: K*w = 24000 (192,000 bytes of coefficients,
    # above the 48 KiB default shared-memory limit of a kernel)
    for n, K, w, seed in [(70001, 37, 4, 1), (50000, 12, 8, 2), (40000, 3000, 8, 3)]:
        rng = np.random.default_rng(seed)
        V = np.linalg.qr(rng.standard_normal((n, K)))[0] if K < 100 else _blocked_orthonormal(n, K, seed)
        W = rng.standard_normal((n, w)) + 3.0 * V[:, :w]
        Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()  # column-major n x K
        Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()  # row-major n x w
        Cd = torch.zeros((K, w), dtype=torch.float64, device="cuda")
        st = _call(lib, Vd, Wd, Cd, n, K, w, stream)
        torch.cuda.synchronize()
        assert st == ns.NS_OK
        _check(ns, V, W, Wd, Cd)


def test_project_noalloc_inside_a_graph_capture(lib, ns):
    """One call outside any capture (the set-up), then a call captured into a CUDA graph
    with global capture mode, where any cudaMalloc would break the capture; two replays
    on fresh inputs match ns_project."""
    import torch
    n, K, w = 60001, 40, 2
    rng = np.random.default_rng(11)
    V = np.linalg.qr(rng.standard_normal((n, K)))[0]
    Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()
    Wd = torch.zeros((n, w), dtype=torch.float64, device="cuda")
    Cd = torch.zeros((K, w), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        W0 = rng.standard_normal((n, w))
        Wd.copy_(torch.from_numpy(W0))
        assert _call(lib, Vd, Wd, Cd, n, K, w, ctypes.c_void_p(s.cuda_stream)) == ns.NS_OK
    torch.cuda.synchronize()
    _check(ns, V, W0, Wd, Cd)
    g = torch.cuda.CUDAGraph()
    status = []
    with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
        status.append(_call(lib, Vd, Wd, Cd, n, K, w, ctypes.c_void_p(s.cuda_stream)))
    assert status == [ns.NS_OK]
    for seed in (12, 13):
        W1 = np.random.default_rng(seed).standard_normal((n, w)) + 2.0 * V[:, :w]
        Wd.copy_(torch.from_numpy(W1))
        Cd.zero_()
        g.replay()
        torch.cuda.synchronize()
        _check(ns, V, W1, Wd, Cd)


FIRST_CALL_IN_CAPTURE = r"""
import ctypes, sys
sys.path.insert(0, {root!r})
import torch
from paper_2407_04634_gb300 import nullspace as ns
lib = ns.load()
n, K, w = 1000, 3, 1
V = torch.zeros((K, n), dtype=torch.float64, device="cuda")
W = torch.zeros((n, w), dtype=torch.float64, device="cuda")
C = torch.zeros((K, w), dtype=torch.float64, device="cuda")
s = torch.cuda.Stream()
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
    st = lib.ns_project_noalloc(n, K, w, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(s.cuda_stream))
print("status", st)
st2 = lib.ns_project_noalloc(n, K, w, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                             ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(s.cuda_stream))
torch.cuda.synchronize()
print("after", st2)
"""


def test_project_noalloc_first_call_inside_capture_is_refused(ns):
    """In a fresh process, a first call made while the stream is being captured returns
    NS_ERR_STATE and enqueues nothing (the capture ends cleanly); the next call outside
    the capture succeeds."""
    out = subprocess.run([sys.executable, "-c", FIRST_CALL_IN_CAPTURE.format(root=ROOT)], capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = out.stdout.split()
    assert lines[lines.index("status") + 1] == str(ns.NS_ERR_STATE)
    assert lines[lines.index("after") + 1] == str(ns.NS_OK)


def test_project_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_2407_04634_gb300 import nullspace as ns
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size checks come first
    assert lib.ns_project_noalloc(2_000_000, 4000, 8, dummy, dummy, dummy, None) == ns.NS_ERR_INVALID_ARG
    assert lib.ns_project_noalloc(40000, 3100, 8, dummy, dummy, dummy, None) == ns.NS_ERR_INVALID_ARG
    assert lib.ns_project_noalloc(1000, 10, 3, dummy, dummy, dummy, None) == ns.NS_ERR_INVALID_ARG
