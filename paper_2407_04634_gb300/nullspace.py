"""ctypes binding of libnullspace (C ABI declared in include/nullspace.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch, when used, only supplies device memory (its caching allocator) and the
current CUDA stream.  There is no CPU fallback: loading fails loudly when the
library cannot be built or loaded.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

NS_OK, NS_ERR_INVALID_ARG, NS_ERR_OOM, NS_ERR_CUDA, NS_ERR_NOT_CONVERGED, NS_ERR_TIMEOUT, NS_ERR_STATE, \
    NS_ERR_REFINE, NS_ERR_NUMERICAL, NS_ERR_IO = range(10)
STATUS = {0: "NS_OK", 1: "NS_ERR_INVALID_ARG", 2: "NS_ERR_OOM", 3: "NS_ERR_CUDA", 4: "NS_ERR_NOT_CONVERGED",
          5: "NS_ERR_TIMEOUT", 6: "NS_ERR_STATE", 7: "NS_ERR_REFINE", 8: "NS_ERR_NUMERICAL", 9: "NS_ERR_IO"}
MODE = {"normal": 0, "spd": 1}
PRECISION = {"fp64": 0, "mixed": 1, "fp64_pairs": 2}
REORTH = {"partial": 0, "full": 1}
GEMM = {"default": 0, "cuda_cores": 1, "tc2": 2, "tc3": 3, "tc_exact": 4}

_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class NsEnv(C.Structure):
    _fields_ = [("alloc", _ALLOC), ("free", _FREE), ("ctx", C.c_void_p), ("stream", C.c_void_p)]


class NsOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("precision", C.c_int), ("reorth", C.c_int), ("max_matvec", C.c_int64),
                ("stop_factor", C.c_double), ("lock_tol_mixed", C.c_double), ("refine", C.c_int),
                ("refine_tol", C.c_double), ("refine_maxit", C.c_int), ("refine_chunk", C.c_int),
                ("use_graphs", C.c_int), ("profile", C.c_int), ("batch_block", C.c_int), ("gemm", C.c_int),
                ("fp64_products", C.c_int), ("spmm_schedule", C.c_int), ("checkpoint_every", C.c_int),
                ("resume", C.c_int), ("checkpoint_path", C.c_char_p), ("precond", C.c_int),
                ("precond_shift", C.c_double)]


class NsStats(C.Structure):
    _fields_ = [("nullity", C.c_int64), ("matvecs", C.c_int64), ("restarts", C.c_int64), ("reorth_X", C.c_int64),
                ("reorth_Z", C.c_int64), ("breakdowns", C.c_int64), ("lock_events", C.c_int64),
                ("ghosts", C.c_int64), ("refine_iters_max", C.c_int64), ("kernel_launches", C.c_int64),
                ("normB", C.c_double), ("normA", C.c_double), ("u_d", C.c_double), ("refine_resid_max", C.c_double), ("orth_before", C.c_double), ("orth_after", C.c_double),
                ("t_lanczos_ms", C.c_double), ("t_refine_ms", C.c_double), ("t_total_ms", C.c_double),
                ("d", C.c_int64), ("resumed_at", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NsCheckpointInfo(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("version", "m", "n", "nnz", "mode", "precision", "d", "restart_len",
                                         "reorth", "gemm", "fp64_products", "spmm_A", "spmm_At")] + \
               [("seed", C.c_uint64)] + [(f, C.c_double) for f in ("eps", "tol_eff", "normA1", "normAinf")] + \
               [(f, C.c_int64) for f in ("matvecs", "restarts", "nullity", "k0")] + [("precond", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NsBatchStats(C.Structure):
    _fields_ = [("count", C.c_int64), ("total_nullity", C.c_int64), ("failed", C.c_int64),
                ("matvecs_total", C.c_int64), ("matvecs_max", C.c_int64), ("kernel_launches", C.c_int64),
                ("lanes", C.c_int), ("grid", C.c_int), ("blocks_per_sm", C.c_int), ("block", C.c_int),
                ("graph", C.c_int),
                ("t_solve_ms", C.c_double), ("t_tune_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# exported symbols and their prototypes (kept in sync with include/nullspace.h)
class NsKernelProf(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("sampled", C.c_int64),
                ("ms_per_launch", C.c_double), ("bytes_per_launch", C.c_double), ("flops_per_launch", C.c_double),
                ("ms_total_est", C.c_double)]


_P = C.c_void_p
SIGNATURES = {
    "ns_default_opts": (None, [C.POINTER(NsOpts)]),
    "ns_create": (C.c_int, [C.POINTER(_P), C.c_int64, C.c_int64, _P, _P, _P, C.c_int, C.c_int, C.c_uint64,
                            C.c_int, C.POINTER(NsEnv)]),
    "ns_solve": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.POINTER(NsOpts)]),
    "ns_read_checkpoint": (C.c_int, [C.c_char_p, C.POINTER(NsCheckpointInfo)]),
    "ns_nullity": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "ns_basis": (C.c_int, [_P, _P, C.c_int64, C.c_int]),
    "ns_stats": (C.c_int, [_P, C.POINTER(NsStats)]),
    "ns_profile": (C.c_int, [_P, C.POINTER(NsKernelProf), C.c_int, C.POINTER(C.c_int)]),
    "ns_last_error": (C.c_char_p, [_P]),
    "ns_destroy": (None, [_P]),
    "ns_get_transpose": (C.c_int, [_P, _P, _P, _P]),
    "ns_get_perturbation": (C.c_int, [_P, _P]),
    "ns_start_block": (C.c_int, [_P, C.c_int, _P]),
    "ns_apply_B": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.c_int, C.c_int]),
    "ns_trace_omega": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(NsOpts), _P]),
    "ns_syev": (C.c_int, [C.c_int, _P, _P, _P]),
    "ns_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "ns_precond_build": (C.c_int, [_P, C.c_double, _P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "ns_precond_factor": (C.c_int, [_P, _P, _P, _P]),
    "ns_inner_precond": (C.c_int, [_P, _P]),
    "ns_apply_precond": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.c_int]),
    "ns_restart_product": (C.c_int, [C.c_int64, C.c_int, C.c_int, _P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                                     _P]),
    "ns_project": (C.c_int, [C.c_int64, C.c_int, C.c_int, _P, _P, _P, C.c_int]),
    "ns_project_noalloc": (C.c_int, [C.c_int64, C.c_int, C.c_int, _P, _P, _P, _P]),
    "ns_batch_create": (C.c_int, [C.POINTER(_P), C.c_int64, _P, _P, _P, _P, C.c_int, C.c_uint64,
                                  C.POINTER(NsEnv)]),
    "ns_batch_solve": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.POINTER(NsOpts)]),
    "ns_batch_results": (C.c_int, [_P, _P, _P, _P]),
    "ns_batch_basis": (C.c_int, [_P, C.c_int64, _P, C.c_int64, C.c_int]),
    "ns_batch_basis_packed": (C.c_int, [_P, _P, C.c_int]),
    "ns_batch_stats": (C.c_int, [_P, C.POINTER(NsBatchStats)]),
    "ns_batch_last_error": (C.c_char_p, [_P]),
    "ns_batch_destroy": (None, [_P]),
}

_LIB = None


def load(path: str | None = None):
    """Build (if needed) and load libnullspace.so; declare every prototype."""
    global _LIB
    if _LIB is not None:
        return _LIB
    lib = C.CDLL(path or _build.build())
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


class NullspaceError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def default_opts(**kw) -> NsOpts:
    lib = load()
    o = NsOpts()
    lib.ns_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "reorth" and isinstance(v, str):
            v = REORTH[v]
        if k == "gemm" and isinstance(v, str):
            v = GEMM[v]
        if k == "checkpoint_path" and v is not None:
            v = os.fsencode(v)
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def read_checkpoint(path) -> dict:
    """The record of a checkpoint file written by a solve (checked: magic, length, checksum)."""
    info = NsCheckpointInfo()
    st = load().ns_read_checkpoint(os.fsencode(path), C.byref(info))
    if st != NS_OK:
        raise NullspaceError(st, f"ns_read_checkpoint({path!r})")
    return info.as_dict()


def torch_env():
    """ns_env backed by PyTorch's caching allocator and current stream."""
    import torch

    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream(dev)

    @_ALLOC
    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
        except Exception:  # the library maps NULL to NS_ERR_OOM
            return None

    @_FREE
    def _free(ptr, nbytes, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    env = NsEnv(_alloc, _free, None, C.c_void_p(stream.cuda_stream))
    env._keep = (_alloc, _free, stream)
    return env


@dataclass
class SolveResult:
    status: int
    nullity: int
    stats: dict


class Handle:
    """One matrix on the device (ns_create); solve / basis / stats / destroy."""

    def __init__(self, rowptr, colind, vals, m: int, n: int, seed: int, mode: str = "normal",
                 env: str | None = "torch"):
        self.lib = load()
        self.m, self.n = int(m), int(n)
        self._env = torch_env() if env == "torch" else None
        on_dev = 0
        if hasattr(rowptr, "data_ptr"):  # torch tensors on the device
            import torch
            on_dev = 1
            fp32 = int(vals.dtype == torch.float32)
            ptrs = [C.c_void_p(t.data_ptr()) for t in (rowptr, colind, vals)]
        else:
            fp32 = int(np.asarray(vals).dtype == np.float32)  # FP32 values go in as they are
            self._keep = (np.ascontiguousarray(rowptr, dtype=np.int64), np.ascontiguousarray(colind, dtype=np.int32),
                          np.ascontiguousarray(vals, dtype=np.float32 if fp32 else np.float64))
            ptrs = [_ptr(a) for a in self._keep]
        h = C.c_void_p()
        st = self.lib.ns_create(C.byref(h), self.m, self.n, *ptrs, fp32, on_dev, C.c_uint64(seed), MODE[mode],
                                C.byref(self._env) if self._env is not None else None)
        if st != NS_OK:
            raise NullspaceError(st, "ns_create failed")
        self.h = h
        self.mode = mode

    def _check(self, st, what):
        if st not in (NS_OK,):
            raise NullspaceError(st, f"{what}: {self.lib.ns_last_error(self.h).decode()}")

    def solve(self, d: int, restart_len: int, tol: float, check: bool = True, **opts) -> SolveResult:
        o = default_opts(**opts)
        st = self.lib.ns_solve(self.h, int(d), int(restart_len), float(tol), C.byref(o))
        if check and st not in (NS_OK,):
            self._check(st, "ns_solve")
        N = C.c_int64()
        self.lib.ns_nullity(self.h, C.byref(N))
        return SolveResult(st, int(N.value), self.stats() if st in (NS_OK, NS_ERR_NOT_CONVERGED, NS_ERR_REFINE) else {})

    def nullity(self) -> int:
        N = C.c_int64()
        self._check(self.lib.ns_nullity(self.h, C.byref(N)), "ns_nullity")
        return int(N.value)

    def basis(self, out=None) -> np.ndarray:
        """n x N FP64 basis; out may be a CUDA torch tensor of shape (N, n) (column-major basis)."""
        N = self.nullity()
        if out is not None and hasattr(out, "data_ptr"):
            self._check(self.lib.ns_basis(self.h, C.c_void_p(out.data_ptr()), self.n, 1), "ns_basis")
            return out
        X = np.zeros((N, self.n), dtype=np.float64)  # column-major n x N == row-major N x n
        self._check(self.lib.ns_basis(self.h, _ptr(X), self.n, 0), "ns_basis")
        return X.T

    def stats(self) -> dict:
        s = NsStats()
        self._check(self.lib.ns_stats(self.h, C.byref(s)), "ns_stats")
        return s.as_dict()

    def profile(self) -> list[dict]:
        """Per-kernel-class CUDA-event measurements of the last solve (opts profile > 0)."""
        arr = (NsKernelProf * 8)()
        cnt = C.c_int()
        self._check(self.lib.ns_profile(self.h, arr, 8, C.byref(cnt)), "ns_profile")
        out = []
        for r in arr[:cnt.value]:
            out.append(dict(name=r.name.decode(), launches=r.launches, sampled=r.sampled,
                            ms_per_launch=r.ms_per_launch, bytes_per_launch=r.bytes_per_launch,
                            flops_per_launch=r.flops_per_launch, ms_total_est=r.ms_total_est))
        return out

    def transpose(self, nnz: int):
        rp = np.zeros(self.n + 1, dtype=np.int64)
        ci = np.zeros(max(nnz, 1), dtype=np.int32)
        va = np.zeros(max(nnz, 1), dtype=np.float64)
        self._check(self.lib.ns_get_transpose(self.h, _ptr(rp), _ptr(ci), _ptr(va)), "ns_get_transpose")
        return rp, ci[:nnz], va[:nnz]

    def perturbation(self) -> np.ndarray:
        D = np.zeros(self.n)
        self._check(self.lib.ns_get_perturbation(self.h, _ptr(D)), "ns_get_perturbation")
        return D

    def start_block(self, d: int) -> np.ndarray:
        Om = np.zeros((self.n, d))
        self._check(self.lib.ns_start_block(self.h, int(d), _ptr(Om)), "ns_start_block")
        return Om

    def apply_B(self, X: np.ndarray, eps: float, precision: str = "fp64", schedule: int = -1) -> np.ndarray:
        """Y = B X; schedule -1 = library default, 64 = TMA-staged, k = k threads per row."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        d = X.shape[1]
        Y = np.zeros_like(X)
        self._check(self.lib.ns_apply_B(self.h, d, _ptr(X), _ptr(Y), float(eps), PRECISION[precision], 0,
                                        int(schedule)), "ns_apply_B")
        return Y

    def precond_build(self, shift: float = 0.1) -> dict:
        """Outer preconditioner (colouring, renumbering, IC(0) factor); returns
        color (original numbering), perm (perm[new] = old), ncolors and nnz_L."""
        color = np.zeros(self.n, dtype=np.int32)
        perm = np.zeros(self.n, dtype=np.int64)
        nnzL = C.c_int64()
        nc = C.c_int32()
        self._check(self.lib.ns_precond_build(self.h, float(shift), _ptr(color), _ptr(perm), C.byref(nnzL),
                                              C.byref(nc)), "ns_precond_build")
        return dict(color=color, perm=perm, nnz_L=int(nnzL.value), ncolors=int(nc.value))

    def precond_factor(self, nnz_L: int):
        """The factor L (CSR arrays rowptr, colind, vals) of the renumbered matrix."""
        rp = np.zeros(self.n + 1, dtype=np.int64)
        ci = np.zeros(max(nnz_L, 1), dtype=np.int32)
        va = np.zeros(max(nnz_L, 1), dtype=np.float64)
        self._check(self.lib.ns_precond_factor(self.h, _ptr(rp), _ptr(ci), _ptr(va)), "ns_precond_factor")
        return rp, ci[:nnz_L], va[:nnz_L]

    def inner_precond(self) -> np.ndarray:
        """Inner preconditioner (normal form): the row scaling s_i = 1/||a_i|| of P_L^-1/2."""
        s = np.zeros(max(self.m, 1), dtype=np.float64)
        self._check(self.lib.ns_inner_precond(self.h, _ptr(s)), "ns_inner_precond")
        return s[:self.m]

    def apply_precond(self, X: np.ndarray, eps: float, precision: str = "fp64") -> np.ndarray:
        """Y = L^-1 A~ L^-T X + eps D X in the renumbered space (SPD handle), or
        Y = A^T P_L^-1 A X + eps D X (normal handle)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.zeros_like(X)
        self._check(self.lib.ns_apply_precond(self.h, X.shape[1], _ptr(X), _ptr(Y), float(eps),
                                              PRECISION[precision], 0), "ns_apply_precond")
        return Y

    def trace_omega(self, d: int, restart_len: int, **opts) -> np.ndarray:
        """W columns of the first cycle ((nb+1) x (nb+1), entry [b, c] = w_{b,c} before any reset)."""
        nbp = restart_len // d + 1
        W = np.zeros((nbp, nbp), order="F")
        o = default_opts(**opts)
        self._check(self.lib.ns_trace_omega(self.h, int(d), int(restart_len), C.byref(o),
                                            C.c_void_p(W.ctypes.data)), "ns_trace_omega")
        return W

    def close(self):
        if getattr(self, "h", None):
            self.lib.ns_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def restart_product(Z: np.ndarray, VZ: np.ndarray, sel, nl: int, d: int, precision: str = "fp64",
                    gemm: str = "default") -> np.ndarray:
    """Z V_Z(:, sel) with the library's restart-product kernel (n x nsel FP64)."""
    lib = load()
    n, R = Z.shape
    Zc = np.asfortranarray(Z, dtype=np.float64)
    Vc = np.asfortranarray(VZ, dtype=np.float64)
    sel = np.ascontiguousarray(sel, dtype=np.int32)
    out = np.zeros((n, sel.size), order="F")
    st = lib.ns_restart_product(n, int(d), R, C.c_void_p(Zc.ctypes.data), C.c_void_p(Vc.ctypes.data), _ptr(sel),
                                sel.size, int(nl), PRECISION[precision], GEMM[gemm], C.c_void_p(out.ctypes.data))
    if st != NS_OK:
        raise NullspaceError(st, "ns_restart_product")
    return out


def fma_peak(precision: str = "fp64") -> float:
    """Measured FMA throughput (TFLOP/s) of the current device's FP64 or FP32 pipe."""
    lib = load()
    v = C.c_double()
    st = lib.ns_fma_peak(PRECISION[precision], C.byref(v))
    if st != NS_OK:
        raise NullspaceError(st, "ns_fma_peak")
    return float(v.value)


def syev(T: np.ndarray):
    """Device eigensolver of the projected matrix (ascending eigenvalues, eigenvectors)."""
    lib = load()
    k = T.shape[0]
    Tc = np.asfortranarray(T, dtype=np.float64)
    th = np.zeros(k)
    V = np.zeros((k, k), order="F")
    st = lib.ns_syev(k, C.c_void_p(Tc.ctypes.data), _ptr(th), C.c_void_p(V.ctypes.data))
    if st != NS_OK:
        raise NullspaceError(st, "ns_syev")
    return th, V


def project(V: np.ndarray, W: np.ndarray, precision: str = "fp64"):
    """CGS2 of W (n x w) against V (n x K) on the device; returns (W', C)."""
    lib = load()
    n, K = V.shape
    w = W.shape[1]
    Vc = np.asfortranarray(V, dtype=np.float64)
    Wc = np.ascontiguousarray(W, dtype=np.float64).copy()
    Cc = np.zeros((K, w))
    st = lib.ns_project(n, K, w, C.c_void_p(Vc.ctypes.data), _ptr(Wc), _ptr(Cc), PRECISION[precision])
    if st != NS_OK:
        raise NullspaceError(st, "ns_project")
    return Wc, Cc


BATCH_ISTATS = ("matvecs", "restarts", "reorths", "refine_iters", "cycles", "cyc_steps", "cyc_reorth", "cyc_eig",
                "cyc_lock", "cyc_restart", "cyc_refine", "sweeps32", "sweeps64")
BATCH_STATUS = {0: "ok", 4: "max_matvec reached", 7: "refinement missed its tolerance", 8: "more than 32 null vectors"}


class Batch:
    """Many independent symmetric PSD matrices solved in one persistent launch (ns_batch_*).

    mats: sequence of (rowptr, colind, vals) host arrays (square CSR, local column
    indices), or objects with .rowptr/.colind/.vals.  Instance i uses Philox key
    seed + i.
    """

    def __init__(self, mats, seed: int, env: str | None = "torch"):
        self.lib = load()
        rps, cis, vas, ns_ = [], [], [], []
        for M in mats:
            rp, ci, va = (M.rowptr, M.colind, M.vals) if hasattr(M, "rowptr") else M
            rps.append(np.asarray(rp, dtype=np.int64))
            cis.append(np.asarray(ci, dtype=np.int32))
            vas.append(np.asarray(va))
            ns_.append(len(rp) - 1)
        if not all(v.dtype == np.float32 for v in vas):
            vas = [v.astype(np.float64) for v in vas]
        self._create(np.asarray(ns_, dtype=np.int64), np.concatenate(rps), np.concatenate(cis),
                     np.concatenate(vas), seed, env)

    @classmethod
    def from_arrays(cls, n, rowptr, colind, vals, seed: int, env: str | None = "torch") -> "Batch":
        """Already concatenated host arrays (the layout ns_batch_create takes)."""
        b = cls.__new__(cls)
        b.lib = load()
        b._create(np.asarray(n, dtype=np.int64), rowptr, colind, vals, seed, env)
        return b

    def _create(self, n, rowptr, colind, vals, seed, env):
        self.count = len(n)
        self.n = n
        fp32 = int(np.asarray(vals).dtype == np.float32)  # FP32 values go in as they are
        self._keep = (np.ascontiguousarray(n, dtype=np.int64), np.ascontiguousarray(rowptr, dtype=np.int64),
                      np.ascontiguousarray(colind, dtype=np.int32),
                      np.ascontiguousarray(vals, dtype=np.float32 if fp32 else np.float64))
        self._env = torch_env() if env == "torch" else None
        h = C.c_void_p()
        st = self.lib.ns_batch_create(C.byref(h), self.count, *[_ptr(a) for a in self._keep], fp32,
                                      C.c_uint64(seed), C.byref(self._env) if self._env is not None else None)
        if st != NS_OK:
            raise NullspaceError(st, "ns_batch_create failed")
        self.h = h

    def _check(self, st, what):
        if st != NS_OK:
            raise NullspaceError(st, f"{what}: {self.lib.ns_batch_last_error(self.h).decode()}")

    def solve(self, restart_len: int, tol: float, check: bool = True, **opts) -> int:
        o = default_opts(**opts)
        st = self.lib.ns_batch_solve(self.h, 1, int(restart_len), float(tol), C.byref(o))
        if check:
            self._check(st, "ns_batch_solve")
        return st

    def results(self):
        """(nullity[count], status[count], istats[count, 11]) of the last solve; istats columns
        are BATCH_ISTATS."""
        N = np.zeros(self.count, dtype=np.int32)
        S = np.zeros(self.count, dtype=np.int32)
        I = np.zeros((self.count, len(BATCH_ISTATS)), dtype=np.int64)
        self._check(self.lib.ns_batch_results(self.h, _ptr(N), _ptr(S), _ptr(I)), "ns_batch_results")
        return N, S, I

    def basis(self, i: int) -> np.ndarray:
        N, _, _ = self.results()
        n = int(self.n[i])
        X = np.zeros((int(N[i]), n), dtype=np.float64)
        self._check(self.lib.ns_batch_basis(self.h, int(i), _ptr(X), n, 0), "ns_batch_basis")
        return X.T

    def basis_packed(self, out=None) -> np.ndarray:
        """Every instance's basis in one transfer: instance i's n_i x N_i block, column-major,
        at offset sum_{j<i} n_j N_j.  out may be a host array or a CUDA torch tensor."""
        N, _, _ = self.results()
        tot = int((self.n * N).sum())
        if out is not None and hasattr(out, "data_ptr"):
            self._check(self.lib.ns_batch_basis_packed(self.h, C.c_void_p(out.data_ptr()), 1), "ns_batch_basis_packed")
            return out
        if out is None:
            out = np.zeros(tot, dtype=np.float64)
        self._check(self.lib.ns_batch_basis_packed(self.h, _ptr(out), 0), "ns_batch_basis_packed")
        return out

    def stats(self) -> dict:
        s = NsBatchStats()
        self._check(self.lib.ns_batch_stats(self.h, C.byref(s)), "ns_batch_stats")
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.ns_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
