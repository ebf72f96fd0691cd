"""Device-side checks of a computed null-space basis, independent of the library.

Used by the full-size GPU tests, where the oracle cannot run: the residual
||A X||_F / ||A||_2 is recomputed with PyTorch's sparse product (cuSPARSE) and a
power-iteration estimate of ||A||_2, and the basis is compared with the
workload's closed-form null space by the largest principal-angle sine.
"""

from __future__ import annotations

import numpy as np


def device_csr(A, device="cuda"):
    """scipy CSR -> torch sparse CSR (FP64) on the device."""
    import torch
    A = A.tocsr()
    return torch.sparse_csr_tensor(torch.as_tensor(A.indptr.astype(np.int64), device=device),
                                   torch.as_tensor(A.indices.astype(np.int64), device=device),
                                   torch.as_tensor(A.data.astype(np.float64), device=device),
                                   size=A.shape, dtype=torch.float64)


def norm2_power(Ad, AdT, iters: int = 150, seed: int = 0) -> float:
    """||A||_2 by power iteration on A^T A (a lower bound, so residual ratios are
    over-estimated, never flattered).  AdT is None for a symmetric A."""
    import torch
    g = torch.Generator(device=Ad.device).manual_seed(seed)
    x = torch.randn((Ad.shape[1], 1), dtype=torch.float64, device=Ad.device, generator=g)
    x /= torch.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = Ad @ x
        y = (AdT @ y) if AdT is not None else (Ad @ y)
        lam = float(torch.linalg.norm(y))
        x = y / lam
    return float(np.sqrt(lam))


def residual_ratio(Ad, X, normA: float, chunk: int = 64) -> float:
    """||A X||_F / ||A||_2 for a device basis X (n x N), in column chunks."""
    import torch
    tot = 0.0
    for c0 in range(0, X.shape[1], chunk):
        R = Ad @ X[:, c0:c0 + chunk].contiguous()
        tot += float(torch.sum(R * R))
    return float(np.sqrt(tot)) / normA


def indicator_sine(labels, X) -> float:
    """Largest principal-angle sine between span(X) and the span of the component
    indicators: ||(I - P) X||_2 with P the projection onto piecewise-constant vectors."""
    import torch
    lab = torch.as_tensor(np.asarray(labels), device=X.device, dtype=torch.long)
    k = int(lab.max()) + 1
    sums = torch.zeros((k, X.shape[1]), dtype=X.dtype, device=X.device).index_add_(0, lab, X)
    cnt = torch.bincount(lab, minlength=k).to(X.dtype)
    Rm = X - (sums / cnt[:, None])[lab]
    return float(np.sqrt(max(np.linalg.eigvalsh((Rm.T @ Rm).double().cpu().numpy())[-1], 0.0)))


def copy_pair_sine(pairs, n: int, X) -> float:
    """Largest principal-angle sine between span(X) and span{(e_s + e_c)/sqrt(2)}."""
    import torch
    pr = torch.as_tensor(np.asarray(pairs), device=X.device, dtype=torch.long)
    PX = torch.zeros_like(X)
    avg = 0.5 * (X[pr[:, 0]] + X[pr[:, 1]])
    PX[pr[:, 0]] = avg
    PX[pr[:, 1]] = avg
    Rm = X - PX
    return float(np.sqrt(max(np.linalg.eigvalsh((Rm.T @ Rm).double().cpu().numpy())[-1], 0.0)))


def orthonormality(X) -> tuple[float, float]:
    """(max |X^T X - I|, ||X^T X - I||_F)."""
    import torch
    E = X.T @ X - torch.eye(X.shape[1], dtype=X.dtype, device=X.device)
    return float(torch.max(torch.abs(E))), float(torch.linalg.norm(E))
