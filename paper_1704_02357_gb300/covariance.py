"""Covariance of P(k, mu) wedges over mocks (Sec. 4.1).

Mocks go through the batched path (pspec_run_batch); their multipoles are turned into wedges
by pspec_wedges on the device; the sample covariance and correlation of the wedges, per k bin
and pooled over k bins, are small host-side matrices compared against the Kaiser-model gamma_mn
(pspec_wedge_gamma_kaiser) and judged by their condition number (smallest over largest
singular value, the paper's definition).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from .pspec import wedges


def mock_wedges(P, ells: Sequence[int], mu_edges, stream=None):
    """P: float64 CUDA tensor (n_mocks, n_ells, nk) -> float64 CUDA tensor (n_mocks, n_mu, nk)."""
    import torch
    out = [wedges(P[i], ells, mu_edges, stream=stream) for i in range(P.shape[0])]
    return torch.stack(out)


def pooled_correlation(W) -> np.ndarray:
    """Correlation between wedges, per k bin over the mocks, averaged over the k bins.
    W: array (n_mocks, n_mu, nk)."""
    W = np.asarray(W, dtype=np.float64)
    n = W.shape[0]
    acc, used = None, 0
    for b in range(W.shape[2]):
        X = W[:, :, b]
        if not np.all(np.isfinite(X)):
            continue
        Z = X - X.mean(axis=0)
        sd = Z.std(axis=0, ddof=1)
        if np.any(sd == 0):
            continue
        Z = Z / sd
        C = Z.T @ Z / (n - 1)
        acc = C if acc is None else acc + C
        used += 1
    if not used:
        raise ValueError("no k bin with finite, varying wedges")
    return acc / used


def correlation(C) -> np.ndarray:
    C = np.asarray(C, dtype=np.float64)
    d = np.sqrt(np.diag(C))
    return C / np.outer(d, d)


def condition_number(M) -> float:
    """Smallest over largest singular value."""
    s = np.linalg.svd(np.asarray(M, dtype=np.float64), compute_uv=False)
    return float(s.min() / s.max())
