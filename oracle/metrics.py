"""Accuracy metrics of an economic QR (test infrastructure only).

loss of orthogonality  ||I - Q^T Q||_2        (Table 1, with the 2-norm of Sec. 1)
relative residual      ||X - Q R||_F / ||X||_F (not defined by the paper; Frobenius)
kappa(A)               sigma_max / sigma_min  (Sec. 1), by LAPACK SVD.
"""
from __future__ import annotations

import numpy as np


def loo(Q: np.ndarray) -> float:
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[1]
    return float(np.linalg.norm(np.eye(n) - Q.T @ Q, 2))


def loo_from_gram(G: np.ndarray) -> float:
    """||I - G||_2 for a precomputed Gram matrix G = Q^T Q."""
    G = np.asarray(G, dtype=np.float64)
    return float(np.linalg.norm(np.eye(G.shape[0]) - G, 2))


def residual(X: np.ndarray, Q: np.ndarray, R: np.ndarray) -> float:
    X = np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm(X - Q @ R) / np.linalg.norm(X))


def kappa(A: np.ndarray) -> float:
    sv = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    return float(sv[0] / sv[-1])
