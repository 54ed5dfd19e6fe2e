"""Seeded synthetic inputs with controlled singular values.

This module only draws test and benchmark matrices.  It holds none of the
factorization's arithmetic and is shared by the CUDA path's tests, the oracle's
tests and the benchmark.

Recipe (the test matrices of Sec. 4 are only called "random"; this is the
construction used throughout):

    X = U diag(sigma) V^T,  U (m x n) and V (n x n) orthonormal factors of the
    Householder QR of seeded N(0,1) matrices, sigma = logspace(0, -log10 kappa, n),

so kappa(X) = kappa up to rounding.  The row-scaled form rescales row i of X to
norm exp(2 z_i), z_i ~ N(0,1) (row norms lognormal with parameters (0, 2)).
"""
from __future__ import annotations

import math

import numpy as np


def sigma_logspaced(n: int, kappa: float) -> np.ndarray:
    """Singular values 1 ... 1/kappa, log-spaced, n of them."""
    if n == 1:
        return np.ones(1)
    return np.logspace(0.0, -math.log10(kappa), n)


def orthonormal_np(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """Orthonormal m x n factor of a Gaussian matrix (LAPACK Householder QR)."""
    g = rng.standard_normal((m, n))
    q, _ = np.linalg.qr(g)
    return q


def make_matrix_np(m: int, n: int, kappa: float, seed: int, row_scaled: bool = False) -> np.ndarray:
    """CPU (numpy) draw of X = U diag(sigma) V^T; column-major (Fortran) float64."""
    rng = np.random.default_rng(seed)
    u = orthonormal_np(rng, m, n)
    v = orthonormal_np(rng, n, n)
    x = (u * sigma_logspaced(n, kappa)[None, :]) @ v.T
    if row_scaled:
        z = rng.standard_normal(m)
        norms = np.linalg.norm(x, axis=1)
        norms[norms == 0] = 1.0
        x = x * (np.exp(2.0 * z) / norms)[:, None]
    return np.asfortranarray(x)


def _orthonormalize_torch(g):
    """Orthonormal factor of a tall Gaussian g on the device by Cholesky QR
    applied twice (CholQR2); the n x n Cholesky factors and inverses are formed
    on the host with numpy.  A tall Gaussian is well conditioned
    (kappa ~ (1 + sqrt(n/m)) / (1 - sqrt(n/m))), so two passes leave
    ||I - U^T U|| = O(u).  Only device matmuls are used, so the draw also works
    where torch's device linear-algebra library cannot be loaded."""
    import torch

    u = g
    for _ in range(2):
        w = (u.T @ u).cpu().numpy()
        L = np.linalg.cholesky(w)
        rinv = np.linalg.inv(L.T)
        u = u @ torch.as_tensor(rinv, dtype=u.dtype, device=u.device)
    return u


def make_matrix_torch(m: int, n: int, kappa: float, seed: int, device: str = "cuda",
                      row_scaled: bool = False):
    """Device draw of the same construction (torch generator on `device`).

    Used for inputs too large to draw on the host in reasonable time.  U is the
    orthonormal factor of a seeded device Gaussian (CholQR2, see above), V the
    Householder factor of a seeded host Gaussian.  Returns a column-major
    float64 tensor (the transpose of a contiguous n x m tensor).  The device
    stream of random numbers differs from numpy's, so a matrix drawn here is
    compared with the oracle by copying it to the host.
    """
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    g = torch.randn(m, n, generator=gen, dtype=torch.float64, device=device)
    u = _orthonormalize_torch(g)
    del g
    v = orthonormal_np(np.random.default_rng(seed), n, n)
    sig = sigma_logspaced(n, kappa)
    vs = torch.as_tensor(v * sig[None, :], dtype=torch.float64, device=device)
    xt = vs @ u.T  # n x m contiguous == column-major m x n
    del u
    if row_scaled:
        z = torch.randn(m, generator=gen, dtype=torch.float64, device=device)
        norms = torch.sqrt((xt * xt).sum(dim=0))
        norms = torch.where(norms == 0, torch.ones_like(norms), norms)
        xt.mul_((torch.exp(2.0 * z) / norms)[None, :])
    return xt.T  # m x n view, stride (1, m)


def make_upper_triangular_np(n: int, kappa: float, seed: int) -> np.ndarray:
    """Seeded upper-triangular R0 with positive diagonal and kappa(R0) ~ kappa.

    R0 = diag(d) (I + N) with N strictly upper triangular, small Gaussian, and d
    log-spaced; used for the closed-form recovery X = Q0 R0.
    """
    rng = np.random.default_rng(seed)
    d = sigma_logspaced(n, kappa)
    nmat = np.triu(rng.standard_normal((n, n)), 1) * (0.5 / math.sqrt(max(n, 1)))
    return np.asfortranarray(d[:, None] * (np.eye(n) + nmat))


def log_uniform_int(rng: np.random.Generator, lo_exp: float, hi_exp: float) -> int:
    """round(2^U(lo_exp, hi_exp))."""
    return int(round(2.0 ** rng.uniform(lo_exp, hi_exp)))
