"""Plain CPU FP64 oracle for reorthogonalized block classical Gram-Schmidt.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with the
CUDA path and must never be used as a fallback for it.

Problem (Sec. 1): the economic QR  X = Q R  of a tall-skinny m x n matrix X with
Q^T Q = I and R upper triangular.  X is split into q = n / s block columns
X = [X_1 ... X_q] of s columns each (Sec. 1, the block partition); bold Q_k
means [Q_1 ... Q_k].  Block indices in comments are 1-based, as in the paper.
Sign convention (the paper is silent): diag(R) > 0, which makes Q and R unique.

Everything is float64 numpy.  Matrix products use numpy's matmul (a library
primitive); the Householder QR, the Cholesky factorization and the triangular
solves are written out.  No blocking, fusion or reordering is applied beyond what
each algorithm states.

Pins (tests/test_oracle_pins.py): agreement with LAPACK QR and with a 60-digit
QR on small inputs, exact recovery of a Hadamard-based closed form, s = n and
s = 1 special cases, recovery of R0 from X = Q0 R0, cross-variant agreement,
the Pythagorean identity, eq. (1) against the direct product, the loss of
orthogonality ordering of Table 1, and LAPACK's R for a ragged last block.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Breakdown", "householder_qr", "tsqr", "chol", "solve_right_upper",
    "solve_left_upper_t", "delayed_projection", "gram", "project_normalize",
    "bcgsi_plus", "bcgsi_plus_p_1s", "bcgsi_plus_p_2s", "bcgs_pipi_plus", "bcgsi_plus_1s", "eager_step",
    "factor",
    "VARIANTS", "EAGER_FAMILY",
]


class Breakdown(Exception):
    """Numerical breakdown of a variant.

    kind: "not_spd"  (a Pythagorean Cholesky met a non-positive pivot),
          "rank_deficient" (an intraorthogonalization produced a zero R diagonal),
          "nonfinite" (a NaN or Inf reached a factor).
    block: 1-based index of the block column being processed.
    """

    def __init__(self, kind: str, block: int):
        super().__init__(f"{kind} at block {block}")
        self.kind = kind
        self.block = block


# ---------------------------------------------------------------------------
# Intraorthogonalization
# ---------------------------------------------------------------------------

def householder_qr(A: np.ndarray, block: int = 1):
    """Economic Householder QR of an m x s block, m >= s, with diag(R) >= 0.

    The "unconditionally stable QR" used as intraorthogonalization (Sec. 1 and
    Sec. 2; TSQR in the paper's experiments, Sec. 4).  For column j the reflector
    H_j = I - tau_j v_j v_j^T maps A[j:, j] to beta_j e_1 with beta_j = -sign(a_jj)
    ||A[j:, j]||; the explicit Q = H_1 ... H_s [I; 0]; finally the signs of R's
    rows and Q's columns are flipped so that diag(R) >= 0.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    m, s = A.shape
    if m < s:
        raise ValueError("householder_qr needs m >= s")
    if not np.all(np.isfinite(A)):
        raise Breakdown("nonfinite", block)
    vs, taus = [], []
    for j in range(s):
        x = A[j:, j]
        alpha = np.linalg.norm(x)
        if alpha == 0.0:
            v = np.zeros(m - j)
            v[0] = 1.0
            vs.append(v)
            taus.append(0.0)
            continue
        x0 = x[0]
        beta = -alpha if x0 >= 0 else alpha
        v = x / (x0 - beta)
        v[0] = 1.0
        tau = (beta - x0) / beta
        # apply H_j to the trailing columns
        if j + 1 < s:
            w = v @ A[j:, j + 1:]
            A[j:, j + 1:] -= tau * np.outer(v, w)
        A[j, j] = beta
        A[j + 1:, j] = 0.0
        vs.append(v)
        taus.append(tau)
    R = np.triu(A[:s, :])
    Q = np.zeros((m, s))
    Q[:s, :s] = np.eye(s)
    for j in range(s - 1, -1, -1):
        v, tau = vs[j], taus[j]
        if tau != 0.0:
            w = v @ Q[j:, :]
            Q[j:, :] -= tau * np.outer(v, w)
    d = np.where(np.diag(R) < 0, -1.0, 1.0)
    R = d[:, None] * R
    Q = Q * d[None, :]
    diag = np.diag(R)
    if not np.all(np.isfinite(R)):
        raise Breakdown("nonfinite", block)
    if np.any(diag == 0.0):
        raise Breakdown("rank_deficient", block)
    return Q, R


def tsqr(A: np.ndarray, block: int = 1):
    """TSQR(A) (Sec. 1, Alg. 1, Alg. 2).

    TSQR is a reduction-tree arrangement of Householder QR whose tree shape the
    paper does not fix; in exact arithmetic it returns the same sign-normalized
    factors as one Householder QR of the whole block, which is what the oracle
    computes.
    """
    return householder_qr(A, block)


# ---------------------------------------------------------------------------
# Small dense kernels
# ---------------------------------------------------------------------------

def chol(A: np.ndarray, block: int = 1) -> np.ndarray:
    """Upper-triangular R with A = R^T R (the chol of Alg. 1 and Alg. 2).

    Right-looking column form: r_jj = sqrt(a_jj - sum_{l<j} r_lj^2),
    r_ji = (a_ji - sum_{l<j} r_lj r_li) / r_jj for i > j.  Only the upper
    triangle of A is read.  A pivot that is not > 0 (or NaN) is a breakdown.
    """
    A = np.asarray(A, dtype=np.float64)
    s = A.shape[0]
    R = np.zeros((s, s))
    for j in range(s):
        d = A[j, j] - np.dot(R[:j, j], R[:j, j])
        if not (d > 0.0) or not np.isfinite(d):
            raise Breakdown("not_spd", block)
        R[j, j] = np.sqrt(d)
        for i in range(j + 1, s):
            R[j, i] = (A[j, i] - np.dot(R[:j, j], R[:j, i])) / R[j, j]
    return R


def solve_right_upper(V: np.ndarray, T: np.ndarray) -> np.ndarray:
    """W = V T^{-1} for upper-triangular T, by substitution over columns:
    w_j = (v_j - sum_{l<j} w_l t_lj) / t_jj."""
    V = np.asarray(V, dtype=np.float64)
    s = T.shape[0]
    W = np.zeros_like(V)
    for j in range(s):
        W[:, j] = (V[:, j] - W[:, :j] @ T[:j, j]) / T[j, j]
    return W


def solve_left_upper_t(T: np.ndarray, M: np.ndarray) -> np.ndarray:
    """W = T^{-T} M for upper-triangular T (T^T is lower), forward substitution
    over rows: w_i = (m_i - sum_{l<i} t_li w_l) / t_ii."""
    M = np.asarray(M, dtype=np.float64)
    s = T.shape[0]
    W = np.zeros_like(M)
    for i in range(s):
        W[i, :] = (M[i, :] - T[:i, i] @ W[:i, :]) / T[i, i]
    return W


def gram(A_blocks, B_blocks) -> np.ndarray:
    """The tall-skinny product [A_1 ...]^T [B_1 ...]: one synchronization point
    (Sec. 3: the only operation with global communication)."""
    A = np.hstack([np.asarray(a, dtype=np.float64) for a in A_blocks])
    B = np.hstack([np.asarray(b, dtype=np.float64) for b in B_blocks])
    return A.T @ B


def project_normalize(V: np.ndarray, Qk: np.ndarray, C: np.ndarray, T: np.ndarray) -> np.ndarray:
    """(V - Q_k C) T^{-1}: the projection plus triangular-solve normalization of
    Alg. 1 (U_{k+1}, Q_{k+1}) and Alg. 2 (U_{k+1}, Q_{k+1})."""
    if Qk.shape[1] == 0:
        return solve_right_upper(V, T)
    return solve_right_upper(np.asarray(V) - Qk @ C, T)


def delayed_projection(Ykk: np.ndarray, Pk: np.ndarray, Yprev: np.ndarray, Zprev: np.ndarray) -> np.ndarray:
    """Eq. (1): Q_k^T X_{k+1} = Y_kk^{-T} (P_k - Y_{1:k-1,k}^T Z_{k-1})."""
    return solve_left_upper_t(Ykk, Pk - Yprev.T @ Zprev)


# ---------------------------------------------------------------------------
# Variants
# ---------------------------------------------------------------------------

def _check(X, s):
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    if s < 1 or n % s != 0 or m < s:
        raise ValueError("need s >= 1, n = q s and m >= s")
    return X, m, n, n // s


def bcgsi_plus(X: np.ndarray, s: int):
    """BCGSI+, the classical reorthogonalized BCGS (Sec. 1; Table 1: 4 syncs per
    block, O(u) loss of orthogonality for O(u) kappa <= 1).

    The paper prints no pseudocode.  Reading: each block is projected twice
    against the previous basis, each projection followed by a TSQR, and R is
    assembled as in Alg. 1:
        [Q_1, R_11] = TSQR(X_1)
        for k = 1..q-1:
            S = Q_k^T X_{k+1};            [U, S_kk] = TSQR(X_{k+1} - Q_k S)
            Y = Q_k^T U;                  [Q_{k+1}, Y_kk] = TSQR(U - Q_k Y)
            R_{1:k,k+1} = S + Y S_kk;     R_{k+1,k+1} = Y_kk S_kk
    """
    X, m, n, q = _check(X, s)
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    blk = lambda k: slice((k - 1) * s, k * s)   # block column k (1-based)
    upto = lambda k: slice(0, k * s)            # block columns 1..k
    Q[:, blk(1)], R[blk(1), blk(1)] = tsqr(X[:, blk(1)], 1)
    for k in range(1, q):
        Qk = Q[:, upto(k)]
        Xk1 = X[:, blk(k + 1)]
        S = gram([Qk], [Xk1])
        U, Skk = tsqr(Xk1 - Qk @ S, k + 1)
        Y = gram([Qk], [U])
        Qn, Ykk = tsqr(U - Qk @ Y, k + 1)
        Q[:, blk(k + 1)] = Qn
        R[upto(k), blk(k + 1)] = S + Y @ Skk
        R[blk(k + 1), blk(k + 1)] = Ykk @ Skk
    return Q, R


def bcgsi_plus_p_1s(X: np.ndarray, s: int):
    """BCGSI+P-1S, Alg. 2: one synchronization per block column.

    Follows Alg. 2 step by step.  Alg. 2's startup assumes q >= 3; for q = 2 the
    sync of its second step has no X_3 columns (the else-branch form), and for
    q = 1 the factorization is TSQR(X_1) alone.
    """
    X, m, n, q = _check(X, s)
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    blk = lambda k: slice((k - 1) * s, k * s)
    upto = lambda k: slice(0, k * s)
    Xb = lambda k: X[:, blk(k)]

    # Step 1: TSQR of X_1, first sync, Pythagorean chol, U_2.
    Q1, R11 = tsqr(Xb(1), 1)
    Q[:, blk(1)], R[blk(1), blk(1)] = Q1, R11
    if q == 1:
        return Q, R
    G = gram([Q1, Xb(2)], [Xb(2)])
    S12, T2 = G[:s], G[s:]
    S22 = chol(T2 - S12.T @ S12, 2)
    U = project_normalize(Xb(2), Q1, S12, S22)                       # U_2

    # Step 2: the synchronization [Q_1 U_2]^T [U_2 X_3] (and T_3).
    if q >= 3:
        G = gram([Q1, U], [U, Xb(3)])
        Y12, Z1, Om, P = G[:s, :s], G[:s, s:], G[s:, :s], G[s:, s:]
        T = gram([Xb(3)], [Xb(3)])                                   # T_3
    else:
        G = gram([Q1, U], [U])
        Y12, Om = G[:s], G[s:]
        Z1 = P = T = None

    # Step 3: Y_22, Q_2, R_12, R_22.
    Ykk = chol(Om - Y12.T @ Y12, 2)
    Q[:, blk(2)] = project_normalize(U, Q1, Y12, Ykk)
    R[blk(1), blk(2)] = S12 + Y12 @ S22
    R[blk(2), blk(2)] = Ykk @ S22
    Yprev, Zprev = Y12, Z1

    for k in range(2, q):                                            # k = 2..q-1
        # S_{1:k,k+1} by eq. (1); S_{k+1,k+1} by the Pythagorean chol.
        S = np.vstack([Zprev, delayed_projection(Ykk, P, Yprev, Zprev)])
        Sd = chol(T - S.T @ S, k + 1)
        Qk = Q[:, upto(k)]
        U = project_normalize(Xb(k + 1), Qk, S, Sd)                  # U_{k+1}
        if k < q - 1:
            G = gram([Qk, U], [U, Xb(k + 2)])
            Y, Z, Om, P = G[:k * s, :s], G[:k * s, s:], G[k * s:, :s], G[k * s:, s:]
            T = gram([Xb(k + 2)], [Xb(k + 2)])                       # T_{k+2}
        else:
            G = gram([Qk, U], [U])
            Y, Om = G[:k * s], G[k * s:]
            Z = P = T = None
        Yd = chol(Om - Y.T @ Y, k + 1)                               # Y_{k+1,k+1}
        Q[:, blk(k + 1)] = project_normalize(U, Qk, Y, Yd)           # Q_{k+1}
        R[upto(k), blk(k + 1)] = S + Y @ Sd
        R[blk(k + 1), blk(k + 1)] = Yd @ Sd
        Ykk, Yprev, Zprev = Yd, Y, Z
    return Q, R


def bcgsi_plus_p_2s(X: np.ndarray, s: int):
    """BCGSI+P-2S (Sec. 2): Alg. 2 with TSQR in place of the Pythagorean chol of
    its first intraorthogonalization (both the startup one and the one in the
    loop), so one more synchronization per block and T is never formed.  The
    paper prints no pseudocode; this is that substitution applied to Alg. 2:
        [Q_1, R_11] = TSQR(X_1);  S_12 = Q_1^T X_2;  [U_2, S_22] = TSQR(X_2 - Q_1 S_12)
        sync [Q_1 U_2]^T [U_2 X_3];  Y_22 = chol(Omega_2 - Y_12^T Y_12);  Q_2, R_12, R_22
        for k = 2..q-1:
            S_{1:k,k+1} by eq. (1);  [U_{k+1}, S_{k+1,k+1}] = TSQR(X_{k+1} - Q_k S_{1:k,k+1})
            sync [Q_k U_{k+1}]^T [U_{k+1} X_{k+2}]  (no X_{k+2} at k = q-1)
            Y_{k+1,k+1} = chol(Omega_{k+1} - Y^T Y);  Q_{k+1};  R_{1:k,k+1};  R_{k+1,k+1}
    """
    X, m, n, q = _check(X, s)
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    blk = lambda k: slice((k - 1) * s, k * s)
    upto = lambda k: slice(0, k * s)
    Xb = lambda k: X[:, blk(k)]

    Q1, R11 = tsqr(Xb(1), 1)
    Q[:, blk(1)], R[blk(1), blk(1)] = Q1, R11
    if q == 1:
        return Q, R
    S12 = gram([Q1], [Xb(2)])
    U, S22 = tsqr(Xb(2) - Q1 @ S12, 2)                               # U_2, S_22

    if q >= 3:
        G = gram([Q1, U], [U, Xb(3)])
        Y12, Z1, Om, P = G[:s, :s], G[:s, s:], G[s:, :s], G[s:, s:]
    else:
        G = gram([Q1, U], [U])
        Y12, Om = G[:s], G[s:]
        Z1 = P = None
    Ykk = chol(Om - Y12.T @ Y12, 2)
    Q[:, blk(2)] = project_normalize(U, Q1, Y12, Ykk)
    R[blk(1), blk(2)] = S12 + Y12 @ S22
    R[blk(2), blk(2)] = Ykk @ S22
    Yprev, Zprev = Y12, Z1

    for k in range(2, q):
        S = np.vstack([Zprev, delayed_projection(Ykk, P, Yprev, Zprev)])
        Qk = Q[:, upto(k)]
        U, Sd = tsqr(Xb(k + 1) - Qk @ S, k + 1)                       # U_{k+1}, S_{k+1,k+1}
        if k < q - 1:
            G = gram([Qk, U], [U, Xb(k + 2)])
            Y, Z, Om, P = G[:k * s, :s], G[:k * s, s:], G[k * s:, :s], G[k * s:, s:]
        else:
            G = gram([Qk, U], [U])
            Y, Om = G[:k * s], G[k * s:]
            Z = P = None
        Yd = chol(Om - Y.T @ Y, k + 1)
        Q[:, blk(k + 1)] = project_normalize(U, Qk, Y, Yd)
        R[upto(k), blk(k + 1)] = S + Y @ Sd
        R[blk(k + 1), blk(k + 1)] = Yd @ Sd
        Ykk, Yprev, Zprev = Yd, Y, Z
    return Q, R


def bcgs_pipi_plus(X: np.ndarray, s: int):
    """BCGS-PIPI+, Alg. 1: two synchronizations per block, both passes normalized
    by the Pythagorean Cholesky (O(u) loss of orthogonality for O(u) kappa^2 <= 1,
    Sec. 2).  Step by step as in Alg. 1:
        [Q_1, R_11] = TSQR(X_1)
        for k = 1..q-1:
            [S; T] = [Q_k X_{k+1}]^T X_{k+1}            (first synchronization)
            S_{k+1,k+1} = chol(T - S^T S)
            U = (X_{k+1} - Q_k S) S_{k+1,k+1}^{-1}
            [Y; Omega] = [Q_k U]^T U                    (second synchronization)
            Y_{k+1,k+1} = chol(Omega - Y^T Y);  Q_{k+1} = (U - Q_k Y) Y_{k+1,k+1}^{-1}
            R_{1:k,k+1} = S + Y S_{k+1,k+1};    R_{k+1,k+1} = Y_{k+1,k+1} S_{k+1,k+1}
    """
    X, m, n, q = _check(X, s)
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    blk = lambda k: slice((k - 1) * s, k * s)
    upto = lambda k: slice(0, k * s)
    Q[:, blk(1)], R[blk(1), blk(1)] = tsqr(X[:, blk(1)], 1)
    for k in range(1, q):
        c = k * s
        Qk = Q[:, upto(k)]
        Xk1 = X[:, blk(k + 1)]
        G1 = gram([Qk, Xk1], [Xk1])
        S, T = G1[:c], G1[c:]
        Skk = chol(T - S.T @ S, k + 1)
        U = project_normalize(Xk1, Qk, S, Skk)
        G2 = gram([Qk, U], [U])
        Y, Om = G2[:c], G2[c:]
        Ykk = chol(Om - Y.T @ Y, k + 1)
        Q[:, blk(k + 1)] = project_normalize(U, Qk, Y, Ykk)
        R[upto(k), blk(k + 1)] = S + Y @ Skk
        R[blk(k + 1), blk(k + 1)] = Ykk @ Skk
    return Q, R


def bcgsi_plus_1s(X: np.ndarray, s: int):
    """BCGSI+1s (also called BCGSI+LS), Sec. 2's one-sync subsection: delayed
    normalization as in Alg. 2, but the first intraorthogonalization is not
    done at all, so the Pythagorean Cholesky line of Alg. 2's loop (and of its
    startup) is dropped: S_{k+1,k+1} = I, U_{k+1} = X_{k+1} - Q_k S_{1:k,k+1}
    and T is never formed.  Table 1: O(u) kappa^2 loss of orthogonality,
    assuming O(u) kappa^3 <= 1.  The paper prints no pseudocode; this is Alg. 2
    with that line removed:
        [Q_1, R_11] = TSQR(X_1);  S_12 = Q_1^T X_2;  U_2 = X_2 - Q_1 S_12
        sync [Q_1 U_2]^T [U_2 X_3];  Y_22 = chol(Omega_2 - Y_12^T Y_12)
        Q_2 = (U_2 - Q_1 Y_12) Y_22^{-1};  R_12 = S_12 + Y_12;  R_22 = Y_22
        for k = 2..q-1:
            S_{1:k,k+1} by eq. (1);  U_{k+1} = X_{k+1} - Q_k S_{1:k,k+1}
            sync [Q_k U_{k+1}]^T [U_{k+1} X_{k+2}]  (no X_{k+2} at k = q-1)
            Y_{k+1,k+1} = chol(Omega_{k+1} - Y^T Y);  Q_{k+1} = (U_{k+1} - Q_k Y) Y_{k+1,k+1}^{-1}
            R_{1:k,k+1} = S_{1:k,k+1} + Y_{1:k,k+1};  R_{k+1,k+1} = Y_{k+1,k+1}
    (Alg. 2's R update with S_{k+1,k+1} = I.)
    """
    X, m, n, q = _check(X, s)
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    blk = lambda k: slice((k - 1) * s, k * s)
    upto = lambda k: slice(0, k * s)
    Xb = lambda k: X[:, blk(k)]

    Q1, R11 = tsqr(Xb(1), 1)
    Q[:, blk(1)], R[blk(1), blk(1)] = Q1, R11
    if q == 1:
        return Q, R
    S12 = gram([Q1], [Xb(2)])
    U = Xb(2) - Q1 @ S12                                             # U_2 (not normalized)

    if q >= 3:
        G = gram([Q1, U], [U, Xb(3)])
        Y12, Z1, Om, P = G[:s, :s], G[:s, s:], G[s:, :s], G[s:, s:]
    else:
        G = gram([Q1, U], [U])
        Y12, Om = G[:s], G[s:]
        Z1 = P = None
    Ykk = chol(Om - Y12.T @ Y12, 2)
    Q[:, blk(2)] = project_normalize(U, Q1, Y12, Ykk)
    R[blk(1), blk(2)] = S12 + Y12
    R[blk(2), blk(2)] = Ykk
    Yprev, Zprev = Y12, Z1

    for k in range(2, q):
        S = np.vstack([Zprev, delayed_projection(Ykk, P, Yprev, Zprev)])
        Qk = Q[:, upto(k)]
        U = Xb(k + 1) - Qk @ S                                       # U_{k+1}
        if k < q - 1:
            G = gram([Qk, U], [U, Xb(k + 2)])
            Y, Z, Om, P = G[:k * s, :s], G[:k * s, s:], G[k * s:, :s], G[k * s:, s:]
        else:
            G = gram([Qk, U], [U])
            Y, Om = G[:k * s], G[k * s:]
            Z = P = None
        Yd = chol(Om - Y.T @ Y, k + 1)
        Q[:, blk(k + 1)] = project_normalize(U, Qk, Y, Yd)
        R[upto(k), blk(k + 1)] = S + Y
        R[blk(k + 1), blk(k + 1)] = Yd
        Ykk, Yprev, Zprev = Yd, Y, Z
    return Q, R


VARIANTS = {
    "bcgsi+": bcgsi_plus,
    "bcgsi+p-1s": bcgsi_plus_p_1s,
    "bcgsi+p-2s": bcgsi_plus_p_2s,
    "bcgs-pipi+": bcgs_pipi_plus,
    "bcgsi+1s": bcgsi_plus_1s,
}


# The variant whose step finalizes a block at once, in the stability range of
# each variant (Table 1): BCGSI+ for BCGSI+ and BCGSI+P-2S, BCGS-PIPI+ for
# BCGSI+P-1S and BCGS-PIPI+, and BCGS-PIPI+ for BCGSI+1s (its range,
# O(u) kappa^2 <= 1, contains BCGSI+1s's O(u) kappa^3 <= 1).
EAGER_FAMILY = {"bcgsi+": "bcgsi+", "bcgsi+p-2s": "bcgsi+", "bcgsi+p-1s": "bcgs-pipi+",
                "bcgs-pipi+": "bcgs-pipi+", "bcgsi+1s": "bcgs-pipi+"}


def eager_step(Qk: np.ndarray, Xn: np.ndarray, family: str, block: int):
    """One block step of BCGSI+ or of BCGS-PIPI+ (Alg. 1) for a new block Xn of
    any width against the final basis Qk; returns Q_new, R_{1:k,new}, R_new,new.
        BCGSI+:      S = Q^T Xn, [U, S_nn] = TSQR(Xn - Q S), Y = Q^T U, [Q_new, Y_nn] = TSQR(U - Q Y)
        BCGS-PIPI+:  [S; T] = [Q Xn]^T Xn, S_nn = chol(T - S^T S), U = (Xn - Q S) S_nn^{-1},
                     [Y; Omega] = [Q U]^T U, Y_nn = chol(Omega - Y^T Y), Q_new = (U - Q Y) Y_nn^{-1}
        R_{1:k,new} = S + Y S_nn,  R_new,new = Y_nn S_nn
    """
    c = Qk.shape[1]
    if family == "bcgsi+":
        S = gram([Qk], [Xn])
        U, Skk = tsqr(Xn - Qk @ S, block)
        Y = gram([Qk], [U])
        Qn, Ykk = tsqr(U - Qk @ Y, block)
    else:
        G1 = gram([Qk, Xn], [Xn])
        S, T = G1[:c], G1[c:]
        Skk = chol(T - S.T @ S, block)
        U = project_normalize(Xn, Qk, S, Skk)
        G2 = gram([Qk, U], [U])
        Y, Om = G2[:c], G2[c:]
        Ykk = chol(Om - Y.T @ Y, block)
        Qn = project_normalize(U, Qk, Y, Ykk)
    return Qn, S + Y @ Skk, Ykk @ Skk


def factor(X: np.ndarray, s: int, variant: str):
    """Dispatch by variant name ("bcgsi+", "bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+",
    "bcgsi+1s").

    n need not be a multiple of s (the paper assumes it is).  Reading for a
    ragged last block of r = n mod s columns: the first n - r columns are
    factored by the variant (its last full block finalized as in its own last
    step), then the ragged block takes one step of EAGER_FAMILY[variant]; for
    n < s the factorization is TSQR(X) alone.
    """
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    r = n % s if s >= 1 else 0
    if s < 1 or r == 0:
        return VARIANTS[variant](X, s)
    if m < n:
        raise ValueError("need m >= n")
    n1 = n - r
    q = n1 // s + 1
    if n1 == 0:
        return tsqr(X, 1)
    Q1, R1 = VARIANTS[variant](X[:, :n1], s)
    Qn, Rt, Rd = eager_step(Q1, X[:, n1:], EAGER_FAMILY[variant], q)
    R = np.zeros((n, n))
    R[:n1, :n1] = R1
    R[:n1, n1:] = Rt
    R[n1:, n1:] = Rd
    return np.hstack([Q1, Qn]), R
