"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each check is a closed form, a
library routine (LAPACK), a 60-digit computation, a special case that reduces to
a textbook algorithm, or an identity of the method (Sec. 1, Alg. 1, Alg. 2,
eq. (1), Table 1).  The mutation tests at the end plant plausible mistakes in
the oracle and check that the pins catch them.
"""
import numpy as np
import pytest

import oracle
from oracle import bcgs as ob
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
VARIANTS = list(oracle.VARIANTS)


def sign_normalized_lapack_qr(X):
    Q, R = np.linalg.qr(X)
    d = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * d[None, :], d[:, None] * R


# ---------------------------------------------------------------- Householder

@pytest.mark.parametrize("m,s", [(1, 1), (5, 1), (8, 8), (50, 7), (300, 24), (1000, 16)])
def test_householder_matches_lapack(m, s):
    X = np.random.default_rng(m * 31 + s).standard_normal((m, s))
    Q, R = oracle.householder_qr(X)
    Ql, Rl = sign_normalized_lapack_qr(X)
    k = oracle.kappa(X)
    tol = 20 * max(m, 8) ** 0.5 * s * k * U64
    assert np.abs(R - Rl).max() / np.abs(Rl).max() < tol
    assert np.abs(Q - Ql).max() < tol
    assert np.all(np.diag(R) > 0)
    assert np.allclose(np.tril(R, -1), 0.0, atol=0)


def mp_qr(X, dps=60):
    """60-digit economic QR by Cholesky of the exactly formed Gram matrix."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = dps
    m, n = X.shape
    A = mp.matrix([[mp.mpf(float(v)) for v in row] for row in X])
    G = A.T * A
    L = mp.cholesky(G)
    R = L.T
    Q = A * mp.inverse(R)
    Rf = np.array([[float(R[i, j]) for j in range(n)] for i in range(n)])
    Qf = np.array([[float(Q[i, j]) for j in range(n)] for i in range(m)])
    return Qf, Rf


@pytest.mark.parametrize("kappa", [1e1, 1e6])
def test_householder_matches_60_digit_qr(kappa):
    X = synth.make_matrix_np(14, 6, kappa, seed=7)
    Qe, Re = mp_qr(X)
    Q, R = oracle.householder_qr(X)
    tol = 50 * 6 * kappa * U64
    assert np.linalg.norm(R - Re) / np.linalg.norm(Re) < tol
    assert np.abs(Q - Qe).max() < tol


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("s", [1, 2, 4])
def test_variants_match_60_digit_qr(variant, s):
    X = synth.make_matrix_np(24, 8, 1e3, seed=11)
    Qe, Re = mp_qr(X)
    Q, R = oracle.factor(X, s, variant)
    tol = 100 * 8 * 1e3 * U64
    assert np.linalg.norm(R - Re) / np.linalg.norm(Re) < tol
    assert np.abs(Q - Qe).max() < tol


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("variant", VARIANTS)
def test_hand_example(variant, golden):
    g = golden("hand_4x2.txt")
    X, R, Q = np.array(g["X"]), np.array(g["R"]), np.array(g["Q"])
    for s in (1, 2):
        Qo, Ro = oracle.factor(X, s, variant)
        assert np.abs(Ro - R).max() < 1e-14 * 10
        assert np.abs(Qo - Q).max() < 1e-15 * 10


def hadamard_case(golden):
    g = golden("hadamard_16x8.txt")
    m, n = g["m"], g["n"]
    h = np.array([[1.0]])
    while h.shape[0] < m:
        h = np.block([[h, h], [h, -h]])
    Q0 = h[:, :n] / 4.0
    R0 = np.array(g["R0"])
    X = np.array(g["X4"]) / 4.0
    assert np.array_equal(Q0 @ R0, X)  # exact in binary
    return X, Q0, R0


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("s", [1, 2, 4, 8])
def test_hadamard_exact_recovery(variant, s, golden):
    X, Q0, R0 = hadamard_case(golden)
    Q, R = oracle.factor(X, s, variant)
    k = oracle.kappa(R0)
    tol = 10 * 8 * k * U64
    assert np.abs(R - R0).max() / np.abs(R0).max() < tol
    assert np.abs(Q - Q0).max() < tol


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_recovery_of_R0(variant, kappa):
    """X = Q0 R0 with known orthonormal Q0 and positive-diagonal R0."""
    m, n, s = 600, 32, 4
    Q0, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((m, n)))
    R0 = synth.make_upper_triangular_np(n, kappa, seed=5)
    X = Q0 @ R0
    Q, R = oracle.factor(X, s, variant)
    k = oracle.kappa(R0)
    tol = 10 * n * k * U64
    assert np.linalg.norm(R - R0) / np.linalg.norm(R0) < tol
    assert np.abs(Q - Q0).max() < tol


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("variant", VARIANTS)
def test_s_equals_n_is_tsqr(variant):
    X = synth.make_matrix_np(200, 12, 1e5, seed=9)
    Q, R = oracle.factor(X, 12, variant)
    Qh, Rh = oracle.householder_qr(X)
    assert np.array_equal(Q, Qh) and np.array_equal(R, Rh)
    Ql, Rl = sign_normalized_lapack_qr(X)
    assert np.abs(R - Rl).max() / np.abs(Rl).max() < 1e-10


def textbook_cgs2(X):
    """Column-wise classical Gram-Schmidt with one reorthogonalization (CGS2),
    vector form, normalization by the 2-norm."""
    m, n = X.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    for j in range(n):
        x = X[:, j].copy()
        r1 = Q[:, :j].T @ x
        v = x - Q[:, :j] @ r1
        r2 = Q[:, :j].T @ v
        w = v - Q[:, :j] @ r2
        nrm = np.sqrt(w @ w)
        Q[:, j] = w / nrm
        R[:j, j] = r1 + r2
        R[j, j] = nrm
    return Q, R


def test_pipi_plus_first_pass_is_pythagorean_cholqr():
    """Alg. 1's first pass of a block equals a Cholesky QR of X_{k+1} - Q_k S:
    S_{k+1,k+1} is its R factor and U its Q factor (Pythagorean identity), checked
    on one block against LAPACK's QR of the projected block."""
    rng = np.random.default_rng(71)
    Qk, _ = np.linalg.qr(rng.standard_normal((600, 12)))
    X2 = rng.standard_normal((600, 4)) * np.array([1.0, 1e-2, 1e2, 3.0])
    Q, R = oracle.bcgs_pipi_plus(np.hstack([Qk @ np.diag(np.arange(1.0, 13.0)), X2]), 4)
    V = X2 - Qk @ (Qk.T @ X2)
    Ql, Rl = sign_normalized_lapack_qr(V)
    # final block of Q spans the projected block with positive diagonal R
    assert np.abs(Q[:, 12:] - Ql).max() < 1e-10
    assert np.abs(np.abs(np.diag(R)[12:]) - np.abs(np.diag(Rl))).max() / np.abs(np.diag(Rl)).max() < 1e-10


def test_s_equals_1_is_cgs2():
    """BCGSI+ with s = 1 is CGSI+ (Sec. 4, Table 2's normalization point)."""
    X = synth.make_matrix_np(400, 20, 1e6, seed=13)
    Q, R = oracle.bcgsi_plus(X, 1)
    Qc, Rc = textbook_cgs2(X)
    # The second pass's diagonal differs from ||v|| only by O(u) terms.
    assert np.linalg.norm(R - Rc) / np.linalg.norm(Rc) < 1e-12
    assert np.abs(Q - Qc).max() < 1e-9


@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_cross_variant_agreement(kappa):
    X = synth.make_matrix_np(1500, 48, kappa, seed=17)
    Rs = [oracle.factor(X, 8, v)[1] for v in VARIANTS]
    for R in Rs[1:]:
        assert np.linalg.norm(R - Rs[0]) / np.linalg.norm(Rs[0]) < 50 * 48 * kappa * U64


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("kappa", [1e2, 1e5, 1e8])
def test_invariants(variant, kappa):
    m, n, s = 3000, 64, 8
    X = synth.make_matrix_np(m, n, kappa, seed=19)
    if variant in ("bcgsi+p-1s", "bcgs-pipi+", "bcgsi+1s") and kappa >= 1e8:
        pytest.skip("outside Table 1's O(u) kappa^2 <= 1 (O(u) kappa^3 <= 1 for BCGSI+1s) range")
    Q, R = oracle.factor(X, s, variant)
    assert np.array_equal(np.tril(R, -1), np.zeros_like(R))
    assert np.all(np.diag(R) > 0)
    nx2 = np.linalg.norm(X, 2) ** 2
    assert np.linalg.norm(X.T @ X - R.T @ R, 2) / nx2 < 100 * n * U64
    assert oracle.residual(X, Q, R) < 1e-14
    # Table 1: O(u) loss of orthogonality, O(u) kappa^2 for BCGSI+1s
    assert oracle.loo(Q) < (10 * n * U64 * kappa ** 2 if variant == "bcgsi+1s" else 1e-13)


def test_pythagorean_identity():
    """T - S^T S equals (X - Q S)^T (X - Q S) for S = Q^T X (Alg. 1, the chol
    step): its Cholesky factor equals the R factor of X - Q S."""
    rng = np.random.default_rng(23)
    Qk, _ = np.linalg.qr(rng.standard_normal((800, 16)))
    X = synth.make_matrix_np(800, 4, 1e2, seed=29) + 0.3 * Qk[:, :4]
    S = Qk.T @ X
    T = X.T @ X
    Rp = oracle.chol(T - S.T @ S)
    _, Rh = oracle.householder_qr(X - Qk @ S)
    assert np.linalg.norm(Rp - Rh) / np.linalg.norm(Rh) < 1e-12


def eq1_error(fn):
    """|Q_k^T X_{k+1} - fn(Y_kk, P_k, Y_{1:k-1,k}, Z_{k-1})| on a case where
    U_k is far from orthogonal to Q_{k-1}, so every term of eq. (1) matters."""
    rng = np.random.default_rng(31)
    m, c, s = 900, 12, 4
    Qprev, _ = np.linalg.qr(rng.standard_normal((m, c)))
    Uk = rng.standard_normal((m, s)) + Qprev[:, :s]
    Xn = rng.standard_normal((m, s)) + Qprev[:, s:2 * s]
    Y = Qprev.T @ Uk
    Om = Uk.T @ Uk
    Ykk = oracle.chol(Om - Y.T @ Y)
    Qk = (Uk - Qprev @ Y) @ np.linalg.inv(Ykk)
    P = Uk.T @ Xn
    Z = Qprev.T @ Xn
    return np.abs(Qk.T @ Xn - fn(Ykk, P, Y, Z)).max()


def test_eq1_delayed_projection_equals_direct():
    """Eq. (1): Q_k^T X_{k+1} = Y_kk^{-T} (P_k - Y_{1:k-1,k}^T Z_{k-1})."""
    assert eq1_error(ob.delayed_projection) < 1e-12


def test_variants_use_eq1(monkeypatch):
    calls = []
    good = ob.delayed_projection

    def counting(*a):
        calls.append(1)
        return good(*a)
    monkeypatch.setattr(ob, "delayed_projection", counting)
    X = synth.make_matrix_np(200, 20, 1e2, seed=71)
    for v in ("bcgsi+p-1s", "bcgsi+p-2s", "bcgsi+1s"):
        calls.clear()
        oracle.factor(X, 4, v)
        assert len(calls) == 5 - 2  # k = 2..q-1


def test_chol_closed_forms():
    a, b, c = 4.0, 2.0, 5.0
    R = oracle.chol(np.array([[a, b], [b, c]]))
    exp = np.array([[2.0, 1.0], [0.0, 2.0]])  # sqrt(4)=2, 2/2=1, sqrt(5-1)=2
    assert np.array_equal(R, exp)
    R0 = synth.make_upper_triangular_np(10, 1e3, seed=37)
    assert np.abs(oracle.chol(R0.T @ R0) - R0).max() / np.abs(R0).max() < 1e-10
    with pytest.raises(oracle.Breakdown) as e:
        oracle.chol(np.array([[1.0, 2.0], [2.0, 1.0]]), block=3)
    assert e.value.kind == "not_spd" and e.value.block == 3


def test_triangular_solves_by_multiplication():
    rng = np.random.default_rng(41)
    T = synth.make_upper_triangular_np(6, 1e2, seed=43)
    V = rng.standard_normal((50, 6))
    W = oracle.solve_right_upper(V, T)
    assert np.abs(W @ T - V).max() < 1e-12
    M = rng.standard_normal((6, 5))
    W2 = oracle.solve_left_upper_t(T, M)
    assert np.abs(T.T @ W2 - M).max() < 1e-12


# ---------------------------------------------------------------- Table 1

def test_table1_loo_ordering():
    """Table 1: BCGSI+ and BCGSI+P-2S keep O(u) loss of orthogonality while
    O(u) kappa <= 1 (here kappa = 1e10), BCGSI+P-1S needs O(u) kappa^2 <= 1 and
    breaks down (or loses orthogonality) at kappa = 1e10."""
    X = synth.make_matrix_np(3000, 64, 1e10, seed=47)
    for v in ("bcgsi+", "bcgsi+p-2s"):
        Q, R = oracle.factor(X, 8, v)
        assert oracle.loo(Q) < 1e-13
    for v in ("bcgsi+p-1s", "bcgs-pipi+"):  # both need O(u) kappa^2 <= 1 (Sec. 2)
        try:
            Q, _ = oracle.factor(X, 8, v)
            assert oracle.loo(Q) > 1e-10
        except oracle.Breakdown as e:
            assert e.kind == "not_spd"


# ---------------------------------------------------------------- degenerate inputs

def test_bcgsi_plus_1s_has_no_first_pythagorean_cholesky():
    """BCGSI+1s drops Alg. 2's first Cholesky line (Sec. 2): U_{k+1} = X_{k+1} -
    Q_k S is formed explicitly and T - S^T S never is.  At kappa = 1e10, where
    O(u) kappa^2 > 1 and BCGSI+P-1S's Pythagorean Cholesky of T - S^T S breaks
    down (Table 1), BCGSI+1s still completes with a backward-stable R; a version
    that kept the dropped line would break down like BCGSI+P-1S."""
    X = synth.make_matrix_np(3000, 64, 1e10, seed=47)
    with pytest.raises(oracle.Breakdown) as e:
        oracle.factor(X, 8, "bcgsi+p-1s")
    assert e.value.kind == "not_spd"
    Q, R = oracle.factor(X, 8, "bcgsi+1s")
    nx2 = np.linalg.norm(X, 2) ** 2
    assert np.linalg.norm(X.T @ X - R.T @ R, 2) / nx2 < 100 * 64 * U64
    assert oracle.residual(X, Q, R) < 1e-14
    assert np.all(np.diag(R) > 0)


def test_bcgsi_plus_1s_loss_of_orthogonality_grows_with_kappa():
    """Table 1: BCGSI+1s's loss of orthogonality is O(u) kappa^2 (bounded by it
    and growing with kappa), BCGSI+P-1S's stays O(u) over the same range."""
    for seed in (19, 47):
        loo = {}
        for kappa in (1e2, 1e8):
            X = synth.make_matrix_np(3000, 64, kappa, seed=seed)
            loo[kappa] = oracle.loo(oracle.factor(X, 8, "bcgsi+1s")[0])
            assert loo[kappa] <= 10 * 64 * U64 * kappa ** 2
            assert oracle.loo(oracle.factor(X, 8, "bcgsi+p-1s")[0]) < 1e-14
        assert loo[1e8] > 10 * loo[1e2]


def test_bcgsi_plus_1s_r_has_identity_first_normalization():
    """With S_{k+1,k+1} = I the R update of Alg. 2 reads R_{1:k,k+1} = S + Y and
    R_{k+1,k+1} = Y_{k+1,k+1}: for q = 2 blocks the factors are TSQR(X_1),
    S_12 = Q_1^T X_2, U_2 = X_2 - Q_1 S_12, [Y_12; Omega] = [Q_1 U_2]^T U_2 and the
    Cholesky of Omega - Y^T Y, written out here from those definitions."""
    X = synth.make_matrix_np(500, 8, 1e3, seed=83)
    Q1, R11 = oracle.householder_qr(X[:, :4])
    S12 = Q1.T @ X[:, 4:]
    U2 = X[:, 4:] - Q1 @ S12
    Y12 = Q1.T @ U2
    L = np.linalg.cholesky(U2.T @ U2 - Y12.T @ Y12)  # lower, L L^T
    Y22 = L.T
    Q, R = oracle.factor(X, 4, "bcgsi+1s")
    assert np.allclose(R[:4, :4], R11, rtol=0, atol=1e-13 * np.abs(R11).max())
    assert np.abs(R[:4, 4:] - (S12 + Y12)).max() < 1e-13 * np.abs(R).max()
    assert np.abs(R[4:, 4:] - Y22).max() < 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("variant", VARIANTS)
def test_breakdowns(variant):
    X = synth.make_matrix_np(100, 8, 1e2, seed=53)
    Xz = X.copy()
    Xz[:, 0:2] = 0.0
    with pytest.raises(oracle.Breakdown) as e:
        oracle.factor(Xz, 2, variant)
    assert e.value.kind == "rank_deficient" and e.value.block == 1
    Xn = X.copy()
    Xn[5, 0] = np.nan
    with pytest.raises(oracle.Breakdown) as e:
        oracle.factor(Xn, 2, variant)
    assert e.value.kind == "nonfinite"
    # n mod s != 0 is a ragged last block (taken by one eager step); m < n is rejected either way
    with pytest.raises(ValueError):
        oracle.factor(X[:5], 3, variant)
    with pytest.raises(ValueError):
        oracle.factor(X[:1], 2, variant)


# ---------------------------------------------------------------- mutations

def _recovery_error(variant):
    m, n, s = 400, 24, 4
    Q0, _ = np.linalg.qr(np.random.default_rng(59).standard_normal((m, n)))
    R0 = synth.make_upper_triangular_np(n, 1e3, seed=61)
    try:
        Q, R = oracle.factor(Q0 @ R0, s, variant)
    except oracle.Breakdown:
        return np.inf  # a breakdown on this well-conditioned input also fails the pin
    return max(np.linalg.norm(R - R0) / np.linalg.norm(R0), np.abs(Q - Q0).max())


def test_mutation_dropped_term_in_eq1_is_caught(monkeypatch):
    monkeypatch.setattr(ob, "delayed_projection",
                        lambda Ykk, P, Y, Z: ob.solve_left_upper_t(Ykk, P))
    assert eq1_error(ob.delayed_projection) > 1e-3


def _solve_pin_error():
    rng = np.random.default_rng(41)
    T = synth.make_upper_triangular_np(6, 1e2, seed=43)
    V = rng.standard_normal((50, 6))
    return np.abs(ob.solve_right_upper(V, T) @ T - V).max()


def test_mutation_transposed_index_in_solve_is_caught(monkeypatch):
    def bad_solve(V, T):
        s = T.shape[0]
        W = np.zeros_like(V)
        for j in range(s):
            W[:, j] = (V[:, j] - W[:, :j] @ T[j, :j]) / T[j, j]
        return W
    assert _solve_pin_error() < 1e-12
    monkeypatch.setattr(ob, "solve_right_upper", bad_solve)
    assert _solve_pin_error() > 1e-3
    # In BCGSI+P-1S and BCGS-PIPI+ the solve by S_{k+1,k+1} (far from identity) is exposed.
    assert _recovery_error("bcgsi+p-1s") > 1e-6
    assert _recovery_error("bcgs-pipi+") > 1e-6


def test_mutation_wrong_sign_in_chol_is_caught(monkeypatch):
    good = ob.chol

    def bad_chol(A, block=1):
        R = good(A, block)
        return R - 2 * np.triu(R, 1)
    R0 = synth.make_upper_triangular_np(10, 1e3, seed=37)
    assert np.abs(ob.chol(R0.T @ R0) - R0).max() < 1e-10
    monkeypatch.setattr(ob, "chol", bad_chol)
    assert np.abs(ob.chol(R0.T @ R0) - R0).max() > 1e-3
    # BCGSI+P-1S's and BCGS-PIPI+'s S_{k+1,k+1} = chol(T - S^T S) is far from
    # identity, and BCGSI+1s's R_{k+1,k+1} = Y_{k+1,k+1} = chol(Omega - Y^T Y) of
    # its unnormalized U; in BCGSI+P-2S chol only factors Omega - Y^T Y ~ I, and
    # BCGSI+ has no chol.
    assert _recovery_error("bcgsi+p-1s") > 1e-6
    assert _recovery_error("bcgs-pipi+") > 1e-6
    assert _recovery_error("bcgsi+1s") > 1e-6


def test_mutation_missing_sign_normalization_is_caught(monkeypatch):
    good = ob.householder_qr

    def bad_hh(A, block=1):
        Q, R = good(A, block)
        return -Q, -R
    monkeypatch.setattr(ob, "householder_qr", bad_hh)
    X = synth.make_matrix_np(50, 6, 1e2, seed=67)
    Q, R = ob.householder_qr(X)
    Ql, Rl = sign_normalized_lapack_qr(X)
    assert np.abs(R - Rl).max() > 1e-3
    for v in VARIANTS:
        assert _recovery_error(v) > 1e-6


# ---- a ragged last block (n mod s != 0): R is unique for a full-rank X with
# positive diagonal, so every variant must reproduce LAPACK's sign-normalized R


def _lapack_r(X):
    _, R = np.linalg.qr(X)
    return np.sign(np.diag(R))[:, None] * R


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m,n,s", [(300, 21, 8), (400, 13, 4), (150, 5, 8), (600, 33, 16), (200, 17, 16)])
def test_ragged_last_block_matches_lapack(variant, m, n, s):
    X = synth.make_matrix_np(m, n, 1e3, seed=m + n + s)
    Q, R = oracle.factor(X, s, variant)
    assert Q.shape == (m, n) and R.shape == (n, n)
    Rl = _lapack_r(X)
    assert np.linalg.norm(R - Rl) / np.linalg.norm(Rl) <= 10 * n * 1e3 * U64
    loo_gate = 10 * n * U64 * 1e3 ** 2 if variant == "bcgsi+1s" else 1e-13  # Table 1
    assert oracle.loo(Q) <= loo_gate and oracle.residual(X, Q, R) <= 1e-14
    assert np.array_equal(np.tril(R, -1), np.zeros_like(R)) and np.all(np.diag(R) > 0)


def test_ragged_first_columns_are_the_variants_own():
    """The full blocks are the variant's factorization of X[:, :n - r] unchanged."""
    X = synth.make_matrix_np(300, 21, 1e4, seed=7)
    for v in VARIANTS:
        Q, R = oracle.factor(X, 8, v)
        Q1, R1 = oracle.factor(X[:, :16], 8, v)
        assert np.array_equal(Q[:, :16], Q1) and np.array_equal(R[:16, :16], R1)


def test_eager_step_families():
    """The ragged step of BCGSI+ and 2S is a BCGSI+ step (TSQR passes), that of
    1S and BCGS-PIPI+ a BCGS-PIPI+ step (Pythagorean passes): at s = n - r the
    results equal the family's own factorization with that block size."""
    X = synth.make_matrix_np(300, 12, 1e3, seed=8)
    # n = 12, s = 8: one full block + a ragged block of 4; BCGSI+ with blocks
    # (8, 4) is the same arithmetic as its loop body on block 2
    Q, R = oracle.factor(X, 8, "bcgsi+p-2s")
    Q1, R1 = oracle.tsqr(X[:, :8], 1)
    Qn, Rt, Rd = oracle.eager_step(Q1, X[:, 8:], "bcgsi+", 2)
    assert np.array_equal(Q[:, 8:], Qn) and np.array_equal(R[:8, 8:], Rt) and np.array_equal(R[8:, 8:], Rd)
    assert oracle.EAGER_FAMILY == {"bcgsi+": "bcgsi+", "bcgsi+p-2s": "bcgsi+",
                                   "bcgsi+p-1s": "bcgs-pipi+", "bcgs-pipi+": "bcgs-pipi+",
                                   "bcgsi+1s": "bcgs-pipi+"}


def test_mutation_lost_coupling_block_in_the_ragged_step_is_caught(monkeypatch):
    """Planting R_{1:k,new} = 0 in the ragged step fails the LAPACK pin."""
    real = ob.eager_step

    def bad(Qk, Xn, family, block):
        Qn, Rt, Rd = real(Qk, Xn, family, block)
        return Qn, 0.0 * Rt, Rd

    X = synth.make_matrix_np(300, 21, 1e3, seed=9)
    Rl = _lapack_r(X)
    _, R = oracle.factor(X, 8, "bcgsi+p-1s")
    assert np.linalg.norm(R - Rl) / np.linalg.norm(Rl) < 1e-12
    monkeypatch.setattr(ob, "eager_step", bad)
    _, R = oracle.factor(X, 8, "bcgsi+p-1s")
    assert np.linalg.norm(R - Rl) / np.linalg.norm(Rl) > 1e-3


def test_mutation_single_pass_ragged_step_is_caught(monkeypatch):
    """Planting a ragged step without its second (reorthogonalization) pass
    fails the loss-of-orthogonality pin at kappa = 1e7."""

    def single(Qk, Xn, family, block):
        S = Qk.T @ Xn
        Qn, Skk = oracle.tsqr(Xn - Qk @ S, block)
        return Qn, S, Skk

    X = synth.make_matrix_np(2000, 40, 1e7, seed=10)
    Q, _ = oracle.factor(X, 16, "bcgsi+p-2s")
    assert oracle.loo(Q) <= 1e-13
    monkeypatch.setattr(ob, "eager_step", single)
    Q, _ = oracle.factor(X, 16, "bcgsi+p-2s")
    assert oracle.loo(Q) > 1e-11
