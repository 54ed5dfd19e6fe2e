"""Per-kernel parity of the CUDA path (through the C ABI) against the oracle's
steps: the Gram reduction (the synchronization of Sec. 3), the projection plus
triangular solve (Alg. 1, Alg. 2), TSQR and chol.

Tolerances are derived from the arithmetic: a sum of K products computed in any
order differs from the exact one by at most (K-1) u sum|a_i b_i|; the Gram kernel
adds chunk_rows products per chunk and then nchunks partials, numpy's matmul its
own order, so their difference is bounded by 2 (chunk_rows + nchunks) u (|A|^T|B|).
"""
import numpy as np
import pytest

import oracle
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu


def chunking(m):
    target = 304
    cr = -(-m // target)
    cr = -(-cr // 16) * 16
    cr = max(cr, 64)
    return cr, -(-m // cr)


@pytest.mark.parametrize("m,ka,kb", [(1, 1, 1), (37, 5, 3), (10000, 64, 16), (100003, 256, 32),
                                     (5000, 520, 32), (1000, 1, 64), (70001, 17, 9)])
def test_gram_parity_and_determinism(cuda, m, ka, kb):
    rng = np.random.default_rng(m + ka * 7 + kb)
    A = rng.standard_normal((m, ka))
    B = rng.standard_normal((m, kb)) * np.exp(rng.standard_normal((m, 1)))
    Ad, Bd = cuda.to_device_colmajor(A), cuda.to_device_colmajor(B)
    C1 = cuda.gram(Ad, Bd).cpu().numpy()
    C2 = cuda.gram(Ad, Bd).cpu().numpy()
    assert np.array_equal(C1, C2)  # fixed reduction order
    Co = oracle.gram([A], [B])
    cr, nc = chunking(m)
    bound = 2 * (cr + nc + 2) * U64 * (np.abs(A).T @ np.abs(B))
    assert np.all(np.abs(C1 - Co) <= bound + 1e-300)


@pytest.mark.parametrize("m,c,s,with_t", [(1, 0, 1, True), (129, 3, 2, True), (10000, 56, 8, True),
                                          (10000, 56, 8, False), (65537, 240, 16, True),
                                          (3000, 96, 32, True), (500, 100, 64, True),
                                          (257, 0, 5, True)])
def test_project_parity(cuda, m, c, s, with_t):
    rng = np.random.default_rng(m + c + s)
    V = rng.standard_normal((m, s))
    Q = np.linalg.qr(rng.standard_normal((m, max(c, 1))))[0][:, :c] if c else np.zeros((m, 0))
    C = rng.standard_normal((c, s))
    T = synth.make_upper_triangular_np(s, 10.0, seed=s) if with_t else None
    Wo = oracle.project_normalize(V, Q, C, T if with_t else np.eye(s))
    Vd = cuda.to_device_colmajor(V)
    Qd = cuda.to_device_colmajor(Q) if c else None
    Cd = cuda.to_device_colmajor(C) if c else None
    Td = cuda.to_device_colmajor(T) if with_t else None
    W = cuda.project(Vd, Qd, Cd, Td).cpu().numpy()
    # |V - QC| error bound (c+1) u (|V| + |Q||C|), amplified by the solve with T
    scale = np.abs(V) + (np.abs(Q) @ np.abs(C) if c else 0)
    kt = oracle.kappa(T) if with_t else 1.0
    tol = 4 * (c + s + 2) * U64 * kt * np.max(scale) / (np.min(np.abs(np.diag(T))) if with_t else 1)
    assert np.max(np.abs(W - Wo)) <= tol


@pytest.mark.parametrize("m,s,kappa", [(1, 1, 1.0), (7, 3, 10.0), (1000, 8, 1e3), (100003, 16, 1e6),
                                       (262149, 32, 1e2), (64, 64, 1e2), (70000, 1, 1.0),
                                       (513, 16, 1e4)])
def test_tsqr_parity(cuda, m, s, kappa):
    X = synth.make_matrix_np(m, s, kappa, seed=m + s) if m >= s else None
    Qo, Ro = oracle.householder_qr(X)
    Q, R, code, _ = cuda.tsqr(cuda.to_device_colmajor(X))
    assert code == 0
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    k = oracle.kappa(X)
    tol = 50 * max(s, 4) * k * U64 * np.sqrt(np.log2(m) + 1)
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) < tol
    assert np.max(np.abs(Q - Qo)) < tol
    assert np.all(np.diag(R) >= 0) and np.array_equal(np.tril(R, -1), np.zeros((s, s)))
    assert oracle.loo(Q) < 1e-13 * max(1.0, np.log2(m))
    assert oracle.residual(X, Q, R) < 1e-14 * max(1.0, np.log2(m))


def test_tsqr_reports_rank_deficiency_and_nonfinite(cuda):
    X = synth.make_matrix_np(3000, 8, 1e2, seed=3)
    Xz = X.copy()
    Xz[:, 3] = 0.0
    _, _, code, blk = cuda.tsqr(cuda.to_device_colmajor(Xz))
    assert cuda.STATUS[code] == "rank_deficient" and blk == 1
    Xn = X.copy()
    Xn[1234, 5] = np.inf
    _, _, code, _ = cuda.tsqr(cuda.to_device_colmajor(Xn))
    assert cuda.STATUS[code] == "nonfinite"


@pytest.mark.parametrize("s", [1, 4, 16, 33, 64])
def test_chol_parity(cuda, s):
    R0 = synth.make_upper_triangular_np(s, 1e3, seed=s)
    A = R0.T @ R0
    R, code = cuda.chol(cuda.to_device_colmajor(A))
    assert code == 0
    R = R.cpu().numpy()
    Ro = oracle.chol(A)
    assert np.max(np.abs(R - Ro)) / np.max(np.abs(Ro)) < 20 * s * 1e6 * U64


def test_chol_reports_not_spd(cuda):
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    _, code = cuda.chol(cuda.to_device_colmajor(A))
    assert cuda.STATUS[code] == "not_spd"
    A = np.array([[np.nan, 0.0], [0.0, 1.0]])
    _, code = cuda.chol(cuda.to_device_colmajor(A))
    assert cuda.STATUS[code] == "nonfinite"


def test_bounded_wait_runs_out_and_reports_timeout(cuda):
    """A device wait on a barrier that nothing completes gives up after its
    bound and records BCGS_ERR_TIMEOUT (no fault, no hang); the context stays
    usable: a factorization right after it succeeds."""
    import torch

    lib = cuda.load_library()
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    assert lib.bcgs_wait_selftest(ws.data_ptr(), ws.numel(), 2_000_000, None) == 0
    code, blk = cuda.factor_status(ws)
    assert cuda.STATUS[code] == "timeout" and blk == 0
    X = synth.make_matrix_np(5000, 32, 1e3, seed=3)
    Q, R, code, _ = cuda.factor(cuda.to_device_colmajor(X), 8, "bcgsi+p-1s")
    assert code == 0 and oracle.residual(X, Q.cpu().numpy(), R.cpu().numpy()) <= 1e-13
