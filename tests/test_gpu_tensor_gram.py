"""The tensor-core Gram engine (bcgs_set_option(BCGS_OPT_GRAM_ENGINE, 2)).

Each operand entry is split exactly into eight 8-bit digits relative to its
column maximum (error-free splitting, Ozaki et al. 2012) and digit pairs with
t + u <= 7 are multiplied on the bf16 tensor cores with exact integer sums; the
error of one product term is at most 2^-57.1 max|a_i| max|b_j| and each chunk
partial is rounded once to FP64, then the partials are added in chunk order.
Derived bound used below, per entry:
    m max|a_i| max|b_j| 2^-57.1 + 2 (nchunks + 2) u (|A|^T |B|)_ij.
"""
import numpy as np
import pytest

import oracle
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu


@pytest.fixture
def tensor(cuda):
    cuda.set_gram_engine("tensor")
    yield cuda
    cuda.set_gram_engine("auto")


def nchunks(m):
    cr = -(-m // 304)
    cr = max(-(-cr // 16) * 16, 64)
    return -(-m // cr)


def test_integer_inputs_are_exact(tensor):
    """Integers of at most 7 bits are single digits: every product and every sum
    is exact, so the result equals the exact integer Gram bit for bit."""
    rng = np.random.default_rng(1)
    m, ka, kb = 50000, 200, 32
    A = rng.integers(-127, 128, size=(m, ka)).astype(np.float64)
    B = rng.integers(-127, 128, size=(m, kb)).astype(np.float64)
    exact = (A.astype(np.int64).T @ B.astype(np.int64)).astype(np.float64)
    C = tensor.gram(tensor.to_device_colmajor(A), tensor.to_device_colmajor(B)).cpu().numpy()
    assert np.array_equal(C, exact)


@pytest.mark.parametrize("m,ka,kb", [(1, 1, 1), (37, 5, 3), (10000, 64, 16), (100003, 256, 32),
                                     (70001, 300, 48), (20000, 17, 64), (4096, 130, 20)])
def test_tensor_gram_parity(tensor, m, ka, kb):
    rng = np.random.default_rng(m + ka + kb)
    A = rng.standard_normal((m, ka))
    B = rng.standard_normal((m, kb)) * np.exp(rng.standard_normal((m, 1)))
    Ad, Bd = tensor.to_device_colmajor(A), tensor.to_device_colmajor(B)
    C1 = tensor.gram(Ad, Bd).cpu().numpy()
    C2 = tensor.gram(Ad, Bd).cpu().numpy()
    assert np.array_equal(C1, C2)
    Co = oracle.gram([A], [B])
    amax_a = np.abs(A).max(axis=0)
    amax_b = np.abs(B).max(axis=0)
    bound = m * np.outer(amax_a, amax_b) * 2.0 ** -57.1 + 2 * (nchunks(m) + 2) * U64 * (np.abs(A).T @ np.abs(B))
    assert np.all(np.abs(C1 - Co) <= bound)


def test_tensor_gram_fp32_inputs_via_factorization(tensor):
    import torch

    X = synth.make_matrix_np(40000, 64, 1e3, seed=4)
    Q, R, code, _ = tensor.factor(tensor.to_device_colmajor(X, dtype=torch.float32), 16, "bcgsi+p-1s")
    assert code == 0
    Qh = Q.double().cpu().numpy()
    assert oracle.loo(Qh) <= 1e-6 and oracle.residual(X, Qh, R.cpu().numpy()) <= 1e-6


def test_tensor_gram_reports_nonfinite(tensor):
    X = synth.make_matrix_np(30000, 32, 1e2, seed=5)
    X[123, 9] = np.inf
    _, _, code, blk = tensor.factor(tensor.to_device_colmajor(X), 8, "bcgsi+p-1s")
    assert tensor.STATUS[code] == "nonfinite" and blk == 2


@pytest.mark.parametrize("variant", ["bcgsi+", "bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+"])
@pytest.mark.parametrize("engine", ["tensor", "fp64"])
def test_variants_on_each_engine(cuda, variant, engine):
    cuda.set_gram_engine(engine)
    try:
        for (m, n, s, kappa) in [(50000, 64, 8, 1e4), (3000, 48, 16, 1e6), (70000, 96, 32, 1e2)]:
            if variant in ("bcgsi+p-1s", "bcgs-pipi+") and kappa > 1e5:
                continue
            X = synth.make_matrix_np(m, n, kappa, seed=m + n)
            Q, R, code, _ = cuda.factor(cuda.to_device_colmajor(X), s, variant)
            assert code == 0
            Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
            Qo, Ro = oracle.factor(X, s, variant)
            assert oracle.residual(X, Qh, Rh) <= 1e-13 and oracle.loo(Qh) <= 1e-12
            tol = 10 * n * oracle.kappa(Ro) * U64
            assert np.linalg.norm(Rh - Ro) / np.linalg.norm(Ro) <= tol
            assert np.max(np.abs(Qh - Qo)) <= tol
    finally:
        cuda.set_gram_engine("auto")


def test_row_scaled_heavy_tails_meet_the_gates(cuda):
    """Row norms lognormal(0, 2): column maxima far above typical entries, the
    hardest case for fixed-point digits; the FP64 gates still hold."""
    cuda.set_gram_engine("tensor")
    try:
        X = synth.make_matrix_np(200000, 64, 1e5, seed=77, row_scaled=True)
        for v in ("bcgsi+", "bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+"):
            Q, R, code, _ = cuda.factor(cuda.to_device_colmajor(X), 16, v)
            assert code == 0
            Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
            assert oracle.residual(X, Qh, Rh) <= 1e-13
            assert oracle.loo(Qh) <= 1e-12
    finally:
        cuda.set_gram_engine("auto")


@pytest.mark.parametrize("m,c,s,with_t", [(129, 3, 2, True), (10000, 56, 8, True), (10000, 56, 8, False),
                                          (65537, 240, 16, True), (3000, 96, 32, True), (1000, 500, 5, True),
                                          (40000, 64, 16, False)])
def test_tensor_project_parity(tensor, m, c, s, with_t):
    """(V - Q C) T^{-1} with Q C on the tensor cores (row exponents of Q, column
    exponents of C) against the oracle; same derived FP64 tolerance as the
    FP64-pipe kernel (the digit error c 2^-57.1 max|q_r| max|c_j| is below it)."""
    rng = np.random.default_rng(m + c + s)
    V = rng.standard_normal((m, s))
    Q = np.linalg.qr(rng.standard_normal((m, c)))[0]
    C = rng.standard_normal((c, s))
    T = synth.make_upper_triangular_np(s, 10.0, seed=s) if with_t else None
    Wo = oracle.project_normalize(V, Q, C, T if with_t else np.eye(s))
    W = tensor.project(tensor.to_device_colmajor(V), tensor.to_device_colmajor(Q),
                       tensor.to_device_colmajor(C),
                       tensor.to_device_colmajor(T) if with_t else None).cpu().numpy()
    scale = np.abs(V) + np.abs(Q) @ np.abs(C)
    kt = oracle.kappa(T) if with_t else 1.0
    tol = 4 * (c + s + 2) * U64 * kt * np.max(scale) / (np.min(np.abs(np.diag(T))) if with_t else 1)
    assert np.max(np.abs(W - Wo)) <= tol
