"""The resident digit store of Q and the projections that read it.

With FP64 storage and the tensor engine, every block column of Q is split once
into exact balanced 8-bit digits (per 128-row block and column exponents) and
kept beside Q; the projections bulk-copy those digits to the tensor cores, and
BCGSI+P-1S / -2S run both projections of a step as one paired pass over
[Q_{1:k-1} U_k] (Q_{1:k} S_{1:k,k+1} = Q_{1:k-1} (Z - Y M) + U_k M with
M = Y_kk^{-1} W, eq. (1) regrouped).  The engine option "tensor" forces this
path for every row count, so ragged small shapes run through it here.
"""
import numpy as np
import pytest

import oracle
from conftest import loo_gate
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu

# (m, n, s, kappa): ragged row blocks, s not a multiple of 8, c not a multiple of
# 16, column groups past 128, s > 16 (single projections only), s = 1 (CGSI+) and 2
SHAPES = [(129, 40, 5, 1e3), (1000, 60, 3, 1e4), (3001, 72, 12, 1e5), (12345, 128, 8, 1e4),
          (20000, 160, 16, 1e5), (5000, 96, 24, 1e3), (700, 64, 4, 1e2), (40000, 272, 16, 1e5),
          (2048, 64, 32, 1e4), (3000, 20, 1, 1e3), (5000, 36, 2, 1e4)]


@pytest.fixture
def tensor(cuda):
    cuda.set_gram_engine("tensor")
    yield cuda
    cuda.set_gram_engine("auto")


def check_against_oracle(X, s, variant, Q, R):
    n = X.shape[1]
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro = oracle.factor(X, s, variant)
    assert oracle.residual(X, Qh, Rh) <= 1e-13
    assert oracle.loo(Qh) <= loo_gate(variant, n, oracle.kappa(Ro), oracle.loo(Qo))
    tol = 10 * n * oracle.kappa(Ro) * U64
    assert np.linalg.norm(Rh - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Qh - Qo)) <= tol


@pytest.mark.parametrize("variant", ["bcgsi+", "bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+", "bcgsi+1s"])
@pytest.mark.parametrize("m,n,s,kappa", SHAPES)
def test_store_path_matches_the_oracle(tensor, variant, m, n, s, kappa):
    if variant in ("bcgsi+p-1s", "bcgs-pipi+") and kappa > 1e5:
        pytest.skip("1S is for kappa <= 1e5")
    X = synth.make_matrix_np(m, n, kappa, seed=m + 3 * n + s)
    Xd = tensor.to_device_colmajor(X)
    Q, R, code, _ = tensor.factor(Xd, s, variant)
    assert code == 0
    check_against_oracle(X, s, variant, Q, R)
    Q2, R2, code2, _ = tensor.factor(Xd, s, variant)
    assert code2 == 0
    assert np.array_equal(Q.cpu().numpy(), Q2.cpu().numpy())
    assert np.array_equal(R.cpu().numpy(), R2.cpu().numpy())


@pytest.mark.parametrize("variant", ["bcgsi+", "bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+", "bcgsi+1s"])
def test_store_and_on_the_fly_paths_agree(tensor, variant):
    """A workspace sized without the store runs the same factorization with the
    on-the-fly tensor projections; both meet the FP64 gates and agree to the
    derived tolerance."""
    import torch

    m, n, s = 30000, 96, 16
    X = synth.make_matrix_np(m, n, 1e4, seed=11)
    Xd = tensor.to_device_colmajor(X)
    Q1, R1, code, _ = tensor.factor(Xd, s, variant)
    assert code == 0
    tensor.set_gram_engine("fp64")
    small = tensor.workspace_size(m, n, s, variant)
    tensor.set_gram_engine("tensor")
    assert small < tensor.workspace_size(m, n, s, variant)
    ws = torch.empty(small, dtype=torch.uint8, device="cuda")
    Q2, R2, code2, _ = tensor.factor(Xd, s, variant, workspace=ws)
    assert code2 == 0
    check_against_oracle(X, s, variant, Q1, R1)
    check_against_oracle(X, s, variant, Q2, R2)
    Ro = R1.cpu().numpy()
    tol = 10 * n * oracle.kappa(Ro) * U64
    assert np.max(np.abs(Q1.cpu().numpy() - Q2.cpu().numpy())) <= tol


def test_store_path_reports_nonfinite(tensor):
    X = synth.make_matrix_np(5000, 48, 1e2, seed=5)
    X[4321, 20] = np.nan
    _, _, code, blk = tensor.factor(tensor.to_device_colmajor(X), 8, "bcgsi+p-2s")
    assert tensor.STATUS[code] == "nonfinite" and blk == 3


def test_store_path_step_by_step_handle(tensor):
    """The store lives in the handle's workspace across steps: a QRHandle fed one
    block per call gives the same bits as one factor call."""
    m, n, s = 9000, 80, 16
    X = synth.make_matrix_np(m, n, 1e4, seed=21)
    Xd = tensor.to_device_colmajor(X)
    Qf, Rf, code, _ = tensor.factor(Xd, s, "bcgsi+p-1s")
    assert code == 0
    h = tensor.QRHandle(m, n, s, "bcgsi+p-1s")
    for j in range(n // s):
        h.step(Xd[:, j * s:(j + 1) * s])
    h.finish()
    code, nfin, _ = h.sync()
    assert code == 0 and nfin == n
    assert np.array_equal(h.Q.cpu().numpy(), Qf.cpu().numpy())
    assert np.array_equal(h.R.cpu().numpy(), Rf.cpu().numpy())
    h.close()


@pytest.mark.parametrize("variant,s,precision", [("bcgsi+p-1s", 16, "fp64"), ("bcgsi+p-2s", 16, "fp64"),
                                                 ("bcgsi+1s", 16, "fp64"), ("bcgsi+p-2s", 32, "fp64"),
                                                 ("bcgsi+p-1s", 32, "fp32")])
def test_run_ahead_split_gives_the_step_by_step_bits(tensor, variant, s, precision):
    """From 2^17 rows a one-call factorization splits each next block of X into
    the store on a side stream while the current step's tail runs; the handle,
    fed one block per call, does not know the next block and splits it in its own
    step.  Both give the same bits, and the oracle's factors."""
    import torch

    m, n = 140000, 6 * s
    X = synth.make_matrix_np(m, n, 1e4, seed=s + 7)
    Xd = tensor.to_device_colmajor(X, dtype=torch.float32 if precision == "fp32" else None)
    Qf, Rf, code, _ = tensor.factor(Xd, s, variant)
    assert code == 0
    h = tensor.QRHandle(m, n, s, variant, precision)
    for j in range(n // s):
        h.step(Xd[:, j * s:(j + 1) * s])
    h.finish()
    code, nfin, _ = h.sync()
    assert code == 0 and nfin == n
    assert np.array_equal(h.Q.cpu().numpy(), Qf.cpu().numpy())
    assert np.array_equal(h.R.cpu().numpy(), Rf.cpu().numpy())
    if precision == "fp64":
        check_against_oracle(X, s, variant, Qf, Rf)


@pytest.mark.parametrize("variant", ["bcgsi+p-1s", "bcgsi+p-2s", "bcgsi+1s"])
def test_run_ahead_split_reports_nonfinite_in_its_own_block(tensor, variant):
    """A NaN in block 5 of X is found by the split run ahead during step 4; the
    failure is recorded where the block's own split would have recorded it, so
    the status names block 5 as it does step by step."""
    m, n, s = 140000, 112, 16
    X = synth.make_matrix_np(m, n, 1e3, seed=3)
    X[77777, 4 * s + 3] = np.nan
    Xd = tensor.to_device_colmajor(X)
    _, _, code, blk = tensor.factor(Xd, s, variant)
    h = tensor.QRHandle(m, n, s, variant)
    for j in range(n // s):
        h.step(Xd[:, j * s:(j + 1) * s])
    h.finish()
    hcode, _, hblk = h.sync()
    assert tensor.STATUS[code] == "nonfinite" and blk == 5
    assert (hcode, hblk) == (code, blk)
