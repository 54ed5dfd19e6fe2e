"""Row-partitioned form (Sec. 3) on one GPU: P ranks emulated by P host threads,
each factoring its block of rows through bcgs_qr_factor_rows; the all-gather is
host-mediated (ThreadAllGather: events, a host barrier and device copies), so no
device code waits on another rank.

Checks: the ranks' rows of Q, stacked, and the replicated R agree with the
oracle's factorization of the whole matrix (the forward bound of the variant
tests), R is the same bits on every rank and on a second run, and a rank's
non-finite rows make every rank report a failure.  One rank through the same
entry point gives bcgs_qr_factor's bits.
"""
import threading

import numpy as np
import pytest

import oracle
from conftest import loo_gate
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu


def run_ranks(cuda, X, s, variant, P, engine="auto"):
    """Factor X over P emulated ranks; returns (Q stacked, [R per rank], [codes], [blocks])."""
    import torch

    from paper_2507_21791_gb300 import rows

    m, n = X.shape
    comm = rows.ThreadAllGather(P)
    parts = [rows.row_partition(m, P, r) for r in range(P)]
    slabs = [cuda.to_device_colmajor(X[r0:r0 + mr]) for r0, mr in parts]
    out = [None] * P
    errors = []

    def work(r):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                Q, R, code, blk = rows.factor_rows(slabs[r], s, variant, r, P, comm.member(r), stream=stream)
                stream.synchronize()
            out[r] = (Q.cpu().numpy(), R.cpu().numpy(), code, blk)
        except Exception as e:  # surfaced by the test below
            errors.append(e)
            comm.barrier.abort()

    cuda.set_gram_engine(engine)
    try:
        threads = [threading.Thread(target=work, args=(r,)) for r in range(P)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=600)
    finally:
        cuda.set_gram_engine("auto")
    assert not errors, errors
    Q = np.vstack([o[0] for o in out])
    return Q, [o[1] for o in out], [o[2] for o in out], [o[3] for o in out]


def check(X, Q, R, s, variant):
    n = X.shape[1]
    Qo, Ro = oracle.factor(X, s, variant)
    k = oracle.kappa(Ro)
    tol = 10 * n * k * U64
    assert oracle.residual(X, Q, R) <= 1e-13
    assert oracle.loo(Q) <= loo_gate(variant, n, k, oracle.loo(Qo))
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Q - Qo)) <= tol


@pytest.mark.parametrize("variant", ["bcgsi+p-1s", "bcgsi+p-2s", "bcgsi+1s", "bcgs-pipi+", "bcgsi+"])
@pytest.mark.parametrize("P", [2, 3])
def test_emulated_ranks_match_the_oracle(cuda, variant, P):
    """m = 70001 rows (slabs above 16384 rows: the digit-store kernels), n = 64, s = 16."""
    X = synth.make_matrix_np(70001, 64, 1e4, seed=400 + P)
    Q, Rs, codes, _ = run_ranks(cuda, X, 16, variant, P)
    assert codes == [0] * P
    for R in Rs[1:]:
        assert np.array_equal(R, Rs[0])  # replicated: the same bits on every rank
    check(X, Q, Rs[0], 16, variant)


@pytest.mark.parametrize("engine", ["fp64", "tensor"])
def test_emulated_ranks_small_slabs_and_ragged_block(cuda, engine):
    """Slabs of a few thousand rows, n = 44 (a ragged last block of 4), both engines."""
    X = synth.make_matrix_np(9000, 44, 1e3, seed=411)
    for variant in ("bcgsi+p-1s", "bcgsi+p-2s"):
        Q, Rs, codes, _ = run_ranks(cuda, X, 8, variant, 4, engine=engine)
        assert codes == [0] * 4
        assert all(np.array_equal(R, Rs[0]) for R in Rs)
        check(X, Q, Rs[0], 8, variant)


def test_emulated_ranks_are_deterministic(cuda):
    X = synth.make_matrix_np(40000, 48, 1e5, seed=412)
    Q1, R1, _, _ = run_ranks(cuda, X, 16, "bcgsi+p-1s", 2)
    Q2, R2, _, _ = run_ranks(cuda, X, 16, "bcgsi+p-1s", 2)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1[0], R2[0])


def test_one_rank_is_the_single_gpu_factorization(cuda):
    from paper_2507_21791_gb300 import rows

    X = synth.make_matrix_np(30000, 64, 1e4, seed=413)
    Xd = cuda.to_device_colmajor(X)
    Q1, R1, c1, _ = cuda.factor(Xd, 16, "bcgsi+p-1s")
    Q2, R2, c2, _ = rows.factor_rows(Xd, 16, "bcgsi+p-1s", 0, 1)
    assert c1 == 0 and c2 == 0
    assert np.array_equal(Q1.cpu().numpy(), Q2.cpu().numpy()) and np.array_equal(R1.cpu().numpy(), R2.cpu().numpy())


def test_a_ranks_nonfinite_rows_fail_every_rank(cuda):
    """A NaN in rank 1's rows of block 3: rank 1 flags it, the NaN it then sends
    makes every other rank fail too, at a block index within one of block 3."""
    X = synth.make_matrix_np(60000, 48, 1e2, seed=414)
    X[45000, 20] = np.nan  # rank 1 of 2 owns the rows from 30080 on
    _, _, codes, blocks = run_ranks(cuda, X, 8, "bcgsi+p-1s", 2)
    assert all(c != 0 for c in codes)
    assert all(2 <= b <= 4 for b in blocks)
