"""A ragged last block (n mod s != 0) on the GPU, through the C ABI, against the
oracle's reading: the full blocks are factored by the variant, its delayed
block finalized, and the ragged block takes one step of the variant of the same
stability range that finalizes at once (BCGS-PIPI+ for 1S and PIPI+, BCGSI+ for
BCGSI+ and 2S); n < s is TSQR alone."""
import numpy as np
import pytest

import oracle
from conftest import loo_gate
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu
VARIANTS = ["bcgsi+", "bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+", "bcgsi+1s"]
# (m, n, s): ragged 4, 4 (store Grams for the full blocks), 5, n < s, 8 (past a
# 128-column tile), 6 with s = 32, a single ragged column
SHAPES = [(10000, 60, 8), (20000, 100, 16), (5000, 21, 8), (3000, 5, 8), (40000, 136, 16),
          (30000, 70, 32), (2000, 9, 8)]


def check(X, s, variant, Q, R):
    n = X.shape[1]
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro = oracle.factor(X, s, variant)
    assert oracle.residual(X, Qh, Rh) <= 1e-13
    assert oracle.loo(Qh) <= loo_gate(variant, n, oracle.kappa(Ro), oracle.loo(Qo))
    tol = 10 * n * oracle.kappa(Ro) * U64
    assert np.linalg.norm(Rh - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Qh - Qo)) <= tol
    assert np.array_equal(np.tril(Rh, -1), np.zeros_like(Rh)) and np.all(np.diag(Rh) > 0)


@pytest.mark.parametrize("engine", ["auto", "tensor", "fp64"])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m,n,s", SHAPES)
def test_ragged_matches_the_oracle(cuda, engine, variant, m, n, s):
    cuda.set_gram_engine(engine)
    try:
        X = synth.make_matrix_np(m, n, 1e4, seed=m + 7 * n + s)
        Q, R, code, _ = cuda.factor(cuda.to_device_colmajor(X), s, variant)
        assert code == 0
        check(X, s, variant, Q, R)
    finally:
        cuda.set_gram_engine("auto")


@pytest.mark.parametrize("variant", VARIANTS)
def test_ragged_step_interface(cuda, variant):
    """Blocks of 8, 8 and 5 columns through bcgs_qr_step: the same bits as one
    factor call; the ragged step leaves every column final."""
    m, n, s = 20000, 21, 8
    X = synth.make_matrix_np(m, n, 1e3, seed=33)
    Xd = cuda.to_device_colmajor(X)
    Qf, Rf, code, _ = cuda.factor(Xd, s, variant)
    assert code == 0
    h = cuda.QRHandle(m, n, s, variant)
    finals = []
    for j in range(3):
        h.step(Xd[:, j * s:min((j + 1) * s, n)])
        code, nf, _ = h.sync()
        assert code == 0
        finals.append(nf)
    assert finals == ([8, 16, 21] if variant in ("bcgsi+", "bcgs-pipi+") else [8, 8, 21])
    with pytest.raises(cuda.BCGSError):
        h.step(Xd[:, :s])
    h.finish()
    code, nf, _ = h.sync()
    assert code == 0 and nf == n
    assert np.array_equal(h.Q.cpu().numpy(), Qf.cpu().numpy())
    assert np.array_equal(h.R.cpu().numpy(), Rf.cpu().numpy())
    h.close()


def test_ragged_host_path_fp32_and_batched(cuda):
    import torch

    m, n, s = 30000, 45, 16
    X = synth.make_matrix_np(m, n, 1e3, seed=44)
    Xd = cuda.to_device_colmajor(X)
    Qd, Rd, code, _ = cuda.factor(Xd, s, "bcgsi+p-1s")
    assert code == 0
    # host path: bit-identical
    Xh = torch.empty((n, m), dtype=torch.float64, pin_memory=True).T
    Xh.copy_(torch.from_numpy(X))
    Qh = torch.empty((n, m), dtype=torch.float64, pin_memory=True).T
    Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True).T
    ws = torch.empty(cuda.workspace_size(m, n, s, "bcgsi+p-1s"), dtype=torch.uint8, device="cuda")
    cuda.factor_host_async(Xh, s, "bcgsi+p-1s", "fp64", Qh, Rh, cuda.empty_colmajor(m, n, torch.float64),
                           cuda.empty_colmajor(m, n, torch.float64), cuda.empty_colmajor(n, n, torch.float64), ws)
    assert cuda.factor_status(ws)[0] == 0
    assert np.array_equal(Qh.numpy(), Qd.cpu().numpy()) and np.array_equal(Rh.numpy(), Rd.cpu().numpy())
    # FP32 storage
    Qf, Rf, code, _ = cuda.factor(cuda.to_device_colmajor(X, dtype=torch.float32), s, "bcgsi+p-2s")
    assert code == 0
    Q32 = Qf.double().cpu().numpy()
    assert oracle.loo(Q32) <= 1e-6 and oracle.residual(X, Q32, Rf.cpu().numpy()) <= 1e-6
    # batched: the same bits as alone
    from paper_2507_21791_gb300.batched import Batch

    b = Batch([Xd, Xd[:10000]], [s, 8], variant="bcgsi+p-1s")
    b.enqueue()
    codes, _ = b.status()
    assert codes == [0, 0]
    assert torch.equal(b.Qs[0], Qd) and torch.equal(b.Rs[0], Rd)
    Q2, R2, code, _ = cuda.factor(Xd[:10000], 8, "bcgsi+p-1s")
    assert code == 0 and torch.equal(b.Qs[1], Q2) and torch.equal(b.Rs[1], R2)
