"""A whole factorization captured into one CUDA graph: the library enqueues
only stream-ordered work (no host synchronization, no allocation), so one
capture of bcgs_qr_factor replays the factorization of whatever the captured X
buffer holds.  Checks: a replay gives the eager call's bits, a replay after new
data is copied into X gives that data's factorization (against the oracle), on
the small configuration (FP64-pipe kernels) and on the digit store path."""
import numpy as np
import pytest

import oracle
from conftest import loo_gate
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,s", [(10000, 64, 8), (65536, 64, 16)])
@pytest.mark.parametrize("variant", ["bcgsi+p-1s", "bcgsi+p-2s", "bcgsi+", "bcgs-pipi+", "bcgsi+1s"])
def test_graph_replay_is_the_eager_factorization(cuda, m, n, s, variant):
    import torch

    from paper_2507_21791_gb300 import bcgs

    X1 = synth.make_matrix_np(m, n, 1e4, seed=m + n)
    X2 = synth.make_matrix_np(m, n, 1e3, seed=m + n + 1)
    Xd = cuda.to_device_colmajor(X1)
    Q = bcgs.empty_colmajor(m, n, torch.float64, Xd.device)
    R = bcgs.empty_colmajor(n, n, torch.float64, Xd.device)
    ws = torch.empty(bcgs.workspace_size(m, n, s, variant), dtype=torch.uint8, device=Xd.device)
    bcgs.factor_async(Xd, s, variant, "fp64", Q, R, ws)
    torch.cuda.synchronize()
    assert bcgs.factor_status(ws)[0] == 0
    Qe, Re = Q.cpu().numpy(), R.cpu().numpy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bcgs.factor_async(Xd, s, variant, "fp64", Q, R, ws)
    Q.zero_()
    R.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert bcgs.factor_status(ws)[0] == 0
    assert np.array_equal(Q.cpu().numpy(), Qe) and np.array_equal(R.cpu().numpy(), Re)
    # new data in the captured buffer
    Xd.copy_(cuda.to_device_colmajor(X2))
    g.replay()
    torch.cuda.synchronize()
    assert bcgs.factor_status(ws)[0] == 0
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro = oracle.factor(X2, s, variant)
    k = oracle.kappa(Ro)
    tol = 10 * n * k * U64
    assert oracle.residual(X2, Qh, Rh) <= 1e-13
    assert oracle.loo(Qh) <= loo_gate(variant, n, k, oracle.loo(Qo))
    assert np.linalg.norm(Rh - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Qh - Qo)) <= tol
