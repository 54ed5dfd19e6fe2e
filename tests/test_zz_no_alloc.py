"""bcgs_gram_noalloc, the Gram product for callers that cannot allocate device
memory or lend the library a workspace (for instance a host framework that owns
every device allocation through its own pool, where a cudaMalloc behind its back
fragments the pool and may synchronize the device).  The entry point keeps its
partial sums in a fixed array inside the library, so the tests check that its
result matches the workspace-based bcgs_gram within the Gram tolerance of
test_gpu_kernels.py, on two calls in a row (the second call reuses the array the
first one left behind), that it meets the oracle's Gram within each engine's
derived bound, that a non-finite input comes back as NaN and not as what an
earlier call left in the array, and that requests beyond the array are refused.

This file is named to be collected last: a run that stops at its first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu


def chunking(m):
    cr = -(-m // 304)
    cr = -(-cr // 16) * 16
    cr = max(cr, 64)
    return cr, -(-m // cr)


def call_noalloc(cuda, A, B):
    import torch

    lib = cuda.load_library()
    m, ka = A.shape
    kb = B.shape[1]
    C = cuda.empty_colmajor(ka, kb, torch.float64, A.device)
    rc = lib.bcgs_gram_noalloc(m, ka, kb, A.data_ptr(), m, B.data_ptr(), m, C.data_ptr(), ka,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, cuda.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def test_noalloc_gram_matches_workspace_gram_on_two_calls(cuda):
    cases = [(200003, 64, 32, 1), (70001, 17, 9, 2)]
    for m, ka, kb, seed in cases:
        rng = np.random.default_rng(seed)
        A = rng.standard_normal((m, ka))
        B = rng.standard_normal((m, kb)) * np.exp(rng.standard_normal((m, 1)))
        Ad, Bd = cuda.to_device_colmajor(A), cuda.to_device_colmajor(B)
        C_ws = cuda.gram(Ad, Bd).cpu().numpy()   # existing entry point, caller workspace
        C_na = call_noalloc(cuda, Ad, Bd)         # no workspace, static partials
        cr, nc = chunking(m)
        bound = 2 * (cr + nc + 2) * U64 * (np.abs(A).T @ np.abs(B))
        assert np.all(np.abs(C_na - C_ws) <= bound + 1e-300)
        # same partition and kernels, so the reduction order is the same as well
        assert np.array_equal(C_na, C_ws)


def tensor_bound(A, B, m):
    """Derived bound of the digit engine (tests/test_gpu_tensor_gram.py): dropped
    digit pairs and truncation, then one rounding per chunk partial and the
    ordered sum of the partials."""
    _, nc = chunking(m)
    amax_a, amax_b = np.abs(A).max(axis=0), np.abs(B).max(axis=0)
    return (m * np.outer(amax_a, amax_b) * 2.0 ** -57.1
            + 2 * (nc + 2) * U64 * (np.abs(A).T @ np.abs(B)))


def test_noalloc_gram_matches_oracle_on_both_engines(cuda):
    """m >= 16384 runs the tensor-core engine, m < 16384 the FP64 pipe (the
    default engine choice); both are compared with the oracle's A^T B entry by
    entry, and the FP64-pipe case bitwise with bcgs_gram."""
    import oracle

    for m, ka, kb, seed in [(200003, 64, 32, 3), (5000, 40, 12, 4)]:
        rng = np.random.default_rng(seed)
        A = rng.standard_normal((m, ka))
        B = rng.standard_normal((m, kb)) * np.exp(rng.standard_normal((m, 1)))
        Ad, Bd = cuda.to_device_colmajor(A), cuda.to_device_colmajor(B)
        Co = oracle.gram([A], [B])
        for _ in range(2):
            C_na = call_noalloc(cuda, Ad, Bd)
            if m >= 16384:
                assert np.all(np.abs(C_na - Co) <= tensor_bound(A, B, m))
            else:
                cr, nc = chunking(m)
                bound = 2 * (cr + nc + 2) * U64 * (np.abs(A).T @ np.abs(B))
                assert np.all(np.abs(C_na - Co) <= bound + 1e-300)
                assert np.array_equal(C_na, cuda.gram(Ad, Bd).cpu().numpy())


def test_noalloc_gram_nonfinite_input_gives_nan_not_stale_sums(cuda):
    """A clean call fills the array; the next call, with an Inf in one column of
    A, must return NaN in that column's row of C (the tensor engine's CTAs that
    see the column write NaN partials), and a clean call after it is right again."""
    m, ka, kb = 70001, 48, 16
    rng = np.random.default_rng(5)
    A = rng.standard_normal((m, ka))
    B = rng.standard_normal((m, kb))
    Ad, Bd = cuda.to_device_colmajor(A), cuda.to_device_colmajor(B)
    C_clean = call_noalloc(cuda, Ad, Bd)
    assert np.all(np.isfinite(C_clean))
    A_bad = A.copy()
    A_bad[12345, 7] = np.inf
    C_bad = call_noalloc(cuda, cuda.to_device_colmajor(A_bad), Bd)
    assert np.all(np.isnan(C_bad[7, :]))
    C_again = call_noalloc(cuda, Ad, Bd)
    assert np.array_equal(C_again, C_clean)


def test_noalloc_gram_refuses_sizes_beyond_its_array(cuda):
    import torch

    lib = cuda.load_library()
    m, ka, kb = 2 ** 20, 256, 64   # 304 chunks x 16384 outputs > 2^20 doubles
    A = torch.zeros((ka, m), dtype=torch.float64, device="cuda").T
    B = torch.zeros((kb, m), dtype=torch.float64, device="cuda").T
    C = torch.zeros((kb, ka), dtype=torch.float64, device="cuda").T
    rc = lib.bcgs_gram_noalloc(m, ka, kb, A.data_ptr(), m, B.data_ptr(), m, C.data_ptr(), ka,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert cuda.STATUS[rc] == "workspace"
