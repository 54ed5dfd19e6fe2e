"""bcgs_gram_noalloc, the Gram product for callers that cannot allocate device
memory or lend the library a workspace (for instance a host framework that owns
every device allocation through its own pool, where a cudaMalloc behind its back
fragments the pool and may synchronize the device).  The entry point keeps its
partial sums in a fixed array inside the library, so the test checks that its
result matches the workspace-based bcgs_gram within the Gram tolerance of
test_gpu_kernels.py, on two calls in a row (the second call reuses the array the
first one left behind), and that requests beyond the array are refused.

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
