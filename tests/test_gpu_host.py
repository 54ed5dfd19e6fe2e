"""End-to-end factorization from host memory (bcgs_qr_factor_host): the block
columns of X stream to the device while earlier blocks are factored and the
final blocks of Q stream back; the host results are bit-identical to the
device-resident call, for every variant, pinned or pageable host memory."""
import numpy as np
import pytest

import oracle
from paper_2507_21791_gb300 import synth

pytestmark = pytest.mark.gpu
VARIANTS = ["bcgsi+", "bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+", "bcgsi+1s"]


def host_colmajor(torch, m, n, dtype, pinned):
    return torch.empty((n, m), dtype=dtype, pin_memory=pinned).T


def run_host(cuda, X, s, variant, precision="fp64", pinned=True):
    import torch

    m, n = X.shape
    dt = torch.float32 if precision == "fp32" else torch.float64
    Xh = host_colmajor(torch, m, n, dt, pinned)
    Xh.copy_(torch.from_numpy(X))
    Qh = host_colmajor(torch, m, n, dt, pinned)
    Rh = host_colmajor(torch, n, n, torch.float64, pinned)
    Xd = cuda.empty_colmajor(m, n, dt)
    Qd = cuda.empty_colmajor(m, n, dt)
    Rd = cuda.empty_colmajor(n, n, torch.float64)
    ws = torch.empty(cuda.workspace_size(m, n, s, variant, precision), dtype=torch.uint8, device="cuda")
    cuda.factor_host_async(Xh, s, variant, precision, Qh, Rh, Xd, Qd, Rd, ws)
    code, blk = cuda.factor_status(ws)
    return Qh.numpy().copy(), Rh.numpy().copy(), code, blk


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m,n,s", [(20000, 64, 8), (40000, 96, 16), (3000, 30, 5)])
def test_host_path_is_bit_identical_to_the_device_path(cuda, variant, m, n, s):
    X = synth.make_matrix_np(m, n, 1e4, seed=m + n + s)
    Qh, Rh, code, _ = run_host(cuda, X, s, variant)
    assert code == 0
    Qd, Rd, code2, _ = cuda.factor(cuda.to_device_colmajor(X), s, variant)
    assert code2 == 0
    assert np.array_equal(Qh, Qd.cpu().numpy())
    assert np.array_equal(Rh, Rd.cpu().numpy())
    assert oracle.residual(X, Qh, Rh) <= 1e-13 and oracle.loo(Qh) <= 1e-12


def test_host_path_with_pageable_memory(cuda):
    X = synth.make_matrix_np(20000, 48, 1e3, seed=3)
    Qh, Rh, code, _ = run_host(cuda, X, 8, "bcgsi+p-1s", pinned=False)
    assert code == 0
    Qd, Rd, _, _ = cuda.factor(cuda.to_device_colmajor(X), 8, "bcgsi+p-1s")
    assert np.array_equal(Qh, Qd.cpu().numpy()) and np.array_equal(Rh, Rd.cpu().numpy())


def test_host_path_fp32_storage(cuda):
    import torch

    X = synth.make_matrix_np(30000, 64, 1e3, seed=4)
    Qh, Rh, code, _ = run_host(cuda, X, 16, "bcgsi+p-1s", precision="fp32")
    assert code == 0
    Qd, Rd, _, _ = cuda.factor(cuda.to_device_colmajor(X, dtype=torch.float32), 16, "bcgsi+p-1s")
    assert np.array_equal(Qh, Qd.cpu().numpy()) and np.array_equal(Rh, Rd.cpu().numpy())


def test_host_path_reports_breakdown(cuda):
    X = synth.make_matrix_np(5000, 32, 1e2, seed=9)
    X[:, 8:16] = 0.0
    _, _, code, blk = run_host(cuda, X, 8, "bcgsi+p-2s")
    assert cuda.STATUS[code] == "rank_deficient" and blk == 2


def test_host_path_from_several_threads(cuda):
    """The copy streams are shared per device: calls from several host threads
    (each on its own stream) still give each caller the bits of a serial call."""
    import threading

    import torch

    shapes = [(20000, 48, 8, "bcgsi+p-1s"), (30000, 64, 16, "bcgsi+p-2s"), (25000, 40, 8, "bcgs-pipi+"),
              (20000, 56, 8, "bcgsi+")]
    Xs = [synth.make_matrix_np(m, n, 1e3, seed=90 + i) for i, (m, n, s, v) in enumerate(shapes)]
    serial = [run_host(cuda, X, s, v)[:2] for X, (m, n, s, v) in zip(Xs, shapes)]
    out = [None] * len(shapes)

    def work(i):
        m, n, s, v = shapes[i]
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            Xh = host_colmajor(torch, m, n, torch.float64, True)
            Xh.copy_(torch.from_numpy(Xs[i]))
            Qh = host_colmajor(torch, m, n, torch.float64, True)
            Rh = host_colmajor(torch, n, n, torch.float64, True)
            Xd, Qd = cuda.empty_colmajor(m, n, torch.float64), cuda.empty_colmajor(m, n, torch.float64)
            Rd = cuda.empty_colmajor(n, n, torch.float64)
            ws = torch.empty(cuda.workspace_size(m, n, s, v), dtype=torch.uint8, device="cuda")
            cuda.factor_host_async(Xh, s, v, "fp64", Qh, Rh, Xd, Qd, Rd, ws, stream=st)
            code, _ = cuda.factor_status(ws, stream=st)
        out[i] = (Qh.numpy().copy(), Rh.numpy().copy(), code)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(shapes))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for (Qs, Rs), (Qt, Rt, code) in zip(serial, out):
        assert code == 0
        assert np.array_equal(Qs, Qt) and np.array_equal(Rs, Rt)
