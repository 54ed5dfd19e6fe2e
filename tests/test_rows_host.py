"""Row-partitioned form (Sec. 3) on the CPU: the row partition and the argument
checks of the C ABI (host-only, no GPU), and, on two gloo ranks, the
partitioned schedule itself.

The gloo test restates Alg. 2 (BCGSI+P-1S) over row slabs with the oracle's
primitives: every Gram is this rank's rows' product, all-gathered through the
package's TorchAllGather and added in rank order, and TSQR factors the local
rows, gathers and stacks the local R factors and factors the stack, as the
library does.  The result must be the oracle's factorization of the whole
matrix (within the forward bound of the variant tests), with the same R on both
ranks, bit for bit.
"""
import ctypes
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT, ensure_library


def lib():
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    return bcgs.load_library()


@pytest.mark.parametrize("m,P", [(1, 1), (127, 2), (128, 2), (1000, 3), (70001, 8), (300, 5), (4194304, 8)])
def test_row_partition_covers_the_rows_in_whole_blocks(m, P):
    from paper_2507_21791_gb300 import rows

    parts = [rows.row_partition(m, P, r) for r in range(P)]
    assert parts[0][0] == 0
    for (r0, n0), (r1, _) in zip(parts, parts[1:]):
        assert r0 + n0 == r1                      # contiguous, in rank order
    assert parts[-1][0] + parts[-1][1] == m       # every row once
    for r0, n in parts:
        assert n == 0 or r0 % 128 == 0            # whole 128-row blocks (a rank may get none)
    sizes = [-(-n // 128) for _, n in parts]      # blocks per rank
    assert max(sizes) - min(sizes) <= 1           # as even as possible


def test_row_partition_rejects_bad_arguments():
    L = lib()
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    for args in [(0, 2, 0), (100, 0, 0), (100, 2, 2), (100, 2, -1)]:
        assert L.bcgs_row_partition(*args, ctypes.byref(a), ctypes.byref(b)) == 1
    assert L.bcgs_row_partition(100, 2, 0, None, ctypes.byref(b)) == 1


def test_factor_rows_argument_checks_without_a_gpu():
    """Rejected before anything is enqueued (fake, never dereferenced pointers)."""
    L = lib()
    X, Q, R, W = 1 << 40, 1 << 41, 1 << 42, 1 << 43
    cb = ctypes.cast(ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p)(lambda *a: 0), ctypes.c_void_p)
    f = L.bcgs_qr_factor_rows
    assert f(1000, 16, 8, 1, 0, X, 1000, Q, 1000, R, 16, W, 1 << 30, None, 0, 2, None, None) == 1  # no callback
    assert f(1000, 16, 8, 1, 0, X, 1000, Q, 1000, R, 16, W, 1 << 30, None, 2, 2, cb, None) == 1    # rank >= nranks
    assert f(1000, 16, 8, 1, 0, X, 1000, Q, 1000, R, 16, W, 1 << 30, None, 0, 0, cb, None) == 1    # nranks < 1
    assert f(5, 16, 8, 1, 0, X, 5, Q, 5, R, 16, W, 1 << 30, None, 0, 2, cb, None) == 1             # m_local < s
    assert f(1000, 16, 8, 1, 0, X, 1000, X + 64, 1000, R, 16, W, 1 << 30, None, 0, 2, cb, None) == 1  # X/Q overlap
    assert f(1000, 16, 8, 7, 0, X, 1000, Q, 1000, R, 16, W, 1 << 30, None, 0, 2, cb, None) == 1    # variant
    # a valid call with a too small workspace stops at the workspace check
    assert f(1000, 16, 8, 1, 0, X, 1000, Q, 1000, R, 16, W, 1024, None, 0, 2, cb, None) == 5


def test_workspace_size_rows():
    L = lib()
    out = ctypes.c_size_t(0)
    # a slab may have fewer rows than n (it needs s for its local TSQR)
    assert L.bcgs_qr_workspace_size_rows(100, 256, 16, 1, 0, 4, ctypes.byref(out)) == 0
    assert L.bcgs_qr_workspace_size_rows(100, 256, 16, 1, 0, 1, ctypes.byref(out)) == 1  # one rank: m >= n
    assert L.bcgs_qr_workspace_size_rows(8, 256, 16, 1, 0, 4, ctypes.byref(out)) == 1    # m_local < s
    one, four = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert L.bcgs_qr_workspace_size_rows(10000, 64, 8, 1, 0, 1, ctypes.byref(one)) == 0
    assert L.bcgs_qr_workspace_size_rows(10000, 64, 8, 1, 0, 4, ctypes.byref(four)) == 0
    plain = ctypes.c_size_t(0)
    assert L.bcgs_qr_workspace_size(10000, 64, 8, 1, 0, ctypes.byref(plain)) == 0
    assert one.value == plain.value
    # the gathered copies of the Gram (4 x 64 x 16 doubles) and a local TSQR block
    assert four.value >= one.value + 4 * 64 * 16 * 8 + 10000 * 8 * 8


WORKER = r"""
import hashlib, json
import numpy as np
import torch
import torch.distributed as dist
import oracle
from paper_2507_21791_gb300 import rows, synth

dist.init_process_group("gloo")
rank, P = dist.get_rank(), dist.get_world_size()
ag = rows.TorchAllGather()
ws = torch.zeros(1 << 22, dtype=torch.uint8)

def gather(A):
    # the library's exchange: every rank's copy, rank after rank
    A = np.asarray(A, dtype=np.float64)
    b = torch.frombuffer(bytearray(A.tobytes()), dtype=torch.uint8)
    nb = b.numel()
    ws[:nb] = b
    assert ag(ws, ws.data_ptr(), ws.data_ptr() + nb, nb, None) == 0
    return [np.frombuffer(ws[nb * (1 + r):nb * (2 + r)].numpy().tobytes(), dtype=np.float64).reshape(A.shape)
            for r in range(P)]

def allsum(A):
    parts = gather(A)
    out = parts[0].copy()
    for p in parts[1:]:
        out = out + p            # rank order
    return out

def tsqr_rows(A):
    # local Householder QR, the stacked local R factors factored again, and
    # this rank's rows of Q = local Q times its block of the stack's Q
    Ql, Rl = oracle.householder_qr(A)
    Qs, R = oracle.householder_qr(np.vstack(gather(Rl)))
    w = A.shape[1]
    return Ql @ Qs[rank * w:(rank + 1) * w], R

def one_sync_rows(X, s):
    # Alg. 2 over row slabs: Grams summed over the ranks, TSQR over the ranks
    m, n = X.shape
    q = n // s
    Q = np.zeros((m, n)); R = np.zeros((n, n))
    blk = lambda k: slice((k - 1) * s, k * s)
    upto = lambda k: slice(0, k * s)
    Xb = lambda k: X[:, blk(k)]
    Q1, R11 = tsqr_rows(Xb(1))
    Q[:, blk(1)], R[blk(1), blk(1)] = Q1, R11
    G = allsum(oracle.gram([Q1, Xb(2)], [Xb(2)]))
    S12, T2 = G[:s], G[s:]
    S22 = oracle.chol(T2 - S12.T @ S12, 2)
    U = oracle.project_normalize(Xb(2), Q1, S12, S22)
    G = allsum(oracle.gram([Q1, U], [U, Xb(3)]))
    Y12, Z1, Om, Pk = G[:s, :s], G[:s, s:], G[s:, :s], G[s:, s:]
    T = allsum(oracle.gram([Xb(3)], [Xb(3)]))
    Ykk = oracle.chol(Om - Y12.T @ Y12, 2)
    Q[:, blk(2)] = oracle.project_normalize(U, Q1, Y12, Ykk)
    R[blk(1), blk(2)] = S12 + Y12 @ S22
    R[blk(2), blk(2)] = Ykk @ S22
    Yprev, Zprev = Y12, Z1
    for k in range(2, q):
        S = np.vstack([Zprev, oracle.delayed_projection(Ykk, Pk, Yprev, Zprev)])
        Sd = oracle.chol(T - S.T @ S, k + 1)
        Qk = Q[:, upto(k)]
        U = oracle.project_normalize(Xb(k + 1), Qk, S, Sd)
        if k < q - 1:
            G = allsum(oracle.gram([Qk, U], [U, Xb(k + 2)]))
            Y, Z, Om, Pk = G[:k * s, :s], G[:k * s, s:], G[k * s:, :s], G[k * s:, s:]
            T = allsum(oracle.gram([Xb(k + 2)], [Xb(k + 2)]))
        else:
            G = allsum(oracle.gram([Qk, U], [U]))
            Y, Om = G[:k * s], G[k * s:]
            Z = Pk = T = None
        Yd = oracle.chol(Om - Y.T @ Y, k + 1)
        Q[:, blk(k + 1)] = oracle.project_normalize(U, Qk, Y, Yd)
        R[upto(k), blk(k + 1)] = S + Y @ Sd
        R[blk(k + 1), blk(k + 1)] = Yd @ Sd
        Ykk, Yprev, Zprev = Yd, Y, Z
    return Q, R

m, n, s, kappa = 3001, 48, 8, 1e4
X = synth.make_matrix_np(m, n, kappa, seed=5)
r0, mr = rows.row_partition(m, P, rank)
Ql, R = one_sync_rows(X[r0:r0 + mr], s)
Qo, Ro = oracle.factor(X, s, "bcgsi+p-1s")
dq = float(np.abs(Ql - Qo[r0:r0 + mr]).max())
dr = float(np.linalg.norm(R - Ro) / np.linalg.norm(Ro))
print(json.dumps({"rank": rank, "rows": [r0, mr], "dq": dq, "dr": dr, "kappa": float(oracle.kappa(Ro)),
                  "r_hash": hashlib.sha256(R.tobytes()).hexdigest()}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_the_oracle_factorization():
    ensure_library()
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda o: o["rank"])
    assert outs[0]["rows"][0] == 0 and outs[0]["rows"][1] + outs[1]["rows"][1] == 3001
    u = np.finfo(np.float64).eps / 2
    for o in outs:
        tol = 10 * 48 * o["kappa"] * u
        assert o["dq"] <= tol and o["dr"] <= tol
    assert outs[0]["r_hash"] == outs[1]["r_hash"]  # the replicated R: the same bits on both ranks
