"""Row-partitioned form (Sec. 3): each rank owns a block of rows of X, Q and U,
and the only global operations are the sums of the tall-skinny products (one
all-reduce per synchronization on the paper's cluster) and TSQR's reduction of
the R factors.

The library (bcgs_qr_factor_rows) runs every block step on the rank's own rows
and, at every synchronization, calls back for one all-gather of a buffer in the
rank's workspace; it adds the gathered copies in rank order with its own kernel.
This module supplies the argument marshalling and two all-gathers:

  * TorchAllGather: one torch.distributed all-gather (NCCL between GPUs,
    gloo between CPU processes), enqueued on the library's stream;
  * ThreadAllGather: P ranks emulated by P host threads on one GPU.  The
    exchange is host-mediated: each rank records an event when its buffer is
    ready, the threads meet at a barrier, and each rank's stream waits for the
    others' events and copies their buffers.  No device code waits on another
    rank, so nothing depends on the ranks' kernels running at the same time.
"""
from __future__ import annotations

import ctypes
import threading

from . import bcgs

ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.c_void_p)


def row_partition(m: int, nranks: int, rank: int) -> tuple[int, int]:
    """(first row, row count) of rank `rank`: whole 128-row blocks, as even as
    possible (bcgs_row_partition)."""
    lib = bcgs.load_library()
    r0, n = ctypes.c_int64(0), ctypes.c_int64(0)
    bcgs._check(lib.bcgs_row_partition(m, nranks, rank, ctypes.byref(r0), ctypes.byref(n)), "bcgs_row_partition")
    return r0.value, n.value


def workspace_size_rows(m_local: int, n: int, s: int, variant: str, nranks: int, precision: str = "fp64") -> int:
    lib = bcgs.load_library()
    out = ctypes.c_size_t(0)
    bcgs._check(lib.bcgs_qr_workspace_size_rows(m_local, n, s, bcgs.VARIANTS[variant], bcgs.PRECISIONS[precision],
                                                nranks, ctypes.byref(out)), "bcgs_qr_workspace_size_rows")
    return out.value


def _slices(ws, send: int, recv: int, nbytes: int, nranks: int):
    """The send and receive buffers as byte slices of the workspace tensor."""
    base = ws.data_ptr()
    so, ro = send - base, recv - base
    if not (0 <= so and so + nbytes <= ws.numel() and 0 <= ro and ro + nranks * nbytes <= ws.numel()):
        raise ValueError("all-gather buffers outside the workspace")
    return ws[so:so + nbytes], ws[ro:ro + nranks * nbytes]


def _stream_of(ptr):
    """The library's stream (a cudaStream_t; null is the legacy default stream)."""
    import torch

    return torch.cuda.ExternalStream(ptr) if ptr else torch.cuda.default_stream()


class TorchAllGather:
    """All-gather through torch.distributed (the default group unless one is
    given): NCCL for device workspaces, gloo for CPU tensors."""

    def __init__(self, group=None):
        self.group = group

    def world(self) -> tuple[int, int]:
        import torch.distributed as dist

        return dist.get_rank(self.group), dist.get_world_size(self.group)

    def __call__(self, ws, send: int, recv: int, nbytes: int, stream) -> int:
        import torch
        import torch.distributed as dist

        _, nranks = self.world()
        send_t, recv_t = _slices(ws, send, recv, nbytes, nranks)
        if ws.is_cuda:
            with torch.cuda.stream(_stream_of(stream)):
                dist.all_gather_into_tensor(recv_t, send_t, group=self.group)
        else:
            parts = list(recv_t.view(nranks, nbytes).unbind(0))
            dist.all_gather(parts, send_t, group=self.group)
        return 0


class ThreadAllGather:
    """P ranks on one GPU, one host thread each (see the module docstring).
    `member(rank)` is the all-gather of one rank."""

    def __init__(self, nranks: int):
        self.nranks = nranks
        self.barrier = threading.Barrier(nranks)
        self.ready = [None] * nranks
        self.done = [None] * nranks

    def member(self, rank: int):
        def call(ws, send: int, recv: int, nbytes: int, stream) -> int:
            import torch

            st = _stream_of(stream)
            send_t, recv_t = _slices(ws, send, recv, nbytes, self.nranks)
            ev = torch.cuda.Event()
            ev.record(st)
            self.ready[rank] = (send_t, ev)
            self.barrier.wait()
            with torch.cuda.stream(st):
                for r in range(self.nranks):
                    src, evr = self.ready[r]
                    st.wait_event(evr)
                    recv_t[r * nbytes:(r + 1) * nbytes].copy_(src)
            done = torch.cuda.Event()
            done.record(st)
            self.done[rank] = done
            self.barrier.wait()
            # a rank overwrites its send buffer only after every peer copied it
            for r in range(self.nranks):
                if r != rank:
                    st.wait_event(self.done[r])
            self.barrier.wait()
            return 0

        return call


def factor_rows(X_local, s: int, variant: str, rank: int, nranks: int, allgather=None, precision: str | None = None,
                Q=None, R=None, workspace=None, stream=None, check_status: bool = True):
    """This rank's part of the row-partitioned factorization: X_local is the
    rank's block of rows (column-major device tensor).  `allgather(ws, send,
    recv, nbytes, stream) -> 0` is called at every synchronization (not needed
    for nranks = 1).  Returns (Q_local, R, status_code, fail_block); with
    check_status False the call only enqueues (status code and block are None)."""
    import torch

    lib = bcgs.load_library()
    if precision is None:
        precision = "fp32" if X_local.dtype == torch.float32 else "fp64"
    m, n = X_local.shape
    dt = torch.float32 if precision == "fp32" else torch.float64
    if Q is None:
        Q = bcgs.empty_colmajor(m, n, dt, X_local.device)
    if R is None:
        R = bcgs.empty_colmajor(n, n, torch.float64, X_local.device)
    if workspace is None:
        workspace = bcgs._workspace(workspace_size_rows(m, n, s, variant, nranks, precision), X_local.device)
    errors = []

    def trampoline(ctx, send, recv, nbytes, strm):
        try:
            return int(allgather(workspace, send, recv, nbytes, strm))
        except Exception as e:  # reported as BCGS_ERR_COMM by the library
            errors.append(e)
            return 1

    cb = ALLGATHER_FN(trampoline) if allgather is not None else None
    sp = bcgs._stream_ptr(stream)
    rc = lib.bcgs_qr_factor_rows(m, n, s, bcgs.VARIANTS[variant], bcgs.PRECISIONS[precision], X_local.data_ptr(),
                                 bcgs._colmajor_ld(X_local), Q.data_ptr(), bcgs._colmajor_ld(Q), R.data_ptr(),
                                 bcgs._colmajor_ld(R), workspace.data_ptr(), workspace.numel(), sp, rank, nranks,
                                 ctypes.cast(cb, ctypes.c_void_p) if cb is not None else None, None)
    if errors:
        raise RuntimeError(f"all-gather failed: {errors[0]!r}")
    bcgs._check(rc, "bcgs_qr_factor_rows")
    if not check_status:
        return Q, R, None, None
    blk = ctypes.c_int32(0)
    code = lib.bcgs_qr_factor_status(workspace.data_ptr(), sp, ctypes.byref(blk))
    return Q, R, code, blk.value
