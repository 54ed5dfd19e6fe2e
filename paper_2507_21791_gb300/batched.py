"""Batched form: many independent, uneven factorizations in one launch.

`Batch` binds caller-side buffers (PyTorch) for a list of problems and enqueues
them with one bcgs_qr_factor_batched call; the library runs them concurrently
on internal streams forked from the caller's stream.  `Batch.capture()` records
that call into one CUDA graph, so every later `replay()` launches the whole batch
at once.  `BlockSizeTuner` is the autotuner: it picks the block size s and the product
engine per instance shape (m bucket, n) by timing the candidates on a
representative instance and caches the choice.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
from dataclasses import dataclass, field

from . import bcgs


class BlockSizeTuner:
    """Choose the block size s (from `candidates`) and the product engine (from
    `engines`) per instance shape (round(log2 m), n) by measured time.

    Any s dividing n gives a QR of X; s only changes the speed (fewer, larger
    synchronizations and intraorthogonalizations) and, slightly, the rounding.
    The engine ("fp64": FP64 pipe; "tensor": exact digit products on the tensor
    cores, with the digit store of Q) changes the speed and the rounding within
    the same bounds.  A choice, once made, is kept (and can be saved), so
    repeated batches of the same shapes use the same (s, engine) and give the
    same bits.  `pick` returns s; `pick_engine` the engine chosen with it.
    """

    def __init__(self, candidates=(4, 8, 16), variant="bcgsi+p-2s", path: str | None = None,
                 engines=("auto",)):
        self.candidates = tuple(candidates)
        self.engines = tuple(engines)
        self.variant = variant
        self.path = path
        self.table: dict[str, tuple[int, str]] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                for k, v in json.load(f).items():
                    self.table[k] = (int(v), "auto") if isinstance(v, int) else (int(v[0]), str(v[1]))

    @staticmethod
    def key(m: int, n: int) -> str:
        return f"{int(round(math.log2(max(m, 1))))}:{n}"

    def save(self):
        if self.path:
            with open(self.path, "w") as f:
                json.dump({k: list(v) for k, v in self.table.items()}, f, indent=1, sort_keys=True)

    def pick(self, m: int, n: int, device="cuda") -> int:
        return self.choose(m, n, device)[0]

    def pick_engine(self, m: int, n: int, device="cuda") -> str:
        return self.choose(m, n, device)[1]

    def choose(self, m: int, n: int, device="cuda") -> tuple[int, str]:
        k = self.key(m, n)
        if k in self.table:
            return self.table[k]
        import torch

        from . import synth

        mr = max(2 ** int(round(math.log2(max(m, 1)))), n)
        X = synth.make_matrix_torch(mr, n, 1e4, seed=12345, device=device)
        best, best_ms = None, float("inf")
        saved = bcgs.get_gram_engine()
        try:
            for eng in self.engines:
                bcgs.set_gram_engine(eng)
                for s in self.candidates:
                    if n % s != 0 or s > n:
                        continue
                    Q = bcgs.empty_colmajor(mr, n, torch.float64, device)
                    R = bcgs.empty_colmajor(n, n, torch.float64, device)
                    ws = torch.empty(bcgs.workspace_size(mr, n, s, self.variant), dtype=torch.uint8,
                                     device=device)
                    bcgs.factor_async(X, s, self.variant, "fp64", Q, R, ws)  # warm-up
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(3):
                        bcgs.factor_async(X, s, self.variant, "fp64", Q, R, ws)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / 3
                    if ms < best_ms:
                        best, best_ms = (s, eng), ms
        finally:
            bcgs.set_gram_engine(saved)
        self.table[k] = best
        return best


@dataclass
class Batch:
    """Caller-side buffers and the problem table of one batch."""
    Xs: list
    s_list: list
    variant: str = "bcgsi+p-2s"
    Qs: list = field(default_factory=list)
    Rs: list = field(default_factory=list)
    variants: list | None = None  # per-problem variants (default: `variant` for all)
    engines: list | None = None   # per-problem engines ("fp64", "auto", "tensor"; default: the option)

    def __post_init__(self):
        import torch

        self.lib = bcgs.load_library()
        n_items = len(self.Xs)
        self.probs = (bcgs.Problem * max(n_items, 1))()
        for i, (X, s) in enumerate(zip(self.Xs, self.s_list)):
            m, n = X.shape
            prec = "fp32" if X.dtype == torch.float32 else "fp64"
            Q = bcgs.empty_colmajor(m, n, X.dtype, X.device)
            R = bcgs.empty_colmajor(n, n, torch.float64, X.device)
            self.Qs.append(Q)
            self.Rs.append(R)
            v = self.variants[i] if self.variants is not None else self.variant
            eng = bcgs.PROBLEM_ENGINES[self.engines[i]] if self.engines is not None else 0
            self.probs[i] = bcgs.Problem(m, n, s, bcgs.VARIANTS[v], bcgs.PRECISIONS[prec],
                                         X.data_ptr(), bcgs._colmajor_ld(X), Q.data_ptr(),
                                         bcgs._colmajor_ld(Q), R.data_ptr(), bcgs._colmajor_ld(R), eng)
        nb = ctypes.c_size_t(0)
        bcgs._check(self.lib.bcgs_qr_batched_workspace_size(n_items, self.probs, ctypes.byref(nb)),
                    "bcgs_qr_batched_workspace_size")
        dev = self.Xs[0].device if n_items else "cuda"
        self.ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=dev)
        self.graph = None

    def __len__(self):
        return len(self.Xs)

    def enqueue(self, stream=None):
        bcgs._check(self.lib.bcgs_qr_factor_batched(len(self), self.probs, self.ws.data_ptr(),
                                                    self.ws.numel(), bcgs._stream_ptr(stream)),
                    "bcgs_qr_factor_batched")

    def capture(self):
        """Record one batched call into a CUDA graph (after an eager warm-up call)."""
        import torch

        self.enqueue()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.enqueue()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def status(self, stream=None):
        codes = (ctypes.c_int32 * max(len(self), 1))()
        blocks = (ctypes.c_int32 * max(len(self), 1))()
        self.lib.bcgs_qr_batched_status(len(self), self.ws.data_ptr(), bcgs._stream_ptr(stream),
                                        codes, blocks)
        return list(codes)[:len(self)], list(blocks)[:len(self)]


def alg_bytes(m: int, n: int, s: int, variant: str, b: int = 8) -> float:
    """Algorithmic HBM bytes of one factorization: passes over the previous basis
    (1 per block for BCGSI+P-1S, 2 for -2S, 4 for BCGSI+ and BCGS-PIPI+) plus the
    block passes."""
    q = n // s
    qpasses = {"bcgsi+p-1s": 1, "bcgsi+p-2s": 2, "bcgsi+": 4, "bcgs-pipi+": 4, "bcgsi+1s": 1}[variant]
    bpasses = {"bcgsi+p-1s": 5, "bcgsi+p-2s": 8, "bcgsi+": 10, "bcgs-pipi+": 6, "bcgsi+1s": 5}[variant]
    return b * m * s * q * (q - 1) / 2 * qpasses + bpasses * b * m * n
