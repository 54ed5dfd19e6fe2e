"""Serving form: a request loop for block-by-block orthogonalization.

A request is a basis of m rows that grows by q blocks of s columns, delivered
one block per call (the shape of an s-step / block Krylov basis).  The server:

  * admits requests first come, first served, while their device memory
    (Q, R and the factorization workspace) fits in an HBM budget;
  * keeps each admitted basis's Q, R and workspace resident on the device
    between its block steps (a QRHandle of the C ABI);
  * interleaves the steps of all admitted bases (continuous batching): each
    basis runs on a stream of a pool, so steps of different bases overlap on
    the GPU, and a new request starts as soon as memory frees up;
  * closes the loop per basis: block j+1 is issued when the call for block j
    has completed (BCGSI+P-1S/-2S finalize block j-1 at step j, eq. (1));
  * finalizes lazily or eagerly per request: "lazy" keeps the delayed
    normalization of BCGSI+P-1S/-2S (one synchronization per block, block j
    final one call later), "eager" runs the variant of the same stability range
    whose blocks are final after their own call (BCGS-PIPI+ for 1S, BCGSI+ for
    2S: one more synchronization per block, Table 1);
  * records per-call latency (issue -> completion), per-block finalization
    latency (issue of the block's call -> completion of the call that makes it
    final) and per-request latency (arrival -> last block final), as p50 / p99,
    overall and per finalize mode.

The scheduling logic talks to a backend with four operations (open, issue,
done, close), so it can be exercised on the CPU with a fake backend.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    arrival: float          # seconds, on the server clock
    m: int
    n: int                  # final number of columns (q blocks of s)
    s: int
    source: int = 0         # index of the pre-generated basis that supplies the blocks
    finalize: str = "lazy"  # "lazy" (delayed normalization) or "eager"
    # runtime state
    admitted: float | None = None
    finished: float | None = None
    next_block: int = 0     # blocks issued so far
    finishing: bool = False
    issued_at: float | None = None
    call_latencies: list = field(default_factory=list)
    block_issued: list = field(default_factory=list)    # issue time of each block's call
    final_latencies: list = field(default_factory=list)  # per block: issue -> final
    n_final: int = 0
    status: int = 0
    slot: object = None     # backend resources

    @property
    def q(self):
        return self.n // self.s


def percentile(xs, p):
    if not xs:
        return None
    xs = sorted(xs)
    k = (len(xs) - 1) * p / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


class Server:
    def __init__(self, backend, budget_bytes: float = 120e9, clock=time.perf_counter):
        self.backend = backend
        self.budget = budget_bytes
        self.clock = clock
        self.reserved = 0.0
        self.peak_reserved = 0.0
        self.queue: collections.deque[Request] = collections.deque()
        self.active: list[Request] = []
        self.done: list[Request] = []
        self.rejected: list[Request] = []
        self.max_active = 0
        self._t0 = None

    def now(self):
        return self.clock() - self._t0

    def submit(self, req: Request):
        need = self.backend.bytes_for(req)
        if need > self.budget:
            req.status = -1
            self.rejected.append(req)
            return
        self.queue.append(req)

    def _admit(self):
        while self.queue:
            req = self.queue[0]
            need = self.backend.bytes_for(req)
            if self.reserved + need > self.budget:
                break
            self.queue.popleft()
            self.reserved += need
            self.peak_reserved = max(self.peak_reserved, self.reserved)
            req.slot = self.backend.open(req)
            req.admitted = self.now()
            self.active.append(req)
        self.max_active = max(self.max_active, len(self.active))

    def _finalized(self, req, nblocks, t):
        while req.n_final < nblocks:
            req.final_latencies.append(t - req.block_issued[req.n_final])
            req.n_final += 1

    def _close(self, req):
        req.status = self.backend.close(req)
        req.finished = self.now()
        self.reserved -= self.backend.bytes_for(req)
        self.done.append(req)

    def _progress(self):
        still = []
        for req in self.active:
            if req.issued_at is not None:
                if not self.backend.done(req):
                    still.append(req)
                    continue
                t = self.now()
                req.call_latencies.append(t - req.issued_at)
                req.issued_at = None
                if req.finishing:
                    self._finalized(req, req.q, t)
                    self._close(req)
                    continue
                self._finalized(req, self.backend.final_blocks(req, req.next_block), t)
            # issue the next call of this basis (its latency counts from here)
            t_issue = self.now()
            if req.next_block < req.q:
                req.block_issued.append(t_issue)
                self.backend.issue_step(req, req.next_block)
                req.next_block += 1
            elif self.backend.needs_finish(req):
                self.backend.issue_finish(req)
                req.finishing = True
            else:  # eager: every block is final after its own call
                self._close(req)
                continue
            req.issued_at = t_issue
            still.append(req)
        self.active = still

    def run(self, requests, duration: float, drain: bool = True, idle_sleep: float = 0.0):
        """Serve `requests` (sorted by arrival) for `duration` seconds of wall
        time, then (if drain) finish the admitted ones without admitting more."""
        self._t0 = self.clock()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        while True:
            t = self.now()
            if t >= duration:
                break
            while pending and pending[0].arrival <= t:
                self.submit(pending.popleft())
            self._admit()
            self._progress()
            if not self.active and not self.queue and not pending:
                break
            if idle_sleep:
                time.sleep(idle_sleep)
        self.unserved = len(pending) + len(self.queue)
        if drain:
            while self.active:
                self._progress()
        return self.report(self.now())

    @staticmethod
    def _latencies(done):
        calls = [x for r in done for x in r.call_latencies]
        finals = [x for r in done for x in r.final_latencies]
        reqs = [r.finished - r.arrival for r in done]
        return {"requests_done": len(done),
                "call_latency_ms": {"p50": _ms(percentile(calls, 50)), "p99": _ms(percentile(calls, 99))},
                "block_final_latency_ms": {"p50": _ms(percentile(finals, 50)), "p99": _ms(percentile(finals, 99))},
                "request_latency_ms": {"p50": _ms(percentile(reqs, 50)), "p99": _ms(percentile(reqs, 99))}}

    def report(self, elapsed):
        """Latency percentiles and throughput over `elapsed` seconds (arrival
        window plus drain)."""
        calls = [x for r in self.done for x in r.call_latencies]
        finals = [x for r in self.done for x in r.final_latencies]
        reqs = [r.finished - r.arrival for r in self.done]
        served = [r.finished - r.admitted for r in self.done]
        modes = sorted({r.finalize for r in self.done})
        return {
            "by_finalize": {mo: self._latencies([r for r in self.done if r.finalize == mo]) for mo in modes},
            "block_final_latency_ms": {"p50": _ms(percentile(finals, 50)), "p99": _ms(percentile(finals, 99))},
            "requests_done": len(self.done), "requests_rejected": len(self.rejected),
            "requests_unserved": getattr(self, "unserved", 0),
            "calls_done": len(calls),
            "call_latency_ms": {"p50": _ms(percentile(calls, 50)), "p99": _ms(percentile(calls, 99))},
            "request_latency_ms": {"p50": _ms(percentile(reqs, 50)), "p99": _ms(percentile(reqs, 99))},
            "service_latency_ms": {"p50": _ms(percentile(served, 50)), "p99": _ms(percentile(served, 99))},
            "throughput_req_per_s": len(self.done) / elapsed if elapsed else None,
            "elapsed_s": elapsed,
            "max_active": self.max_active, "peak_reserved_gb": self.peak_reserved / 1e9,
            "budget_gb": self.budget / 1e9,
            "failed": sum(1 for r in self.done if r.status != 0),
        }


def _ms(x):
    return None if x is None else 1e3 * x


# the variant of the same stability range (Table 1) whose blocks are final
# after their own step, for the "eager" finalize mode
EAGER = {"bcgsi+p-1s": "bcgs-pipi+", "bcgsi+p-2s": "bcgsi+", "bcgs-pipi+": "bcgs-pipi+", "bcgsi+": "bcgsi+",
         "bcgsi+1s": "bcgs-pipi+"}
DELAYED = ("bcgsi+p-1s", "bcgsi+p-2s", "bcgsi+1s")


def final_blocks_after(variant: str, steps: int) -> int:
    """Blocks of Q final after `steps` steps (before the finish call): delayed
    normalization (Sec. 2) keeps the newest block provisional under
    BCGSI+P-1S/-2S and BCGSI+1s, except that block 1 comes final from TSQR."""
    if variant in DELAYED:
        return max(steps - 1, 1) if steps >= 1 else 0
    return steps


class GpuBackend:
    """Backend over the C ABI: one QRHandle per admitted basis, streams from a pool."""

    def __init__(self, sources, variant="bcgsi+p-2s", nstreams=32, device="cuda"):
        import torch

        from . import bcgs

        self.torch, self.bcgs = torch, bcgs
        self.sources = sources      # list of column-major device tensors (m_i x n_i)
        self.variant = variant
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(nstreams)]
        self._next_stream = 0
        self._bytes = {}

    def variant_for(self, req: Request) -> str:
        return EAGER[self.variant] if getattr(req, "finalize", "lazy") == "eager" else self.variant

    def final_blocks(self, req: Request, steps: int) -> int:
        return final_blocks_after(self.variant_for(req), steps)

    def needs_finish(self, req: Request) -> bool:
        return self.variant_for(req) in DELAYED

    def bytes_for(self, req: Request) -> float:
        v = self.variant_for(req)
        key = (req.m, req.n, req.s, v)
        if key not in self._bytes:
            ws = self.bcgs.workspace_size(req.m, req.n, req.s, v)
            self._bytes[key] = ws + 8.0 * (req.m * req.n + req.n * req.n)
        return self._bytes[key]

    def open(self, req: Request):
        stream = self.streams[self._next_stream % len(self.streams)]
        self._next_stream += 1
        with self.torch.cuda.stream(stream):
            h = self.bcgs.QRHandle(req.m, req.n, req.s, self.variant_for(req), device=self.device,
                                   stream=stream)
        return {"h": h, "stream": stream, "ev": None}

    def _record(self, req):
        ev = self.torch.cuda.Event()
        ev.record(req.slot["stream"])
        req.slot["ev"] = ev

    def issue_step(self, req: Request, j: int):
        X = self.sources[req.source]
        req.slot["h"].step(X[:req.m, j * req.s:(j + 1) * req.s])
        self._record(req)

    def issue_finish(self, req: Request):
        req.slot["h"].finish()
        self._record(req)

    def done(self, req: Request) -> bool:
        ev = req.slot["ev"]
        return ev is None or ev.query()

    def close(self, req: Request) -> int:
        code, _, _ = req.slot["h"].sync()
        req.result = (req.slot["h"].Q, req.slot["h"].R)
        req.slot["h"].close()
        req.slot = None
        return code


def make_requests(rate: float, duration: float, sources_meta, seed: int = 0, eager_frac: float = 0.0):
    """Poisson arrivals at `rate` per second over `duration` seconds; request k
    takes its shape and blocks from source k mod len(sources_meta) (a pool of
    pre-generated bases stands in for per-request generation) and asks for
    eager finalization with probability eager_frac."""
    import numpy as np

    rng = np.random.default_rng(seed)
    rng_mode = np.random.default_rng(seed + 7919)  # arrivals do not depend on eager_frac
    t, out, k = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        src = k % len(sources_meta)
        m, n, s = sources_meta[src]
        mode = "eager" if rng_mode.random() < eager_frac else "lazy"
        out.append(Request(rid=k, arrival=t, m=m, n=n, s=s, source=src, finalize=mode))
        k += 1
    return out


def draw_sources(count: int, seed: int = 0, m_exp=(14, 20), p_range=(4, 32), s_choices=(4, 8, 16),
                 kappa_exp=(1, 8), device="cuda"):
    """Pre-generated bases: m = 2^U(m_exp), q ~ U{p_range} blocks of s columns,
    kappa = 10^U(kappa_exp); X = U diag(sigma) V^T on the device."""
    import numpy as np

    from . import synth

    rng = np.random.default_rng(seed)
    meta, xs = [], []
    for i in range(count):
        m = synth.log_uniform_int(rng, *m_exp)
        q = int(rng.integers(p_range[0], p_range[1] + 1))
        s = int(rng.choice(s_choices))
        n = q * s
        m = max(m, n)
        kappa = 10.0 ** rng.uniform(*kappa_exp)
        xs.append(synth.make_matrix_torch(m, n, kappa, seed=seed * 1000 + i, device=device))
        meta.append((m, n, s))
    return xs, meta
