"""Host-side logic of the serving loop (no GPU): admission by HBM budget, FIFO
order, the closed loop per basis (block j+1 only after call j completed), the
finish call after the last block, and the latency report.  A fake backend
completes each call after a fixed number of polls."""
import itertools

import pytest

from paper_2507_21791_gb300.serving import Request, Server, final_blocks_after, make_requests, percentile


class FakeBackend:
    def __init__(self, polls_per_call=3, bytes_per_col=1.0):
        self.polls = polls_per_call
        self.bpc = bytes_per_col
        self.log = []
        self.open_now = 0
        self.max_open = 0

    def bytes_for(self, req):
        return self.bpc * req.m * req.n

    # lazy = delayed normalization (BCGSI+P-2S), eager = BCGSI+
    def final_blocks(self, req, steps):
        return final_blocks_after("bcgsi+" if req.finalize == "eager" else "bcgsi+p-2s", steps)

    def needs_finish(self, req):
        return req.finalize != "eager"

    def open(self, req):
        self.open_now += 1
        self.max_open = max(self.max_open, self.open_now)
        self.log.append(("open", req.rid))
        return {"left": 0}

    def issue_step(self, req, j):
        assert req.slot["left"] == 0, "a call was issued while the previous one was in flight"
        self.log.append(("step", req.rid, j))
        req.slot["left"] = self.polls

    def issue_finish(self, req):
        assert req.slot["left"] == 0
        self.log.append(("finish", req.rid))
        req.slot["left"] = self.polls

    def done(self, req):
        req.slot["left"] -= 1
        return req.slot["left"] <= 0

    def close(self, req):
        self.open_now -= 1
        self.log.append(("close", req.rid))
        return 0


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4
        return self.t


def make(n_req, m=100, n=8, s=2, gap=0.0):
    return [Request(rid=i, arrival=i * gap, m=m, n=n, s=s) for i in range(n_req)]


def test_every_request_completes_in_order_of_its_blocks():
    be = FakeBackend()
    srv = Server(be, budget_bytes=1e9, clock=FakeClock())
    rep = srv.run(make(5), duration=10.0)
    assert rep["requests_done"] == 5 and rep["failed"] == 0
    for rid in range(5):
        ev = [e for e in be.log if e[1] == rid]
        assert ev[0] == ("open", rid)
        assert [e[2] for e in ev if e[0] == "step"] == [0, 1, 2, 3]
        assert ev[-2] == ("finish", rid) and ev[-1] == ("close", rid)
    # 4 blocks + finish = 5 calls per request
    assert rep["calls_done"] == 25


def test_budget_is_never_exceeded_and_admission_is_fifo():
    be = FakeBackend()
    per = 100 * 8
    srv = Server(be, budget_bytes=2.5 * per, clock=FakeClock())
    rep = srv.run(make(7), duration=10.0)
    assert rep["requests_done"] == 7
    assert srv.peak_reserved <= 2.5 * per
    assert be.max_open == 2
    opens = [e[1] for e in be.log if e[0] == "open"]
    assert opens == sorted(opens)


def test_oversized_request_is_rejected_not_queued():
    be = FakeBackend()
    srv = Server(be, budget_bytes=1000.0, clock=FakeClock())
    reqs = make(2) + [Request(rid=9, arrival=0.0, m=10_000, n=8, s=2)]
    rep = srv.run(reqs, duration=10.0)
    assert rep["requests_rejected"] == 1 and srv.rejected[0].rid == 9


def test_requests_overlap_when_memory_allows():
    be = FakeBackend(polls_per_call=5)
    srv = Server(be, budget_bytes=1e9, clock=FakeClock())
    srv.run(make(6), duration=10.0)
    assert srv.max_active == 6
    # steps of different bases interleave
    steps = [e[1] for e in be.log if e[0] == "step"]
    assert any(a != b for a, b in itertools.pairwise(steps[:6]))


def test_run_stops_admitting_at_duration_and_drains():
    be = FakeBackend(polls_per_call=50)
    clock = FakeClock()
    srv = Server(be, budget_bytes=1e9, clock=clock)
    reqs = make(100, gap=0.01)
    rep = srv.run(reqs, duration=0.05)
    assert rep["requests_unserved"] > 0
    assert not srv.active  # drained
    assert rep["requests_done"] + rep["requests_unserved"] == 100


def test_percentile():
    xs = list(range(101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile([], 50) is None


def test_block_size_tuner_keys_and_persistence(tmp_path):
    from paper_2507_21791_gb300.batched import BlockSizeTuner, alg_bytes

    t = BlockSizeTuner(path=str(tmp_path / "t.json"))
    assert t.key(4096, 64) == "12:64" and t.key(5000, 64) == "12:64" and t.key(6000, 64) == "13:64"
    t.table["12:64"] = (8, "fp64")
    t.save()
    t2 = BlockSizeTuner(path=str(tmp_path / "t.json"))
    assert t2.pick(4096, 64) == 8 and t2.pick_engine(4096, 64) == "fp64"  # cached, no GPU needed
    # a table saved with s only reads as the default engine
    (tmp_path / "old.json").write_text('{"13:32": 16}')
    assert BlockSizeTuner(path=str(tmp_path / "old.json")).choose(8192, 32) == (16, "auto")
    assert alg_bytes(1000, 64, 8, "bcgsi+") > alg_bytes(1000, 64, 8, "bcgsi+p-2s") > alg_bytes(1000, 64, 8, "bcgsi+p-1s")


def test_final_blocks_follow_delayed_normalization():
    assert [final_blocks_after("bcgsi+p-1s", k) for k in range(5)] == [0, 1, 1, 2, 3]
    assert [final_blocks_after("bcgsi+p-2s", k) for k in range(5)] == [0, 1, 1, 2, 3]
    assert [final_blocks_after("bcgs-pipi+", k) for k in range(5)] == [0, 1, 2, 3, 4]
    assert [final_blocks_after("bcgsi+", k) for k in range(5)] == [0, 1, 2, 3, 4]


def test_eager_requests_skip_the_finish_call_and_finalize_each_block_in_its_call():
    be = FakeBackend(polls_per_call=3)
    reqs = make(4, n=8, s=2)
    for r in reqs[::2]:
        r.finalize = "eager"
    rep = Server(be, budget_bytes=1e9, clock=FakeClock()).run(reqs, duration=1.0)
    assert rep["requests_done"] == 4 and set(rep["by_finalize"]) == {"eager", "lazy"}
    for r in reqs:
        finishes = [e for e in be.log if e[0] == "finish" and e[1] == r.rid]
        assert len(finishes) == (0 if r.finalize == "eager" else 1)
        assert r.n_final == r.q and len(r.final_latencies) == r.q
        if r.finalize == "eager":
            # each block is final when its own call completes
            assert r.final_latencies == pytest.approx(r.call_latencies)
        else:
            # block 1 final with its own call (TSQR), blocks 2..q-1 one call later, the last at finish
            assert len(r.call_latencies) == r.q + 1
            assert r.final_latencies[0] == pytest.approx(r.call_latencies[0])
            for b in range(1, r.q):
                assert r.final_latencies[b] > r.call_latencies[b]


def test_eager_fraction_does_not_move_arrivals():
    meta = [(100, 8, 2)]
    a = make_requests(50.0, 1.0, meta, seed=3, eager_frac=0.0)
    b = make_requests(50.0, 1.0, meta, seed=3, eager_frac=0.5)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(r.finalize == "lazy" for r in a)
    assert 0 < sum(r.finalize == "eager" for r in b) < len(b)
