"""The batched and served forms on the GPU.

Batched: one bcgs_qr_factor_batched call (and its CUDA-graph replay) over uneven
problems gives, for every problem, the same bits as bcgs_qr_factor alone, and
every problem's Q and R agree with the oracle's entry by entry.  Served: each
basis's Q and R are the same alone and in the mix (bitwise: the reduction order
depends only on the problem's shape), and every admitted request agrees with
the oracle.  Oracle agreement is the forward bound of the variant tests:
    residual <= 1e-13, LOO <= 1e-12,
    ||R - R_oracle||_F / ||R_oracle||_F <= 10 n kappa u,  max |Q - Q_oracle| <= 10 n kappa u.
"""
import numpy as np
import pytest

import oracle
from paper_2507_21791_gb300 import synth

U64 = np.finfo(np.float64).eps / 2
pytestmark = pytest.mark.gpu


def check_oracle(X, Q, R, s, variant):
    """The gates and the forward bound against the oracle's factorization of X."""
    n = X.shape[1]
    Qo, Ro = oracle.factor(X, s, variant)
    tol = 10 * n * oracle.kappa(Ro) * U64
    assert oracle.residual(X, Q, R) <= 1e-13
    assert oracle.loo(Q) <= 1e-12
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= tol
    assert np.max(np.abs(Q - Qo)) <= tol


def test_batched_matches_single_and_graph_replay(cuda):
    import torch

    from paper_2507_21791_gb300.batched import Batch

    rng = np.random.default_rng(3)
    Xs, ss, Xh = [], [], []
    for i in range(12):
        m = int(2 ** rng.uniform(12, 15))
        n = int(rng.choice([32, 64]))
        s = int(rng.choice([4, 8, 16]))
        X = synth.make_matrix_np(m, n, 10 ** rng.uniform(1, 6), seed=100 + i)
        Xh.append(X)
        Xs.append(cuda.to_device_colmajor(X))
        ss.append(s)
    b = Batch(Xs, ss, variant="bcgsi+p-2s")
    b.enqueue()
    codes, _ = b.status()
    assert codes == [0] * len(Xs)
    first = [(q.clone(), r.clone()) for q, r in zip(b.Qs, b.Rs)]
    for i, (X, s) in enumerate(zip(Xs, ss)):
        Q, R, code, _ = cuda.factor(X, s, "bcgsi+p-2s")
        assert code == 0
        assert torch.equal(Q, b.Qs[i]) and torch.equal(R, b.Rs[i])
        check_oracle(Xh[i], b.Qs[i].cpu().numpy(), b.Rs[i].cpu().numpy(), s, "bcgsi+p-2s")
    for q in b.Qs:
        q.zero_()
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    codes, _ = b.status()
    assert codes == [0] * len(Xs)
    for (q0, r0), q, r in zip(first, b.Qs, b.Rs):
        assert torch.equal(q0, q) and torch.equal(r0, r)


def test_batched_per_problem_engines(cuda):
    """Problems that name their own engine (FP64 pipe, tensor cores from the
    threshold, tensor cores always) in one batch: each gives the bits of
    bcgs_qr_factor under that engine alone, and agrees with the oracle; the
    global option is left as it was."""
    import torch

    from paper_2507_21791_gb300.batched import Batch

    shapes = [(5000, 32, 8, "tensor"), (5000, 32, 8, "fp64"), (20000, 64, 16, "fp64"),
              (20000, 64, 16, "auto"), (9000, 64, 16, "tensor"), (3000, 32, 4, "tensor")]
    Xh = [synth.make_matrix_np(m, n, 1e4, seed=900 + i) for i, (m, n, _, _) in enumerate(shapes)]
    Xs = [cuda.to_device_colmajor(X) for X in Xh]
    ss = [s for _, _, s, _ in shapes]
    engines = [e for _, _, _, e in shapes]
    before = cuda.get_gram_engine()
    b = Batch(Xs, ss, variant="bcgsi+p-2s", engines=engines)
    b.enqueue()
    codes, _ = b.status()
    assert codes == [0] * len(Xs)
    assert cuda.get_gram_engine() == before
    for i, (X, s, eng) in enumerate(zip(Xs, ss, engines)):
        cuda.set_gram_engine(eng)
        try:
            Q, R, code, _ = cuda.factor(X, s, "bcgsi+p-2s")
        finally:
            cuda.set_gram_engine(before)
        assert code == 0
        assert torch.equal(Q, b.Qs[i]) and torch.equal(R, b.Rs[i])
        check_oracle(Xh[i], b.Qs[i].cpu().numpy(), b.Rs[i].cpu().numpy(), s, "bcgsi+p-2s")


def test_batched_store_path_every_variant_against_oracle(cuda):
    """Instances of m >= 16384 rows, n = 128 and s in {8, 16}: the batch runs the
    digit-store kernels (tensor-core Gram and projection).  Mixed variants in one
    batch; each result is bitwise the single call's and within the oracle bound."""
    import torch

    from paper_2507_21791_gb300.batched import Batch

    rng = np.random.default_rng(11)
    plan = [("bcgsi+p-1s", 16, 1e4), ("bcgsi+p-1s", 8, 1e5), ("bcgs-pipi+", 16, 1e4),
            ("bcgsi+p-2s", 16, 1e7), ("bcgsi+p-2s", 8, 1e3), ("bcgsi+", 16, 1e6)]
    Xs, Xh, ss, vs = [], [], [], []
    for i, (v, s, kappa) in enumerate(plan):
        m = int(2 ** rng.uniform(14, 16.2))
        X = synth.make_matrix_np(m, 128, kappa, seed=300 + i)
        Xh.append(X)
        Xs.append(cuda.to_device_colmajor(X))
        ss.append(s)
        vs.append(v)
    b = Batch(Xs, ss, variants=vs)
    b.enqueue()
    codes, _ = b.status()
    assert codes == [0] * len(Xs)
    for i in range(len(Xs)):
        Q, R, code, _ = cuda.factor(Xs[i], ss[i], vs[i])
        assert code == 0
        assert torch.equal(Q, b.Qs[i]) and torch.equal(R, b.Rs[i])
        check_oracle(Xh[i], b.Qs[i].cpu().numpy(), b.Rs[i].cpu().numpy(), ss[i], vs[i])


def _serve(cuda, sources, meta, rids, arrivals, budget=8e9, modes=None):
    from paper_2507_21791_gb300.serving import GpuBackend, Request, Server

    be = GpuBackend(sources, variant="bcgsi+p-2s", nstreams=8)
    srv = Server(be, budget_bytes=budget)
    modes = modes or ["lazy"] * len(rids)
    reqs = [Request(rid=r, arrival=a, m=meta[r][0], n=meta[r][1], s=meta[r][2], source=r, finalize=f)
            for r, a, f in zip(rids, arrivals, modes)]
    rep = srv.run(reqs, duration=120.0)
    return {r.rid: r for r in srv.done}, rep


def test_served_results_are_the_same_alone_and_in_the_mix(cuda):
    import torch

    from paper_2507_21791_gb300.serving import draw_sources

    sources, meta = draw_sources(10, seed=5, m_exp=(12, 15), p_range=(2, 6))
    targets = [0, 3, 7]
    alone = {}
    for r in targets:
        done, rep = _serve(cuda, sources, meta, [r], [0.0])
        assert rep["failed"] == 0
        alone[r] = done[r].result
    done, rep = _serve(cuda, sources, meta, list(range(10)), [0.0] * 10)
    assert rep["requests_done"] == 10 and rep["failed"] == 0 and rep["max_active"] > 1
    for r in targets:
        Qa, Ra = alone[r]
        Qm, Rm = done[r].result
        assert torch.equal(Qa, Qm) and torch.equal(Ra, Rm)
    for r, req in done.items():
        m, n, s = meta[r]
        X = sources[r][:m, :n].cpu().numpy()
        check_oracle(X, req.result[0].cpu().numpy(), req.result[1].cpu().numpy(), s, "bcgsi+p-2s")


def test_server_respects_the_budget(cuda):
    from paper_2507_21791_gb300.serving import draw_sources

    sources, meta = draw_sources(8, seed=6, m_exp=(13, 15), p_range=(2, 4))
    from paper_2507_21791_gb300.serving import GpuBackend

    be = GpuBackend(sources, variant="bcgsi+p-2s")
    per = max(be.bytes_for(type("R", (), {"m": m, "n": n, "s": s})) for m, n, s in meta)
    done, rep = _serve(cuda, sources, meta, list(range(8)), [0.0] * 8, budget=2.2 * per)
    assert rep["requests_done"] == 8
    assert rep["peak_reserved_gb"] * 1e9 <= 2.2 * per


def test_eager_and_lazy_finalize_give_their_variants_results(cuda):
    """Eager requests run BCGSI+ (every block final after its own call), lazy ones
    BCGSI+P-2S (delayed normalization); each served result is bitwise the same
    as that variant's factorization alone."""
    import torch

    from paper_2507_21791_gb300.serving import draw_sources

    sources, meta = draw_sources(6, seed=8, m_exp=(12, 15), p_range=(2, 6))
    modes = ["eager", "lazy"] * 3
    done, rep = _serve(cuda, sources, meta, list(range(6)), [0.0] * 6, modes=modes)
    assert rep["requests_done"] == 6 and rep["failed"] == 0
    assert set(rep["by_finalize"]) == {"eager", "lazy"}
    for r, req in done.items():
        m, n, s = meta[r]
        variant = "bcgsi+" if modes[r] == "eager" else "bcgsi+p-2s"
        Q, R, code, _ = cuda.factor(sources[r][:m, :n], s, variant)
        assert code == 0
        assert torch.equal(Q, req.result[0]) and torch.equal(R, req.result[1])
        assert len(req.final_latencies) == req.q
        check_oracle(sources[r][:m, :n].cpu().numpy(), Q.cpu().numpy(), R.cpu().numpy(), s, variant)


def test_served_store_path_against_oracle(cuda):
    """Bases of 2^14 .. 2^16 rows (the digit-store kernels) served together; every
    result within the oracle bound."""
    from paper_2507_21791_gb300.serving import draw_sources

    sources, meta = draw_sources(5, seed=9, m_exp=(14, 16), p_range=(2, 5), s_choices=(8, 16),
                                 kappa_exp=(1, 6))
    done, rep = _serve(cuda, sources, meta, list(range(5)), [0.0] * 5)
    assert rep["requests_done"] == 5 and rep["failed"] == 0
    for r, req in done.items():
        m, n, s = meta[r]
        X = sources[r][:m, :n].cpu().numpy()
        check_oracle(X, req.result[0].cpu().numpy(), req.result[1].cpu().numpy(), s, "bcgsi+p-2s")
