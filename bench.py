#!/usr/bin/env python
"""Benchmark of the GB300 BCGS QR library.

Workload (one step = one whole factorization, i.e. every block step of the hot
path over one synthetic matrix): single FP64 economic QR of X = U diag(sigma) V^T,
m = 2^22 rows, n = 256 columns, block size s = 16 (q = 16 blocks),
kappa = 1e5 (inside every variant's O(u)-loss-of-orthogonality range, so the
variants are compared at equal loss of orthogonality), BCGSI+P-1S timed; BCGSI+,
BCGSI+P-2S and BCGS-PIPI+ (Alg. 1) are timed the same way for the speedup.

value  = algorithmic HBM bytes of the fused BCGSI+P-1S schedule per step / time
         (GB/s); bytes per step = 8 m s q(q-1)/2 (each block reads the previous
         basis once) + 5 * 8 m n (X twice, U written and read, Q written).
e2e    = the same metric through bcgs_qr_factor_host with pinned host buffers:
         the host->device copy of X and the device->host copy of Q and R are
         inside the timed region (overlapped with the factorization, block by
         block).
X (8.6 GB) and Q (8.6 GB) are far larger than the 129 MB L2, so no L2 flush is
needed between steps.

`--impl reference` times the CPU oracle (the method's plain FP64 restatement)
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BCGSI+P-1S HBM GB/s & speedup vs BCGSI+ at equal loss-of-orth.; p99 latency"
M, N, S, KAPPA = 2 ** 22, 256, 16, 1e5
WORKLOAD = "single FP64 QR m=2^22 n=256 s=16 (q=16) BCGSI+P-1S, X=U diag(sigma) V^T kappa=1e5"
FP64_PEAK_TFLOPS = 1.25  # GB300 FP64 rate of the profiling recipe's table (nominal)
# DRAM traffic of a kernel relative to its algorithmic bytes, from one ncu capture
# of the current kernel on a smaller case (the committed ncu summaries); traffic
# grows with the rows processed, so a full launch moves this ratio times its
# algorithmic bytes.  A kernel that changed since its capture has no entry
# (traffic reported as null).
# nominal HBM3e bandwidth of a GB300 (the spec sheet); the roofline's peak is the
# measured copy bandwidth, the spec fraction is reported beside it
HBM_SPEC_GBS = 7900.0

TRAFFIC_RATIO = {
    # FP64-pipe Gram, ncu capture at m = 524288, 256 x 32 outputs:
    # (1.208285 GB + 3.823 MB) / (524288 * 288 * 8 B + 304 * 256 * 32 * 8 B)
    "gram_partial_kernel": (1.208285e9 + 3.823104e6) / (524288 * 288 * 8 + 304 * 256 * 32 * 8),
    # store projection, ncu capture at m = 262144, K = 208, s = 16: (804.284 MB + 57.819 MB) / (8 * 262144 * 256 B);
    # the seven-digit stream is 14 B per element of Q against 8 algorithmic bytes
    "proj_store_kernel": (804.283904e6 + 57.819136e6) / (8 * 262144 * 256),
    # store Gram, ncu capture at m = 262144, na = 224, nb = 32: (825.621 MB + 9.010 MB) / (8 * 262144 * 256 B)
    "gram_store_kernel": (825.621248e6 + 9.010432e6) / (8 * 262144 * 256),
}


def measured_peaks():
    """HBM copy bandwidth measured on the GB300s (MEASURED_PEAKS.json,
    written by the pool's driver), else the profiling recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "of measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "of fallback (profiling recipe)"}
ORACLE_SAMPLE_ROWS = 2 ** 17


def alg_bytes_1s(m, n, s, b=8):
    q = n // s
    return b * m * s * q * (q - 1) / 2 + 5 * b * m * n


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-compare", action="store_true", help="skip timing BCGSI+ and -2S")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-forms", action="store_true",
                   help="skip the FP32-storage, batched and serving forms")
    p.add_argument("--forms", default="small_config,fp32_storage,block_sizes,batched,serving",
                   help="comma-separated forms to time (default: all)")
    p.add_argument("--kernel", default=None, choices=["gram", "project", "tsqr"],
                   help="time one building block alone (for profiling on small cases)")
    p.add_argument("--m", type=int, default=2 ** 19, help="rows for --kernel")
    p.add_argument("--rows", type=int, default=None,
                   help="rows of the factorization (default 2^22; smaller for profiling captures)")
    p.add_argument("--partition", default="rows", choices=["rows", "replicas"],
                   help="with N > 1 GPUs: rows = one factorization of the stacked N x 2^22-row matrix, each "
                        "rank holding 2^22 rows (Sec. 3, one all-gather per synchronization over NCCL); "
                        "replicas = N independent factorizations")
    p.add_argument("--engine", default="auto", choices=["auto", "fp64", "tensor"],
                   help="inner-product engine of the Gram and projection kernels")
    return p.parse_args()


# ------------------------------------------------------------------ CPU oracle

ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle
from paper_2507_21791_gb300 import synth
m, n, s, kappa, budget = {m}, {n}, {s}, {kappa}, {budget}
X = synth.make_matrix_np(m, n, kappa, seed=1101)
reps, t0 = 0, time.perf_counter()
while True:
    Q, R = oracle.bcgsi_plus_p_1s(X, s)
    reps += 1
    el = time.perf_counter() - t0
    if el >= budget or reps >= 20:
        break
print(json.dumps({{"reps": reps, "seconds": el, "loo": oracle.loo(Q),
                   "residual": oracle.residual(X, Q, R)}}))
"""


def run_oracle_sample(budget_s=10.0, rows=ORACLE_SAMPLE_ROWS):
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = ORACLE_SNIPPET.format(root=ROOT, m=rows, n=N, s=S, kappa=KAPPA, budget=budget_s)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    gbs = alg_bytes_1s(rows, N, S) * out["reps"] / out["seconds"] / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"BCGSI+P-1S oracle (numpy FP64) on m={rows} rows x n={N}, s={S}, "
                      f"kappa={KAPPA:g}; {out['reps']} factorization(s) in {out['seconds']:.1f} s; "
                      f"GB/s = algorithmic bytes of that m per factorization / time",
            "seconds": out["seconds"], "loo": out["loo"], "residual": out["residual"]}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm

def main_ours(args):
    Mr = args.rows if args.rows else M  # rows of the factorization
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2507_21791_gb300.replicas import dist_env, max_over_ranks, whole_job_gbs

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # Oracle sample first, in a fresh process, before heavy GPU work.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = run_oracle_sample()

    import __graft_entry__

    if not os.path.exists(os.path.join(ROOT, "paper_2507_21791_gb300", "libbcgs_qr.so")):
        __graft_entry__.build()
    from paper_2507_21791_gb300 import bcgs, synth

    bcgs.load_library()
    bcgs.set_gram_engine(args.engine)
    engine = args.engine
    stream = torch.cuda.current_stream(dev)
    X = synth.make_matrix_torch(Mr, N, KAPPA, seed=1000 + 1 * 100 + rank, device=str(dev))
    torch.cuda.synchronize()

    # N > 1 GPUs, row partition (Sec. 3): this rank's X is its 2^22-row slab of the
    # stacked matrix, and every synchronization all-gathers the ranks' local Grams
    # (or TSQR factors) over NCCL; the library adds them in rank order
    by_rows = world > 1 and args.partition == "rows"
    if by_rows:
        from paper_2507_21791_gb300 import rows as rows_mod

        comm = rows_mod.TorchAllGather()

    def workspace_for(variant):
        if by_rows:
            return torch.empty(rows_mod.workspace_size_rows(Mr, N, S, variant, world), dtype=torch.uint8,
                               device=dev)
        return torch.empty(bcgs.workspace_size(Mr, N, S, variant), dtype=torch.uint8, device=dev)

    def factor_enqueue(Xd_, variant, Q, R, ws):
        if by_rows:
            rows_mod.factor_rows(Xd_, S, variant, rank, world, comm, "fp64", Q, R, ws, check_status=False)
        else:
            bcgs.factor_async(Xd_, S, variant, "fp64", Q, R, ws)

    def global_sum(x: float) -> float:
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        if world > 1 and by_rows:
            dist.all_reduce(t)
        return float(t.item())

    def run_variant(variant, profile=False):
        Q = bcgs.empty_colmajor(Mr, N, torch.float64, dev)
        R = bcgs.empty_colmajor(N, N, torch.float64, dev)
        ws = workspace_for(variant)
        for _ in range(args.warmup):
            factor_enqueue(X, variant, Q, R, ws)
        code, blk = bcgs.factor_status(ws)
        if code != 0:
            raise RuntimeError(f"{variant}: status {bcgs.STATUS[code]} at block {blk}")
        barrier()
        clocks = ClockSampler(local) if profile else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
            bcgs.profile_enable(True)
        l0 = bcgs.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            factor_enqueue(X, variant, Q, R, ws)
        e1.record(stream)
        barrier()
        launches = bcgs.launch_count() - l0
        ms = e0.elapsed_time(e1) / args.steps
        prof = None
        if clocks:
            prof = {k: bcgs.profile_read(k) for k in bcgs.PROFILE_CLASSES}
            bcgs.profile_enable(False)
            prof["clocks"] = clocks.stop()
        code, blk = bcgs.factor_status(ws)
        if code != 0:
            raise RuntimeError(f"{variant}: status {bcgs.STATUS[code]} at block {blk}")
        eye = torch.eye(N, dtype=torch.float64, device=dev)
        QtQ = Q.T @ Q
        if by_rows:  # the Gram of the whole Q: the sum over the ranks' rows
            dist.all_reduce(QtQ)
        G = (eye - QtQ).cpu().numpy()
        loo = float(np.linalg.norm(G, 2))
        D = X - Q @ R
        res = math.sqrt(global_sum((D * D).sum().item()) / global_sum((X * X).sum().item()))
        del D
        del ws
        return {"ms": ms, "launches": launches, "loo": loo, "residual": res, "prof": prof,
                "Q": Q, "R": R}

    main = run_variant("bcgsi+p-1s", profile=True)
    ms_max = max_over_ranks(main["ms"], dev)
    value = whole_job_gbs(world, alg_bytes_1s(Mr, N, S), ms_max)

    # e2e through the public API with pinned host buffers
    Xh = torch.empty((N, Mr), dtype=torch.float64, pin_memory=True).T
    Xh.copy_(X)
    Qh = torch.empty((N, Mr), dtype=torch.float64, pin_memory=True).T
    Rh = torch.empty((N, N), dtype=torch.float64, pin_memory=True).T
    Xd = bcgs.empty_colmajor(Mr, N, torch.float64, dev)
    Qd, Rd = main["Q"], main["R"]
    ws = workspace_for("bcgsi+p-1s")

    def e2e_step():
        if by_rows:
            # this rank's slab in, the row-partitioned factorization, its rows of Q and R out
            Xd.copy_(Xh, non_blocking=True)
            factor_enqueue(Xd, "bcgsi+p-1s", Qd, Rd, ws)
            Qh.copy_(Qd, non_blocking=True)
            Rh.copy_(Rd, non_blocking=True)
            return
        # bcgs_qr_factor_host: X streams in block by block while earlier blocks are
        # factored, final blocks of Q stream back, R at the end
        bcgs.factor_host_async(Xh, S, "bcgsi+p-1s", "fp64", Qh, Rh, Xd, Qd, Rd, ws)

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    ms_e2e = max_over_ranks(ms_e2e, dev)
    e2e_value = whole_job_gbs(world, alg_bytes_1s(Mr, N, S), ms_e2e)
    del ws, Xd, Xh, Qh, Rh

    compare = {}
    if not args.no_compare and not by_rows:
        for v in ("bcgsi+", "bcgsi+p-2s", "bcgs-pipi+", "bcgsi+1s"):
            r = run_variant(v)
            compare[v] = {"ms": r["ms"], "loo": r["loo"], "residual": r["residual"]}
            del r
    compare["bcgsi+p-1s"] = {"ms": main["ms"], "loo": main["loo"], "residual": main["residual"]}
    speedup = None
    if "bcgsi+" in compare:
        speedup = {v: compare["bcgsi+"]["ms"] / compare[v]["ms"]
                   for v in ("bcgsi+p-1s", "bcgsi+p-2s", "bcgs-pipi+", "bcgsi+1s")}

    forms = None
    if not args.no_forms and world == 1:
        del main["Q"], main["R"]
        runners = {"small_config": lambda: bench_small(args, dev, stream),
                   "fp32_storage": lambda: bench_fp32(args, dev, stream),
                   "block_sizes": lambda: bench_block_sizes(args, dev, stream),
                   "batched": lambda: bench_batched(args, dev, stream),
                   "serving": lambda: bench_serving(args, dev)}
        wanted = [f for f in args.forms.split(",") if f]
        unknown = [f for f in wanted if f not in runners]
        if unknown:
            raise SystemExit(f"unknown forms: {unknown}")
        forms = {}
        gc.collect()
        torch.cuda.empty_cache()
        for f in wanted:
            forms[f] = runners[f]()
            # each form's buffers (and the private pools of its captured graphs)
            # go back before the next form allocates
            gc.collect()
            torch.cuda.empty_cache()

    prof = main["prof"]
    peaks = measured_peaks()
    step_ms_total = sum(prof[k][1] for k in bcgs.PROFILE_CLASSES)
    # dominant kernel class of the timed region (by summed event time)
    dom = max(("gram_partial", "project"), key=lambda k: prof[k][1])
    gl, gms, gfl, gby = prof[dom]
    # with the tensor engine at this size the factorization keeps Q as digit tiles
    # (the store) and both kernel classes read it
    kernel_name = {"gram_partial": "gram_store_kernel" if engine != "fp64" else "gram_partial_kernel",
                   "project": "proj_store_kernel" if engine != "fp64" else "project_kernel"}[dom]
    if engine == "fp64":
        achieved = gfl / (gms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": kernel_name + " (FP64 DFMA)", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "peak_source": "FP64 rate of the profiling recipe (nominal; a DFMA probe measured 1.20)"}
    else:
        achieved = gby / (gms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": kernel_name + " (exact f16 digit products on tcgen05, "
                                                          "operands from the resident digit store)",
                    "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"],
                    "frac_of_spec": achieved / HBM_SPEC_GBS,
                    "fp64_equivalent_tflops": gfl / (gms * 1e-3) / 1e12}
    roofline.update({
        "traffic": TRAFFIC_RATIO[kernel_name] * gby / max(gl, 1) if kernel_name in TRAFFIC_RATIO else None,
        "traffic_note": "bytes per launch: ncu dram read+write / algorithmic bytes of a smaller capture, "
                        "times this run's algorithmic bytes per launch (null: not captured for this kernel)",
        "launches": gl, "avg_launch_ms": gms / max(gl, 1),
        "share_of_timed_kernel_time": gms / step_ms_total if step_ms_total else None,
        "step_hbm_frac_of_measured_copy": value / peaks["hbm_gbs"],
    })
    others = {}
    for k in ("gram_partial", "project", "tsqr", "store_split"):
        n_, ms_, fl_, by_ = prof[k]
        if ms_ > 0:
            others[k] = {"ms_per_step": ms_ / args.steps, "alg_gbs": by_ / (ms_ * 1e-3) / 1e9,
                         "fp64_equiv_tflops": fl_ / (ms_ * 1e-3) / 1e12}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if Mr == M else WORKLOAD.replace("m=2^22", f"m={Mr}"),
                   "m": Mr, "n": N, "s": S, "kappa": KAPPA,
                   "variant": "bcgsi+p-1s",
                   "parallelism": (f"rows{world}" if by_rows else "replicas") if world > 1 else "single",
                   "global_rows": Mr * world if by_rows else Mr,
                   "l2": "inputs larger than L2 (X and Q 8.6 GB each); no flush"},
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": Mr * N * 8,
                "d2h_bytes_per_step": Mr * N * 8 + N * N * 8, "ms_per_step": ms_e2e},
        "gpu_launches": main["launches"],
        "roofline": roofline,
        "kernels": others,
        "engine": engine,
        "speedup_vs_bcgsi_plus_at_equal_loo": speedup,
        "variants": compare,
        "clocks": prof["clocks"],
        "kernel_time_ms_per_step": {k: prof[k][1] / args.steps for k in bcgs.PROFILE_CLASSES},
        "cpu_baseline": cpu,
        "forms": forms,
        "p99_latency_ms": (forms["serving"]["lambda_2000"]["call_latency_ms"]["p99"]
                           if forms and "serving" in forms else None),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ forms

def _timed(fn, warmup, steps, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_fp32(args, dev, stream):
    """Precision form: m = 2^24, n = 128, s = 32, BCGSI+P-1S, X and Q in FP32,
    Gram / Cholesky / R in FP64; accuracy against the FP64 X."""
    import numpy as np
    import torch

    from paper_2507_21791_gb300 import bcgs, synth

    m, n, s, kappa = 2 ** 24, 128, 32, 1e4
    X64 = synth.make_matrix_torch(m, n, kappa, seed=1200, device=str(dev))
    X = X64.float()
    Q = bcgs.empty_colmajor(m, n, torch.float32, dev)
    R = bcgs.empty_colmajor(n, n, torch.float64, dev)
    ws = torch.empty(bcgs.workspace_size(m, n, s, "bcgsi+p-1s", "fp32"), dtype=torch.uint8, device=dev)
    ms = _timed(lambda: bcgs.factor_async(X, s, "bcgsi+p-1s", "fp32", Q, R, ws), args.warmup,
                args.steps, stream)
    # one more factorization with the per-class event profile
    bcgs.profile_enable(True)
    bcgs.factor_async(X, s, "bcgsi+p-1s", "fp32", Q, R, ws)
    torch.cuda.synchronize()
    classes = {k: round(bcgs.profile_read(k)[1], 2) for k in bcgs.PROFILE_CLASSES}
    bcgs.profile_enable(False)
    code, blk = bcgs.factor_status(ws)
    Qd = Q.double()
    eye = torch.eye(n, dtype=torch.float64, device=dev)
    loo = float(np.linalg.norm((eye - Qd.T @ Qd).cpu().numpy(), 2))
    D = X64 - Qd @ R
    res = math.sqrt((D * D).sum().item() / (X64 * X64).sum().item())
    del D, Qd, X64
    return {"workload": f"FP32 storage m=2^24 n=128 s=32 BCGSI+P-1S kappa={kappa:g}",
            "value": alg_bytes_1s(m, n, s, b=4) / (ms * 1e-3) / 1e9, "unit": "GB/s",
            "ms_per_step": ms, "status": bcgs.STATUS[code], "loo": loo,
            "residual_vs_fp64_x": res, "ms_per_class": classes,
            "bound": "FP64 ALU (products accumulated in FP64)"}


# Table 2 of the paper: speedup over CGSI+ (BCGSI+ with s = 1) at 10^6 x 400 on
# 64 nodes, by variant and block size s
TABLE2_64_NODES = {
    "bcgsi+p-2s": {1: 1.3, 2: 2.6, 4: 5.2, 8: 10.2, 16: 15.9},
    "bcgsi+p-1s": {1: 2.8, 2: 5.4, 4: 10.8, 8: 20.0, 16: 37.5},
    "bcgs-pipi+": {1: 1.6, 2: 3.0, 4: 5.9, 8: 11.7, 16: 22.7},
    "bcgsi+1s": {1: 2.9, 2: 5.8, 4: 10.6, 8: 21.2, 16: 37.8},
    "bcgsi+": {1: 1.0, 2: 1.4, 4: 2.7, 8: 5.4, 16: 8.8},
}


def bench_small(args, dev, stream):
    """Small configuration (m = 10^4, n = 64, s = 8, kappa = 1e4): the whole
    factorization stays in L2, so it is bound by kernel launches and the
    grid-wide reductions, the one-GPU analog of the synchronization-bound regime
    of Sec. 4.  Per variant: microseconds per factorization (3 warm-ups, 20
    timed), kernel launches and synchronizations (Gram reductions and TSQR trees)
    per factorization."""
    import torch

    from paper_2507_21791_gb300 import bcgs, synth

    m, n, s, kappa = 10_000, 64, 8, 1e4
    X = synth.make_matrix_torch(m, n, kappa, seed=1000, device=str(dev))
    Q = bcgs.empty_colmajor(m, n, torch.float64, dev)
    R = bcgs.empty_colmajor(n, n, torch.float64, dev)
    out = {}
    for v in ("bcgsi+", "bcgsi+p-2s", "bcgsi+p-1s", "bcgs-pipi+", "bcgsi+1s"):
        ws = torch.empty(bcgs.workspace_size(m, n, s, v), dtype=torch.uint8, device=dev)

        def run():
            bcgs.factor_async(X, s, v, "fp64", Q, R, ws)

        run()
        torch.cuda.synchronize()
        l0 = bcgs.launch_count()
        run()
        torch.cuda.synchronize()
        launches = bcgs.launch_count() - l0
        bcgs.profile_enable(True)
        run()
        torch.cuda.synchronize()
        syncs = bcgs.profile_read("gram_reduce")[0] + bcgs.profile_read("tsqr")[0]
        classes = {k: round(bcgs.profile_read(k)[1] * 1e3, 1) for k in bcgs.PROFILE_CLASSES}
        bcgs.profile_enable(False)
        ms = _timed(run, 3, 20, stream)
        # the same factorization captured once into a CUDA graph and replayed
        # (one graph launch per factorization: no host launch overhead per kernel)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run()
        gms = _timed(g.replay, 3, 50, stream)
        # the same with the tensor-core engine at this size (digit store, exact digit products)
        saved = bcgs.get_gram_engine()
        bcgs.set_gram_engine("tensor")
        try:
            ws_t = torch.empty(bcgs.workspace_size(m, n, s, v), dtype=torch.uint8, device=dev)
            gt = torch.cuda.CUDAGraph()
            bcgs.factor_async(X, s, v, "fp64", Q, R, ws_t)
            torch.cuda.synchronize()
            with torch.cuda.graph(gt):
                bcgs.factor_async(X, s, v, "fp64", Q, R, ws_t)
            tms = _timed(gt.replay, 3, 50, stream)
            tstatus = bcgs.STATUS[bcgs.factor_status(ws_t)[0]]
            del gt, ws_t
        finally:
            bcgs.set_gram_engine(saved)
        out[v] = {"us_per_factorization": ms * 1e3, "us_per_factorization_graph": gms * 1e3,
                  "us_per_block_step_graph": gms * 1e3 / (n // s), "us_per_class_eager": classes,
                  "us_per_factorization_graph_tensor_engine": tms * 1e3, "status_tensor_engine": tstatus,
                  "kernel_launches": launches,
                  "synchronizations": int(syncs), "status": bcgs.STATUS[bcgs.factor_status(ws)[0]]}
        del g
        del ws
    return {"workload": f"m=10^4 n=64 s=8 kappa={kappa:g}, FP64, L2-resident", "variants": out,
            "note": "launch- and synchronization-bound: no HBM fraction; *_graph: one CUDA graph replay "
                    "per factorization"}


def bench_block_sizes(args, dev, stream):
    """Block-size form, the one-GPU analog of Table 2: m = 10^6, n = 400,
    s in {1, 2, 4, 8, 16}, every variant timed as one factorization (one warm-up,
    one timed run each); speedup over CGSI+ = BCGSI+ with s = 1."""
    import torch

    from paper_2507_21791_gb300 import bcgs, synth

    m, n, kappa = 10 ** 6, 400, 1e5
    X = synth.make_matrix_torch(m, n, kappa, seed=1300, device=str(dev))
    Q = bcgs.empty_colmajor(m, n, torch.float64, dev)
    R = bcgs.empty_colmajor(n, n, torch.float64, dev)
    ms, status = {}, {}
    for v in TABLE2_64_NODES:
        ms[v], status[v] = {}, {}
        for s in (1, 2, 4, 8, 16):
            ws = torch.empty(bcgs.workspace_size(m, n, s, v), dtype=torch.uint8, device=dev)
            ms[v][s] = _timed(lambda: bcgs.factor_async(X, s, v, "fp64", Q, R, ws), 1, 1, stream)
            status[v][s] = bcgs.STATUS[bcgs.factor_status(ws)[0]]
            del ws
    base = ms["bcgsi+"][1]
    speedup = {v: {s: base / t for s, t in row.items()} for v, row in ms.items()}
    return {"workload": f"m=10^6 n=400 kappa={kappa:g}, s in (1, 2, 4, 8, 16), FP64",
            "ms": ms, "status": status, "speedup_vs_cgsi_plus": speedup,
            "paper_speedup_64_nodes": TABLE2_64_NODES,
            "note": "one warm-up and one timed factorization per cell; CGSI+ = BCGSI+ at s = 1"}


def bench_batched(args, dev, stream):
    """Batched form: 512 FP64 QRs, m = round(2^U(12,18)), n in {32, 64, 128},
    kappa = 10^U(1,8), s and the product engine (FP64 pipe or tensor cores)
    picked per shape by the autotuner from {4, 8, 16} x {fp64, tensor};
    BCGSI+P-2S (kappa up to 1e8 is outside BCGSI+P-1S's O(u) kappa^2 <= 1
    range); the batch is one CUDA-graph launch."""
    import numpy as np
    import torch

    from paper_2507_21791_gb300 import synth
    from paper_2507_21791_gb300.batched import Batch, BlockSizeTuner, alg_bytes

    rng = np.random.default_rng(1300)
    tuner = BlockSizeTuner(candidates=(4, 8, 16), variant="bcgsi+p-2s", engines=("fp64", "tensor"))
    Xs, ss, engs, total = [], [], [], 0.0
    for i in range(512):
        m = synth.log_uniform_int(rng, 12, 18)
        n = int(rng.choice([32, 64, 128]))
        kappa = 10.0 ** rng.uniform(1, 8)
        Xs.append(synth.make_matrix_torch(m, n, kappa, seed=1300 + i, device=str(dev)))
    for X in Xs:
        m, n = X.shape
        s_, e_ = tuner.choose(m, n, device=str(dev))
        ss.append(s_)
        engs.append(e_)
        total += alg_bytes(m, n, ss[-1], "bcgsi+p-2s")
    b = Batch(Xs, ss, variant="bcgsi+p-2s", engines=engs)
    b.capture()
    ms = _timed(b.replay, args.warmup, args.steps, stream)
    codes, _ = b.status()
    return {"workload": "512 FP64 QRs m=2^U(12,18) n in {32,64,128} kappa=10^U(1,8) BCGSI+P-2S, "
                        "one CUDA-graph launch", "value": total / (ms * 1e-3) / 1e9, "unit": "GB/s",
            "instances_per_s": 512 / (ms * 1e-3), "ms_per_batch": ms,
            "failed": sum(1 for c in codes if c != 0),
            "autotuned_s_engine": {k: list(v) for k, v in sorted(tuner.table.items())}}


def bench_serving(args, dev):
    """Serving form: Poisson requests (Krylov-like bases: m = 2^U(14,20), q ~ U{4..32}
    blocks of s in {4, 8, 16}, kappa up to 1e8), one block per call, Q and R
    resident, admission against a 120 GB budget, BCGSI+P-2S."""
    import torch

    from paper_2507_21791_gb300.serving import GpuBackend, Server, draw_sources, make_requests

    sources, meta = draw_sources(24, seed=1400, device=str(dev))
    out = {}
    # the same unsaturated arrivals with lazy (delayed) and eager finalization
    for rate, window, eager, key in ((2000.0, 4.0, 0.0, "lambda_2000"), (10.0, 4.0, 0.0, "lambda_10"),
                                     (10.0, 4.0, 1.0, "lambda_10_eager")):
        be = GpuBackend(sources, variant="bcgsi+p-2s", nstreams=32, device=str(dev))
        srv = Server(be, budget_bytes=120e9)
        reqs = make_requests(rate, window, meta, seed=int(rate), eager_frac=eager)
        rep = srv.run(reqs, duration=window)
        rep["offered_req_per_s"] = rate
        rep["arrivals"] = len(reqs)
        out[key] = rep
        # the resident bases of this run go back before the next run admits its own
        del srv, be
        gc.collect()
        torch.cuda.empty_cache()
    return {"workload": "Poisson Krylov-basis requests, m=2^U(14,20), q~U{4..32}, s in {4,8,16}, "
                        "120 GB budget, BCGSI+P-2S (lazy) or BCGSI+ (eager finalize), pool of 24 "
                        "pre-generated bases", **out}


def main_kernel(args):
    """One building block of the cfg shape (n = 256, s = 16) on m rows, alone:
    gram = the largest synchronization of a BCGSI+P-1S factorization,
    [Q_{1:14} U X]^T [U X] (256 x 32); project = U = (X - Q_{1:15} S) S_kk^{-1};
    tsqr = TSQR of an m x 16 block."""
    import torch

    import __graft_entry__

    if not os.path.exists(os.path.join(ROOT, "paper_2507_21791_gb300", "libbcgs_qr.so")):
        __graft_entry__.build()
    from paper_2507_21791_gb300 import bcgs, synth

    bcgs.load_library()
    bcgs.set_gram_engine(args.engine)
    m = args.m
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    A = torch.randn((N, m), dtype=torch.float64, device="cuda", generator=g).T
    B = torch.randn((2 * S, m), dtype=torch.float64, device="cuda", generator=g).T
    C = torch.randn((N - S, S), dtype=torch.float64, device="cuda", generator=g).T.contiguous().T
    T = (torch.eye(S, dtype=torch.float64, device="cuda") * 2.0).T
    X16 = synth.make_matrix_torch(m, S, 1e3, seed=9)

    def once():
        if args.kernel == "gram":
            bcgs.gram(A, B)
        elif args.kernel == "project":
            bcgs.project(B[:, :S], A[:, :N - S], C[:N - S], T)
        else:
            bcgs.tsqr(X16)

    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    bcgs.profile_enable(True)
    for _ in range(args.steps):
        once()
    torch.cuda.synchronize()
    cls = {"gram": "gram_partial", "project": "project", "tsqr": "tsqr"}[args.kernel]
    n, ms, fl, by = bcgs.profile_read(cls)
    bcgs.profile_enable(False)
    print(json.dumps({"kernel": args.kernel, "m": m, "engine": bcgs.get_gram_engine(),
                      "launches": n, "avg_ms": ms / max(n, 1),
                      "tflops": fl / (ms * 1e-3) / 1e12, "alg_gbs": by / (ms * 1e-3) / 1e9}))


def main_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    info = None
    budget = 4.0
    for i in range(args.warmup + args.steps):
        info = run_oracle_sample(budget_s=budget, rows=2 ** 15)
        if i >= args.warmup:
            per_step.append(info["value"])
    value = statistics.median(per_step)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "s": S, "kappa": KAPPA,
                   "variant": "bcgsi+p-1s", "sample_rows": 2 ** 15},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": info["cores"], "kind": "oracle",
                         "sample": info["sample"]},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.kernel:
        main_kernel(a)
    elif a.impl == "reference":
        main_reference(a)
    else:
        main_ours(a)
