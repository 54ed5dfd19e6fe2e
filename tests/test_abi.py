"""The C ABI library loads and exports every symbol include/bcgs_qr.h declares;
host-side argument checks (no GPU needed: they return before any CUDA call)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT, ensure_library


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "bcgs_qr.h")).read()
    return sorted(set(re.findall(r"^BCGS_API\s+[\w\s\*]+?\b(bcgs_\w+)\s*\(", hdr, flags=re.M)))


def test_header_declares_the_expected_entry_points():
    syms = declared_symbols()
    for name in ("bcgs_qr_init", "bcgs_qr_step", "bcgs_qr_factor", "bcgs_qr_finish", "bcgs_qr_sync",
                 "bcgs_qr_factor_batched", "bcgs_gram", "bcgs_project", "bcgs_tsqr", "bcgs_chol"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    bound = {n for n, _, _ in bcgs.SIGNATURES}
    assert bound == set(declared_symbols())


def test_status_strings_and_version():
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    assert lib.bcgs_version() >= 100
    for code in range(9):
        assert len(lib.bcgs_status_string(code)) > 0
    assert lib.bcgs_status_string(99) == b"unknown status"


def test_workspace_size_queries():
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    m, n, s = 10000, 64, 8
    sizes = {v: bcgs.workspace_size(m, n, s, v) for v in bcgs.VARIANTS}
    # 1S needs no separate projected block V, BCGS-PIPI+ neither V nor the paired
    # coefficients; BCGSI+ and 2S keep V for their TSQR
    assert sizes["bcgsi+p-1s"] < sizes["bcgsi+p-2s"]
    assert sizes["bcgs-pipi+"] < sizes["bcgsi+p-1s"] and sizes["bcgs-pipi+"] < sizes["bcgsi+"]
    assert bcgs.workspace_size(m, n, s, "bcgsi+p-1s", "fp32") < sizes["bcgsi+p-1s"]
    # FP64 engine: U, the TSQR tree and the row maxima, a few m x s blocks
    old = bcgs.get_gram_engine()
    try:
        bcgs.set_gram_engine("fp64")
        small = bcgs.workspace_size(2 ** 22, 256, 16, "bcgsi+p-1s")
        small32 = bcgs.workspace_size(2 ** 22, 256, 16, "bcgsi+p-1s", "fp32")
        bcgs.set_gram_engine("tensor")
        big = bcgs.workspace_size(2 ** 22, 256, 16, "bcgsi+p-1s")
        # the tensor engine adds the digit store of Q: 14 bytes per element
        # (seven f16 digits) plus one exponent per 128 rows and column, for
        # both storage types
        fp32 = bcgs.workspace_size(2 ** 22, 256, 16, "bcgsi+p-1s", "fp32")
    finally:
        bcgs.set_gram_engine(old)
    assert 2 ** 22 * 16 * 8 < small < 2 ** 22 * 16 * 8 * 3
    # digits, one exponent per 128 rows and column, and 32 exponents per row
    # block for the coefficient side of the projections
    store = 2 ** 22 * 256 * 14 + (2 ** 22 // 128) * 256 * 4 + (2 ** 22 // 128) * 32 * 4
    assert big - small == pytest.approx(store, abs=2 ** 12)
    assert fp32 - small32 == pytest.approx(store, abs=2 ** 12)
    assert small32 < small and fp32 < big  # FP32 blocks of U and V


@pytest.mark.parametrize("m,n,s", [(100, 0, 8), (100, 16, 0), (4, 8, 8), (100, 64, 65),
                                   (100, 4096, 8)])
def test_invalid_shapes_rejected_without_a_gpu(m, n, s):
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    out = ctypes.c_size_t(0)
    assert lib.bcgs_qr_workspace_size(m, n, s, 1, 0, ctypes.byref(out)) == 1
    # factor with bogus pointers: rejected before anything is enqueued
    assert lib.bcgs_qr_factor(m, n, s, 1, 0, 8, m, 16, m, 32, n, 256, 1 << 20, None) == 1


def test_bad_enums_and_null_pointers_rejected():
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    out = ctypes.c_size_t(0)
    assert lib.bcgs_qr_workspace_size(100, 16, 8, 5, 0, ctypes.byref(out)) == 1
    assert lib.bcgs_qr_workspace_size(100, 16, 8, 4, 0, ctypes.byref(out)) == 0  # BCGSI+1s
    assert lib.bcgs_qr_workspace_size(100, 16, 8, -1, 0, ctypes.byref(out)) == 1
    assert lib.bcgs_qr_workspace_size(100, 16, 8, 3, 0, ctypes.byref(out)) == 0
    assert lib.bcgs_qr_workspace_size(100, 16, 8, 1, 2, ctypes.byref(out)) == 1
    assert lib.bcgs_qr_factor(100, 16, 8, 1, 0, None, 100, 16, 100, 32, 16, 256, 1 << 20, None) == 1
    h = ctypes.c_void_p(None)
    assert lib.bcgs_qr_init(ctypes.byref(h), 100, 16, 8, 1, 0, None, 100, 32, 16, 256, 1 << 20, None) == 1
    assert lib.bcgs_qr_step(None, None, 100) == 1
    # host entry point: null host or device pointers, leading dimensions below m
    assert lib.bcgs_qr_factor_host(100, 16, 8, 1, 0, None, 100, 8, 100, 8, 16, 8, 100, 8, 100, 8, 16, 256,
                                   1 << 20, None) == 1
    assert lib.bcgs_qr_factor_host(100, 16, 8, 1, 0, 8, 99, 8, 100, 8, 16, 8, 100, 8, 100, 8, 16, 256,
                                   1 << 20, None) == 1
    X, Q = 1 << 40, 1 << 41  # distinct (never dereferenced) device addresses
    # misaligned workspace
    assert lib.bcgs_qr_factor(100, 16, 8, 1, 0, X, 100, Q, 100, 32, 16, 257, 1 << 20, None) == 5
    # too small workspace
    assert lib.bcgs_qr_factor(100, 16, 8, 1, 0, X, 100, Q, 100, 32, 16, 256, 1024, None) == 5


@pytest.mark.parametrize("precision,esz", [(0, 8), (1, 4)])
def test_overlapping_x_and_q_rejected_without_a_gpu(precision, esz):
    """In-place factorization is not supported: X and Q whose memory overlaps
    are rejected with BCGS_ERR_INVALID_ARG before anything is enqueued (the
    check is host-side pointer arithmetic; the pointers are never read)."""
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    m, n, s = 100, 16, 8
    X = 1 << 40
    last = X + ((n - 1) * m + m) * esz  # one past the last byte of X
    for Q in (X, X + 8 * esz, last - esz, X - 3 * m * esz):
        assert lib.bcgs_qr_factor(m, n, s, 1, precision, X, m, Q, m, 32, n, 256, 1 << 20, None) == 1
        assert lib.bcgs_qr_factor_host(m, n, s, 1, precision, 8, m, 8, m, 8, n, X, m, Q, m, 32, n, 256,
                                       1 << 20, None) == 1
    # touching but not overlapping: the call goes on to the next check (a too
    # small workspace, BCGS_ERR_WORKSPACE), so the test is not over-eager
    assert lib.bcgs_qr_factor(m, n, s, 1, precision, X, m, last, m, 32, n, 256, 1024, None) == 5
    assert lib.bcgs_qr_factor(m, n, s, 1, precision, X, m, X - (n * m) * esz, m, 32, n, 256, 1024, None) == 5
    # batched: one overlapping problem rejects the whole call
    probs = (bcgs.Problem * 2)()
    probs[0] = bcgs.Problem(m, n, s, 1, precision, X, m, 1 << 42, m, 32, n, 0)
    probs[1] = bcgs.Problem(m, n, s, 1, precision, 1 << 43, m, (1 << 43) + 8, m, 32, n, 0)
    need = ctypes.c_size_t(0)
    assert lib.bcgs_qr_batched_workspace_size(2, probs, ctypes.byref(need)) == 0
    assert lib.bcgs_qr_factor_batched(2, probs, 1 << 44, need.value, None) == 1


def test_batched_problem_engine_field():
    """bcgs_problem.engine: 0..3 accepted, anything else INVALID_ARG; with the
    tensor engine for every size the workspace holds the digit store (larger),
    with the FP64 pipe it does not (host-only: no GPU needed)."""
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    m, n, s = 4096, 64, 16
    sizes = {}
    for name, eng in bcgs.PROBLEM_ENGINES.items():
        probs = (bcgs.Problem * 1)()
        probs[0] = bcgs.Problem(m, n, s, 1, 0, 1 << 40, m, 1 << 42, m, 1 << 44, n, eng)
        need = ctypes.c_size_t(0)
        assert lib.bcgs_qr_batched_workspace_size(1, probs, ctypes.byref(need)) == 0
        sizes[name] = need.value
    assert sizes["tensor"] > sizes["fp64"]
    assert sizes["auto"] == sizes["fp64"]  # 4096 rows: below the default tensor-core threshold
    for bad in (-1, 4):
        probs = (bcgs.Problem * 1)()
        probs[0] = bcgs.Problem(m, n, s, 1, 0, 1 << 40, m, 1 << 42, m, 1 << 44, n, bad)
        need = ctypes.c_size_t(0)
        assert lib.bcgs_qr_batched_workspace_size(1, probs, ctypes.byref(need)) == 1


def test_debug_sync_option():
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    assert lib.bcgs_get_option(3) == 0
    assert lib.bcgs_set_option(3, 2) == 1
    assert lib.bcgs_set_option(3, 1) == 0 and lib.bcgs_get_option(3) == 1
    assert lib.bcgs_set_option(3, 0) == 0 and lib.bcgs_get_option(3) == 0


@pytest.mark.parametrize("m,n,s", [(100, 30, 8), (100, 5, 8), (1000, 17, 16)])
def test_ragged_shapes_accepted(m, n, s):
    """n need not be a multiple of s: the last block is ragged (n mod s columns)."""
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    out = ctypes.c_size_t(0)
    for variant in range(5):
        assert lib.bcgs_qr_workspace_size(m, n, s, variant, 0, ctypes.byref(out)) == 0
        assert out.value > 0


def test_wait_selftest_argument_checks():
    """bcgs_wait_selftest rejects bad arguments before touching the GPU."""
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    lib = bcgs.load_library()
    assert lib.bcgs_wait_selftest(None, 256, 1000, None) == 1
    assert lib.bcgs_wait_selftest(256, 128, 1000, None) == 1
    assert lib.bcgs_wait_selftest(256, 256, 0, None) == 1
    assert lib.bcgs_wait_selftest(256, 256, 3_000_000_000, None) == 1
    assert lib.bcgs_wait_selftest(257, 256, 1000, None) == 5
