"""ctypes binding of the C ABI in include/bcgs_qr.h (argument marshalling only).

Every numerical step runs in the CUDA library libbcgs_qr.so built from csrc/;
this module only allocates caller-side buffers with PyTorch, passes device
pointers, sizes and the current CUDA stream, and reads status codes.  If the
library is missing it raises; there is no other implementation to fall back on.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbcgs_qr.so")

VARIANTS = {"bcgsi+": 0, "bcgsi+p-1s": 1, "bcgsi+p-2s": 2, "bcgs-pipi+": 3, "bcgsi+1s": 4}
PRECISIONS = {"fp64": 0, "fp32": 1}
STATUS = {
    0: "ok", 1: "invalid_arg", 2: "not_spd", 3: "rank_deficient", 4: "nonfinite",
    5: "workspace", 6: "timeout", 7: "state", 8: "cuda", 9: "comm",
}

# Every symbol declared in include/bcgs_qr.h: (name, restype, argtypes).
_i64, _i32, _vp, _sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t
_pi32, _psz = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t)


class Problem(ctypes.Structure):
    """bcgs_problem."""
    _fields_ = [("m", _i64), ("n", _i32), ("s", _i32), ("variant", _i32), ("precision", _i32),
                ("X", _vp), ("ldx", _i64), ("Q", _vp), ("ldq", _i64), ("R", _vp), ("ldr", _i32),
                ("engine", _i32)]

# bcgs_problem.engine: 0 = the global option, else 1 + the option value
PROBLEM_ENGINES = {"default": 0, "fp64": 1, "auto": 2, "tensor": 3}


SIGNATURES = [
    ("bcgs_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("bcgs_version", ctypes.c_int, []),
    ("bcgs_qr_workspace_size", ctypes.c_int, [_i64, _i32, _i32, ctypes.c_int, ctypes.c_int, _psz]),
    ("bcgs_qr_factor", ctypes.c_int, [_i64, _i32, _i32, ctypes.c_int, ctypes.c_int, _vp, _i64, _vp,
                                      _i64, _vp, _i32, _vp, _sz, _vp]),
    ("bcgs_qr_factor_host", ctypes.c_int, [_i64, _i32, _i32, ctypes.c_int, ctypes.c_int, _vp, _i64, _vp,
                                           _i64, _vp, _i32, _vp, _i64, _vp, _i64, _vp, _i32, _vp, _sz, _vp]),
    ("bcgs_qr_factor_status", ctypes.c_int, [_vp, _vp, _pi32]),
    ("bcgs_wait_selftest", ctypes.c_int, [_vp, _sz, _i64, _vp]),
    ("bcgs_qr_init", ctypes.c_int, [ctypes.POINTER(_vp), _i64, _i32, _i32, ctypes.c_int, ctypes.c_int,
                                    _vp, _i64, _vp, _i32, _vp, _sz, _vp]),
    ("bcgs_qr_step", ctypes.c_int, [_vp, _vp, _i64]),
    ("bcgs_qr_finish", ctypes.c_int, [_vp]),
    ("bcgs_qr_sync", ctypes.c_int, [_vp, _pi32, _pi32]),
    ("bcgs_qr_set_stream", ctypes.c_int, [_vp, _vp]),
    ("bcgs_qr_destroy", ctypes.c_int, [_vp]),
    ("bcgs_qr_batched_workspace_size", ctypes.c_int, [_i32, ctypes.POINTER(Problem), _psz]),
    ("bcgs_qr_factor_batched", ctypes.c_int, [_i32, ctypes.POINTER(Problem), _vp, _sz, _vp]),
    ("bcgs_qr_batched_status", ctypes.c_int, [_i32, _vp, _vp, _pi32, _pi32]),
    ("bcgs_gram_workspace_size", ctypes.c_int, [_i64, _i32, _i32, _psz]),
    ("bcgs_gram", ctypes.c_int, [_i64, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _i32, _vp, _sz, _vp]),
    ("bcgs_project", ctypes.c_int, [_i64, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _i32, _vp, _i32,
                                    _vp, _i64, _vp]),
    ("bcgs_tsqr_workspace_size", ctypes.c_int, [_i64, _i32, _psz]),
    ("bcgs_tsqr", ctypes.c_int, [_i64, _i32, _vp, _i64, _vp, _i64, _vp, _i32, _vp, _sz, _vp]),
    ("bcgs_chol", ctypes.c_int, [_i32, _vp, _i32, _vp, _i32, _vp, _sz, _vp]),
    ("bcgs_gram_noalloc", ctypes.c_int, [_i64, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _i32, _vp]),
    ("bcgs_row_partition", ctypes.c_int, [_i64, _i32, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    ("bcgs_qr_workspace_size_rows", ctypes.c_int, [_i64, _i32, _i32, ctypes.c_int, ctypes.c_int, _i32, _psz]),
    ("bcgs_qr_factor_rows", ctypes.c_int, [_i64, _i32, _i32, ctypes.c_int, ctypes.c_int, _vp, _i64, _vp, _i64,
                                           _vp, _i32, _vp, _sz, _vp, _i32, _i32, _vp, _vp]),
    ("bcgs_set_option", ctypes.c_int, [ctypes.c_int, ctypes.c_int64]),
    ("bcgs_get_option", ctypes.c_int64, [ctypes.c_int]),
    ("bcgs_launch_count", ctypes.c_int64, []),
    ("bcgs_profile_enable", ctypes.c_int, [ctypes.c_int]),
    ("bcgs_profile_reset", ctypes.c_int, []),
    ("bcgs_profile_read", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
]

PROFILE_CLASSES = {"gram_partial": 0, "gram_reduce": 1, "project": 2, "tsqr": 3, "tail": 4,
                   "store_split": 5}

_lib = None


class BCGSError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


def load_library(reload: bool = False):
    """Load libbcgs_qr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and not reload:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != 0:
        raise BCGSError(rc, where)


def _stream_ptr(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor_ld(t) -> int:
    """Leading dimension of a column-major (stride (1, ld)) 2-D tensor."""
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("expected a column-major 2-D tensor (stride(0) == 1)")
    return max(t.stride(1), t.shape[0]) if t.shape[1] > 1 else max(t.shape[0], 1)


def empty_colmajor(m: int, n: int, dtype, device="cuda"):
    import torch

    return torch.empty((n, m), dtype=dtype, device=device).T


def _workspace(nbytes: int, device):
    import torch

    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def workspace_size(m: int, n_max: int, s: int, variant: str, precision: str = "fp64") -> int:
    lib = load_library()
    out = ctypes.c_size_t(0)
    _check(lib.bcgs_qr_workspace_size(m, n_max, s, VARIANTS[variant], PRECISIONS[precision],
                                      ctypes.byref(out)), "bcgs_qr_workspace_size")
    return out.value


def factor(X, s: int, variant: str = "bcgsi+p-1s", precision: str | None = None, Q=None, R=None,
           workspace=None, stream=None, check_status: bool = True):
    """Economic QR of the column-major device tensor X (float64, or float32 for the
    FP32-storage form).  Returns (Q, R, status_code, fail_block)."""
    import torch

    lib = load_library()
    if precision is None:
        precision = "fp32" if X.dtype == torch.float32 else "fp64"
    m, n = X.shape
    ldx = _colmajor_ld(X)
    dt = torch.float32 if precision == "fp32" else torch.float64
    if Q is None:
        Q = empty_colmajor(m, n, dt, X.device)
    if R is None:
        R = empty_colmajor(n, n, torch.float64, X.device)
    nbytes = workspace_size(m, n, s, variant, precision)
    if workspace is None:
        workspace = _workspace(nbytes, X.device)
    sp = _stream_ptr(stream)
    rc = lib.bcgs_qr_factor(m, n, s, VARIANTS[variant], PRECISIONS[precision], X.data_ptr(), ldx,
                            Q.data_ptr(), _colmajor_ld(Q), R.data_ptr(), _colmajor_ld(R),
                            workspace.data_ptr(), workspace.numel(), sp)
    _check(rc, "bcgs_qr_factor")
    if not check_status:
        return Q, R, None, None
    blk = ctypes.c_int32(0)
    code = lib.bcgs_qr_factor_status(workspace.data_ptr(), sp, ctypes.byref(blk))
    return Q, R, code, blk.value


def factor_async(X, s, variant, precision, Q, R, workspace, stream=None):
    """Enqueue only (no status read): for timing loops and graph capture."""
    lib = load_library()
    m, n = X.shape
    rc = lib.bcgs_qr_factor(m, n, s, VARIANTS[variant], PRECISIONS[precision], X.data_ptr(),
                            _colmajor_ld(X), Q.data_ptr(), _colmajor_ld(Q), R.data_ptr(),
                            _colmajor_ld(R), workspace.data_ptr(), workspace.numel(),
                            _stream_ptr(stream))
    _check(rc, "bcgs_qr_factor")


def factor_host_async(Xh, s, variant, precision, Qh, Rh, Xd, Qd, Rd, workspace, stream=None):
    """End-to-end factorization from host memory (bcgs_qr_factor_host): Xh, Qh,
    Rh are column-major CPU tensors (pinned for the copies to overlap the
    factorization), Xd, Qd, Rd column-major device tensors of the same shapes.
    Enqueue only; the host results are complete once the stream is."""
    lib = load_library()
    m, n = Xh.shape
    for name, t, dev in (("Xh", Xh, False), ("Qh", Qh, False), ("Rh", Rh, False), ("Xd", Xd, True),
                         ("Qd", Qd, True), ("Rd", Rd, True)):
        if t.is_cuda != dev:
            raise ValueError(f"{name} must be a {'device' if dev else 'host'} tensor")
    rc = lib.bcgs_qr_factor_host(m, n, s, VARIANTS[variant], PRECISIONS[precision], Xh.data_ptr(),
                                 _colmajor_ld(Xh), Qh.data_ptr(), _colmajor_ld(Qh), Rh.data_ptr(),
                                 _colmajor_ld(Rh), Xd.data_ptr(), _colmajor_ld(Xd), Qd.data_ptr(),
                                 _colmajor_ld(Qd), Rd.data_ptr(), _colmajor_ld(Rd), workspace.data_ptr(),
                                 workspace.numel(), _stream_ptr(stream))
    _check(rc, "bcgs_qr_factor_host")


def factor_status(workspace, stream=None):
    lib = load_library()
    blk = ctypes.c_int32(0)
    code = lib.bcgs_qr_factor_status(workspace.data_ptr(), _stream_ptr(stream), ctypes.byref(blk))
    return code, blk.value


class QRHandle:
    """Block-by-block factorization (bcgs_qr_init / step / finish / sync)."""

    def __init__(self, m: int, n_max: int, s: int, variant: str = "bcgsi+p-1s",
                 precision: str = "fp64", device="cuda", Q=None, R=None, workspace=None,
                 stream=None):
        import torch

        self.lib = load_library()
        self.m, self.n_max, self.s = m, n_max, s
        self.variant, self.precision = variant, precision
        dt = torch.float32 if precision == "fp32" else torch.float64
        self.Q = Q if Q is not None else empty_colmajor(m, n_max, dt, device)
        self.R = R if R is not None else empty_colmajor(n_max, n_max, torch.float64, device)
        nbytes = workspace_size(m, n_max, s, variant, precision)
        self.workspace = workspace if workspace is not None else _workspace(nbytes, device)
        self._h = ctypes.c_void_p(None)
        self._stream = stream
        rc = self.lib.bcgs_qr_init(ctypes.byref(self._h), m, n_max, s, VARIANTS[variant],
                                   PRECISIONS[precision], self.Q.data_ptr(), _colmajor_ld(self.Q),
                                   self.R.data_ptr(), _colmajor_ld(self.R),
                                   self.workspace.data_ptr(), self.workspace.numel(),
                                   _stream_ptr(stream))
        _check(rc, "bcgs_qr_init")

    def step(self, Xj):
        _check(self.lib.bcgs_qr_step(self._h, Xj.data_ptr(), _colmajor_ld(Xj)), "bcgs_qr_step")

    def finish(self):
        _check(self.lib.bcgs_qr_finish(self._h), "bcgs_qr_finish")

    def set_stream(self, stream):
        self._stream = stream
        _check(self.lib.bcgs_qr_set_stream(self._h, _stream_ptr(stream)), "bcgs_qr_set_stream")

    def sync(self):
        nf, fb = ctypes.c_int32(0), ctypes.c_int32(0)
        code = self.lib.bcgs_qr_sync(self._h, ctypes.byref(nf), ctypes.byref(fb))
        return code, nf.value, fb.value

    def close(self):
        if self._h:
            self.lib.bcgs_qr_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class BatchItem:
    X: object
    s: int
    variant: str = "bcgsi+p-1s"


def factor_batched(items, stream=None):
    """Factor many independent problems (list of BatchItem); returns
    ([(Q, R)], codes, fail_blocks)."""
    import torch

    lib = load_library()
    probs = (Problem * len(items))()
    outs = []
    for i, it in enumerate(items):
        X = it.X
        m, n = X.shape
        prec = "fp32" if X.dtype == torch.float32 else "fp64"
        Q = empty_colmajor(m, n, X.dtype, X.device)
        R = empty_colmajor(n, n, torch.float64, X.device)
        outs.append((Q, R))
        probs[i] = Problem(m, n, it.s, VARIANTS[it.variant], PRECISIONS[prec], X.data_ptr(),
                           _colmajor_ld(X), Q.data_ptr(), _colmajor_ld(Q), R.data_ptr(),
                           _colmajor_ld(R), 0)
    nb = ctypes.c_size_t(0)
    _check(lib.bcgs_qr_batched_workspace_size(len(items), probs, ctypes.byref(nb)),
           "bcgs_qr_batched_workspace_size")
    dev = items[0].X.device if items else "cuda"
    ws = _workspace(nb.value, dev)
    sp = _stream_ptr(stream)
    _check(lib.bcgs_qr_factor_batched(len(items), probs, ws.data_ptr(), ws.numel(), sp),
           "bcgs_qr_factor_batched")
    codes = (ctypes.c_int32 * max(len(items), 1))()
    blocks = (ctypes.c_int32 * max(len(items), 1))()
    lib.bcgs_qr_batched_status(len(items), ws.data_ptr(), sp, codes, blocks)
    return outs, list(codes)[:len(items)], list(blocks)[:len(items)]


# ---------------------------------------------------------------- building blocks

def gram(A, B, stream=None):
    """C = A^T B (FP64)."""
    import torch

    lib = load_library()
    m, ka = A.shape
    kb = B.shape[1]
    C = empty_colmajor(ka, kb, torch.float64, A.device)
    nb = ctypes.c_size_t(0)
    _check(lib.bcgs_gram_workspace_size(m, ka, kb, ctypes.byref(nb)), "bcgs_gram_workspace_size")
    ws = _workspace(nb.value, A.device)
    _check(lib.bcgs_gram(m, ka, kb, A.data_ptr(), _colmajor_ld(A), B.data_ptr(), _colmajor_ld(B),
                         C.data_ptr(), _colmajor_ld(C), ws.data_ptr(), ws.numel(),
                         _stream_ptr(stream)), "bcgs_gram")
    return C


def gram_noalloc(A, B, C=None, stream=None):
    """C = A^T B through bcgs_gram_noalloc (no device memory is allocated by the
    library; C is allocated here unless given)."""
    import torch

    lib = load_library()
    m, ka = A.shape
    kb = B.shape[1]
    if C is None:
        C = empty_colmajor(ka, kb, torch.float64, A.device)
    _check(lib.bcgs_gram_noalloc(m, ka, kb, A.data_ptr(), _colmajor_ld(A), B.data_ptr(),
                                 _colmajor_ld(B), C.data_ptr(), _colmajor_ld(C),
                                 _stream_ptr(stream)), "bcgs_gram_noalloc")
    return C


def project(V, Q, C, T=None, stream=None):
    """W = (V - Q C) T^{-1} (FP64); Q may be None (c = 0)."""
    import torch

    lib = load_library()
    m, s = V.shape
    c = 0 if Q is None else Q.shape[1]
    W = empty_colmajor(m, s, torch.float64, V.device)
    rc = lib.bcgs_project(m, c, s, V.data_ptr(), _colmajor_ld(V),
                          Q.data_ptr() if c else None, _colmajor_ld(Q) if c else m,
                          C.data_ptr() if c else None, _colmajor_ld(C) if c else 1,
                          T.data_ptr() if T is not None else None,
                          _colmajor_ld(T) if T is not None else s,
                          W.data_ptr(), _colmajor_ld(W), _stream_ptr(stream))
    _check(rc, "bcgs_project")
    return W


def tsqr(A, stream=None):
    """[Q, R] = TSQR(A) (FP64); returns (Q, R, status, fail_block)."""
    import torch

    lib = load_library()
    m, s = A.shape
    Q = empty_colmajor(m, s, torch.float64, A.device)
    R = empty_colmajor(s, s, torch.float64, A.device)
    nb = ctypes.c_size_t(0)
    _check(lib.bcgs_tsqr_workspace_size(m, s, ctypes.byref(nb)), "bcgs_tsqr_workspace_size")
    ws = _workspace(nb.value, A.device)
    sp = _stream_ptr(stream)
    _check(lib.bcgs_tsqr(m, s, A.data_ptr(), _colmajor_ld(A), Q.data_ptr(), _colmajor_ld(Q),
                         R.data_ptr(), _colmajor_ld(R), ws.data_ptr(), ws.numel(), sp), "bcgs_tsqr")
    blk = ctypes.c_int32(0)
    code = lib.bcgs_qr_factor_status(ws.data_ptr(), sp, ctypes.byref(blk))
    return Q, R, code, blk.value


def chol(A, stream=None):
    """Upper Cholesky factor (FP64, s <= 64); returns (R, status)."""
    import torch

    lib = load_library()
    s = A.shape[0]
    R = empty_colmajor(s, s, torch.float64, A.device)
    ws = _workspace(256, A.device)
    sp = _stream_ptr(stream)
    _check(lib.bcgs_chol(s, A.data_ptr(), _colmajor_ld(A), R.data_ptr(), _colmajor_ld(R),
                         ws.data_ptr(), ws.numel(), sp), "bcgs_chol")
    blk = ctypes.c_int32(0)
    code = lib.bcgs_qr_factor_status(ws.data_ptr(), sp, ctypes.byref(blk))
    return R, code


OPT_GRAM_ENGINE, OPT_TC_MIN_ROWS = 1, 2
ENGINES = {"fp64": 0, "auto": 1, "tensor": 2}


def set_gram_engine(engine: str = "auto", min_rows: int | None = None):
    """Choose the Gram engine: "fp64" (FP64 pipe), "auto" (tensor cores for
    large shapes, the default) or "tensor" (whenever the shape allows)."""
    lib = load_library()
    _check(lib.bcgs_set_option(OPT_GRAM_ENGINE, ENGINES[engine]), "bcgs_set_option")
    if min_rows is not None:
        _check(lib.bcgs_set_option(OPT_TC_MIN_ROWS, int(min_rows)), "bcgs_set_option")


def get_gram_engine() -> str:
    v = load_library().bcgs_get_option(OPT_GRAM_ENGINE)
    return {0: "fp64", 1: "auto", 2: "tensor"}[int(v)]


def launch_count() -> int:
    return int(load_library().bcgs_launch_count())


def profile_enable(on: bool = True):
    lib = load_library()
    lib.bcgs_profile_reset()
    lib.bcgs_profile_enable(1 if on else 0)


def profile_read(cls: str):
    """(launches, total_ms, flops, bytes) of a kernel class since profile_enable."""
    lib = load_library()
    n = ctypes.c_int64(0)
    ms, fl, by = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(lib.bcgs_profile_read(PROFILE_CLASSES[cls], ctypes.byref(n), ctypes.byref(ms),
                                 ctypes.byref(fl), ctypes.byref(by)), "bcgs_profile_read")
    return n.value, ms.value, fl.value, by.value


def to_device_colmajor(x_np, device="cuda", dtype=None):
    """Copy a numpy (any layout) matrix to a column-major device tensor."""
    import numpy as np
    import torch

    arr = np.ascontiguousarray(np.asarray(x_np).T)
    t = torch.from_numpy(arr)
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device).T
