"""ctypes binding of libtucker.so: argument marshalling only.

Every computation happens in the CUDA library; this module converts torch
tensors (device or pinned/host memory) into the plain pointers and sizes of
the C ABI declared in include/tucker.h, and raises on a non-OK status.

Tensor convention: a tensor of size I_1 x ... x I_N is passed as any
contiguous torch tensor whose memory holds it with i_1 fastest (e.g. a torch
tensor of shape (I_N, ..., I_1)); ``dims`` gives (I_1, ..., I_N). Factor
matrices are returned as (I_n, R_n) tensors with column-major strides; the
core as a flat tensor in r_1-fastest order (``core.view(R_N, ..., R_1)``).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import torch

from . import build as _build

_LIB = None

TUCKER_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
                4: "numerical failure", 5: "timeout", 6: "unsupported", 7: "over budget"}
PROB = {"nearly_optimal": 0, "uniform": 1}
FORM = {"paper": 0, "range": 1, "related": 2}
PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16x1": 3}
FLAG_ASYNC = 1
FLAG_WORKLIST = 2


class TuckerError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(status, status)} (status {status})")


class Opts(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("form", C.c_int32), ("prec", C.c_int32), ("flags", C.c_uint32),
                ("alpha", C.c_double), ("stream", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("rel_error", C.POINTER(C.c_double)),
                ("sample_idx", C.POINTER(C.c_void_p))]


class ServerOpts(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("max_inflight", C.c_int32), ("budget_bytes", C.c_size_t),
                ("form", C.c_int32), ("prec", C.c_int32), ("tick_max", C.c_int32), ("tick_elems", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("which", C.c_int32), ("dt", C.c_int), ("A", C.c_void_p),
                ("dims", C.POINTER(C.c_int64)), ("N", C.c_int32), ("ranks", C.POINTER(C.c_int32)),
                ("P", C.c_int32), ("q", C.c_int32), ("c", C.c_int64), ("prob", C.c_int), ("seed", C.c_uint64),
                ("U", C.POINTER(C.c_void_p)), ("G", C.c_void_p)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("throughput", C.c_double), ("peak_bytes", C.c_size_t), ("peak_inflight", C.c_int32),
                ("ticks", C.c_uint64), ("tick_requests", C.c_uint64)]


_VP, _I64, _I32, _U64, _U32, _INT, _DBL = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_uint32, C.c_int, C.c_double
_P = C.POINTER
_SIGS = {
    "tucker_rthosvd": [_VP, _INT, _P(_I64), _INT, _P(_I32), _I32, _I32, _I64, _INT, _U64, _P(_VP), _VP, _P(Opts)],
    "tucker_rsthosvd": [_VP, _INT, _P(_I64), _INT, _P(_I32), _I32, _I32, _I64, _INT, _U64, _P(_VP), _VP, _P(Opts)],
    "tucker_workspace_size": [_INT, _INT, _P(_I64), _INT, _P(_I32), _I32, _I32, _I64, _P(Opts), _P(C.c_size_t)],
    "tucker_plan_describe": [_INT, _INT, _P(_I64), _INT, _P(_I32), _I32, _I32, _I64, _P(Opts), C.c_char_p,
                             C.c_size_t],
    "tucker_status_string": [_INT],
    "tucker_last_cuda_error": [],
    "tucker_last_device_status": [],
    "tucker_gaussian": [_VP, _INT, _I64, _I64, _U64, _U32, _P(Opts)],
    "tucker_power_step": [_VP, _INT, _P(_I64), _INT, _INT, _VP, _I64, _VP, _P(Opts)],
    "tucker_range_sketch": [_VP, _INT, _P(_I64), _INT, _INT, _I64, _U64, _VP, _P(Opts)],
    "tucker_fiber_norms": [_VP, _INT, _P(_I64), _INT, _INT, _VP, _P(Opts)],
    "tucker_fiber_norms12": [_VP, _INT, _P(_I64), _INT, _VP, _VP, _P(Opts)],
    "tucker_fiber_norms123": [_VP, _INT, _P(_I64), _INT, _VP, _VP, _VP, _P(Opts)],
    "tucker_fiber_norms123_workspace_size": [_P(_I64), _INT, _P(C.c_size_t)],
    "tucker_quantize_weights": [_VP, _I64, _INT, _VP, _P(Opts)],
    "tucker_sample_fibers": [_VP, _I64, _I64, _U64, _INT, _VP, _VP, _P(Opts)],
    "tucker_gather_fibers": [_VP, _INT, _P(_I64), _INT, _INT, _VP, _VP, _I64, _VP, _P(Opts)],
    "tucker_leading_factor": [_VP, _INT, _I64, _I64, _I64, _VP, _P(Opts)],
    "tucker_ttm": [_VP, _INT, _P(_I64), _INT, _INT, _VP, _I64, _INT, _VP, _P(Opts)],
    "tucker_relative_error": [_VP, _INT, _P(_I64), _INT, _P(_I32), _P(_VP), _VP, _P(_DBL), _P(Opts)],
    "tucker_power_step_noalloc": [_VP, _INT, _P(_I64), _INT, _INT, _VP, _I64, _VP, _P(Opts)],
    "tucker_quantize_weights_max": [_VP, _I64, _DBL, _VP, _P(Opts)],
    "tucker_sample_fibers_slab": [_VP, _I64, _I64, _U64, _INT, _U64, _U64, _I64, _VP, _VP, _P(Opts)],
    "tucker_cholqr": [_VP, _INT, _I64, _I64, _VP, _VP, _P(Opts)],
    "tucker_leading_factor_chain": [_VP, _INT, _I64, _I64, _I64, _VP, _INT, _VP, _P(Opts)],
    "tucker_sample_factor": [_VP, _INT, _I64, _I64, _I64, _I32, _I32, _U64, _INT, _VP, _P(Opts)],
    "tucker_check_wait_timeout": [_I32, _P(Opts)],
    "tucker_gram": [_VP, _INT, _P(_I64), _INT, _INT, _VP, _P(Opts)],
    "tucker_rsthosvd_adaptive": [_VP, _INT, _P(_I64), _INT, _DBL, _I32, _I32, _U64, _P(_VP), _VP, _P(_I32),
                                 _P(Opts)],
    "tucker_server_create": [_P(ServerOpts), _P(_VP)],
    "tucker_server_submit": [_VP, _P(Request), _P(_U64)],
    "tucker_server_wait": [_VP, _U64, _I64, _P(_INT)],
    "tucker_server_stats_get": [_VP, _P(ServerStats)],
    "tucker_server_destroy": [_VP],
    "tucker_batch_workspace_size": [_INT, _VP, _P(Opts), _P(C.c_size_t)],
    "tucker_batch_run": [_INT, _VP, _P(Opts)],
    "tucker_batch_describe": [_INT, _VP, _P(Opts), C.c_char_p, C.c_size_t],
    "tucker_autotune_enable": [_INT],
    "tucker_autotune_count": [],
    "tucker_autotune_entry": [_I64],
    "tucker_launch_count": [],
    "tucker_profile_enable": [_INT],
    "tucker_profile_read": [_INT, _P(_I64), _P(_DBL), _P(_DBL), _P(_DBL)],
}
_RESTYPES = {"tucker_status_string": C.c_char_p, "tucker_launch_count": C.c_int64,
             "tucker_last_cuda_error": C.c_char_p, "tucker_autotune_count": C.c_int64,
             "tucker_autotune_entry": C.c_char_p}
KERNEL_CLASSES = {"power": 0, "ttm": 1, "gather": 2, "norms": 3, "extract": 4, "sample": 5, "power_bf16": 6,
                  "power_tf32": 7, "ttm_bf16": 8, "power_bf16x1": 9, "ttm_wide": 10, "power_wide1": 11,
                  "power_wide2": 12, "range_wide": 13, "gram_wide": 14, "worklist": 15}


def lib():
    """The loaded library; builds it first if it is missing. Raises if it cannot."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not found at {path}")
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, C.c_int)
        _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIGS)


def _check(fn: str, status: int):
    if status != TUCKER_OK:
        err = TuckerError(fn, status)
        if status in (2, 3):
            err.args = (err.args[0] + " [" + lib().tucker_last_cuda_error().decode() + "]",)
        raise err


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return 0
    if t.dtype == torch.float64:
        return 1
    raise TypeError(f"unsupported dtype {t.dtype}")


def _i64(xs) -> C.Array:
    return (C.c_int64 * len(xs))(*[int(x) for x in xs])


def _i32(xs) -> C.Array:
    return (C.c_int32 * len(xs))(*[int(x) for x in xs])


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream or None
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def make_opts(form="paper", prec="fp32", alpha=0.0, stream=None, workspace: Optional[torch.Tensor] = None,
              rel_error: Optional[C.c_double] = None, sample_idx=None, flags=0) -> Opts:
    o = Opts()
    o.struct_size = C.sizeof(Opts)
    o.form = FORM[form]
    o.prec = PREC[prec]
    o.flags = flags
    o.alpha = float(alpha)
    o.stream = _stream_handle(stream)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    if rel_error is not None:
        o.rel_error = C.pointer(rel_error)
    if sample_idx is not None:
        arr = (C.c_void_p * len(sample_idx))(*[t.data_ptr() for t in sample_idx])
        o._keep = arr
        o.sample_idx = C.cast(arr, C.POINTER(C.c_void_p))
    return o


def _ptr(t: torch.Tensor) -> int:
    if not t.is_contiguous() and not (t.dim() == 2 and t.stride(0) == 1):
        raise ValueError("tensor memory must be contiguous")
    return t.data_ptr()


def _problem(which: str, A: torch.Tensor, dims, ranks):
    """Checks one decomposition's arguments before they reach the C ABI, which
    reads N extents and N ranks and the tensor as dense memory, i_1 fastest.
    Returns (dims, ranks) as int lists."""
    if which not in ("T", "ST"):
        raise ValueError(f"which must be 'T' or 'ST', not {which!r}")
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    if not dims or len(ranks) != len(dims):
        raise ValueError("dims and ranks must be non-empty and of equal length")
    _dt(A)
    if not A.is_contiguous():
        raise ValueError("A must be contiguous (dense, i_1 fastest)")
    if A.numel() != int(torch.tensor(dims).prod()):
        raise ValueError("A.numel() must equal prod(dims)")
    return dims, ranks


def _view(A: torch.Tensor, dims, mode: int):
    """Checks a mode view (dense tensor, N extents, 0 <= mode < N) before the C
    ABI reads prod(dims) entries; returns dims as ints."""
    dims = [int(d) for d in dims]
    _dt(A)
    if not dims or not 0 <= int(mode) < len(dims):
        raise ValueError("mode must index one of the N extents")
    if not A.is_contiguous() or A.numel() != int(torch.tensor(dims).prod()):
        raise ValueError("A must be a dense tensor (i_1 fastest) of prod(dims) entries")
    return dims


def _colmajor_rows(X: torch.Tensor, rows: int, dtype, name: str) -> torch.Tensor:
    """X as a column-major 2-D matrix with `rows` rows and the given dtype (a
    copy when its strides are not column-major)."""
    if X.dim() != 2 or X.shape[0] != rows or X.dtype != dtype:
        raise ValueError(f"{name} must be a {rows} x k matrix of dtype {dtype}")
    if X.shape[1] > 1 and X.stride(0) != 1 or X.shape[1] > 1 and rows > 1 and X.stride(1) != rows:
        X = X.t().contiguous().t()
    return X


def _outputs(out, A: torch.Tensor, dims, ranks, device):
    """Caller-supplied (U list, G) checked against the ABI's layouts (U_n
    column-major I_n x R_n, G dense with prod(ranks) entries, A's dtype), or
    new tensors on device."""
    if out is None:
        U = [factor_tensor(I, R, A.dtype, device) for I, R in zip(dims, ranks)]
        G = torch.empty(int(torch.tensor(ranks).prod()), dtype=A.dtype, device=device)
        return U, G
    U, G = out
    if len(U) != len(dims):
        raise ValueError("out must hold one factor per mode")
    for u, I, R in zip(U, dims, ranks):
        if tuple(u.shape) != (I, R) or u.dtype != A.dtype or (R > 1 and u.stride(0) != 1) or \
                (I > 1 and R > 1 and u.stride(1) != I):
            raise ValueError("each U_n must be a column-major I_n x R_n tensor of A's dtype")
    if G.numel() != int(torch.tensor(ranks).prod()) or G.dtype != A.dtype or not G.is_contiguous():
        raise ValueError("G must be a contiguous tensor of prod(ranks) entries of A's dtype")
    return list(U), G


def factor_tensor(I: int, R: int, dtype, device) -> torch.Tensor:
    """An (I, R) tensor with column-major strides (the ABI's matrix layout)."""
    return torch.empty((R, I), dtype=dtype, device=device).t()


def workspace_size(which: str, dims, ranks, P=10, q=1, c=0, dtype=torch.float32, **kw) -> int:
    if which not in ("T", "ST"):
        raise ValueError(f"which must be 'T' or 'ST', not {which!r}")
    if len(ranks) != len(dims):
        raise ValueError("dims and ranks must be of equal length")
    n = C.c_size_t(0)
    o = make_opts(**kw)
    st = lib().tucker_workspace_size(0 if which == "T" else 1, 0 if dtype == torch.float32 else 1,
                                     _i64(dims), len(dims), _i32(ranks), int(P), int(q), int(c), C.byref(o),
                                     C.byref(n))
    _check("tucker_workspace_size", st)
    return int(n.value)


def batch_describe(specs, dtype=torch.float32, form="paper", prec="fp32") -> str:
    """The work list a batch would run (tucker_batch_describe with
    TUCKER_FLAG_WORKLIST): one line per step or grouped orthonormalisation.
    ``specs``: dicts with which, dims, ranks and optionally P, q, c, seed; host
    only (no buffers are touched)."""
    arr = (Request * len(specs))()
    keep = []
    for k, r in enumerate(specs):
        dims, ranks = list(r["dims"]), list(r["ranks"])
        d64, r32 = _i64(dims), _i32(ranks)
        Up = (C.c_void_p * len(dims))(*([256] * len(dims)))
        arr[k] = Request(C.sizeof(Request), 0 if r["which"] == "T" else 1, 0 if dtype == torch.float32 else 1, 256,
                         d64, len(dims), r32, int(r.get("P", 5)), int(r.get("q", 1)), int(r.get("c", 0)),
                         PROB[r.get("prob", "uniform")], int(r.get("seed", 0)), Up, 256)
        keep.append((d64, r32, Up))
    buf = C.create_string_buffer(1 << 16)
    o = make_opts(form=form, prec=prec, flags=FLAG_WORKLIST)
    _check("tucker_batch_describe", lib().tucker_batch_describe(len(specs), C.cast(arr, C.c_void_p), C.byref(o), buf,
                                                                len(buf)))
    return buf.value.decode()


def plan_describe(which: str, dims, ranks, P=10, q=1, c=0, dtype=torch.float32, **kw) -> str:
    """The arithmetic each mode of a driver call takes (tucker_plan_describe),
    one line per mode; host only."""
    if which not in ("T", "ST"):
        raise ValueError(f"which must be 'T' or 'ST', not {which!r}")
    if len(ranks) != len(dims):
        raise ValueError("dims and ranks must be of equal length")
    buf = C.create_string_buffer(256 * max(1, len(dims)) + 1)
    o = make_opts(**kw)
    _check("tucker_plan_describe",
           lib().tucker_plan_describe(0 if which == "T" else 1, 0 if dtype == torch.float32 else 1, _i64(dims),
                                      len(dims), _i32(ranks), int(P), int(q), int(c), C.byref(o), buf,
                                      len(buf)))
    return buf.value.decode()


def decompose(which: str, A: torch.Tensor, dims: Sequence[int], ranks: Sequence[int], P=10, q=1, c=0,
              prob="uniform", seed=0, form="paper", prec="fp32", alpha=0.0, stream=None, workspace=None,
              want_rel_error=False, want_samples=False, out=None, flags=0):
    """Randomized T-HOSVD (which='T', Algorithms 1/4) or ST-HOSVD (which='ST',
    Algorithms 2/5). Returns (U list, G flat[, rel_error][, sample indices])."""
    dims, ranks = _problem(which, A, dims, ranks)
    N = len(dims)
    dev = A.device
    U, G = _outputs(out, A, dims, ranks, dev)
    re = C.c_double(float("nan")) if want_rel_error else None
    samples = None
    if want_samples:
        samples = []
        # sizes follow T_n = min(c, J_n) with J_n of the tensor each mode works on
        cur = list(dims)
        for n in range(N):
            J = 1
            for m in range(N):
                if m != n:
                    J *= cur[m]
            T = min(c, J) if c > 0 else (int(-(-alpha * J // 1)) if alpha > 0 else 0)
            samples.append(torch.full((max(T, 1),), -1, dtype=torch.int64, device=dev))
            if which == "ST":
                cur[n] = ranks[n]
    o = make_opts(form, prec, alpha, stream, workspace, re, samples, flags)
    Uptrs = (C.c_void_p * N)(*[u.data_ptr() for u in U])
    fn = lib().tucker_rthosvd if which == "T" else lib().tucker_rsthosvd
    st = fn(A.data_ptr(), _dt(A), _i64(dims), N, _i32(ranks), int(P), int(q), int(c), PROB[prob],
            C.c_uint64(int(seed) & (2**64 - 1)), Uptrs, G.data_ptr(), C.byref(o))
    _check("tucker_rthosvd" if which == "T" else "tucker_rsthosvd", st)
    res = [U, G]
    if want_rel_error:
        res.append(re.value)
    if want_samples:
        res.append(samples)
    return tuple(res)


def rthosvd(A, dims, ranks, **kw):
    return decompose("T", A, dims, ranks, **kw)


def rsthosvd(A, dims, ranks, **kw):
    return decompose("ST", A, dims, ranks, **kw)


def rsthosvd_adaptive(A, dims, eps, q=1, L0=8, seed=0, form="paper", prec="fp32", stream=None,
                      want_rel_error=False):
    """tucker_rsthosvd_adaptive (Problem 2): ranks chosen so that the relative
    error is at most eps. A is a device tensor. Returns (U list of I_n x r_n,
    G flat of prod(r_n), ranks[, rel_error])."""
    dims = [int(d) for d in dims]
    N = len(dims)
    if A.numel() != math.prod(dims):
        raise ValueError("A must hold prod(dims) elements")
    dev = A.device
    Ubuf = [factor_tensor(I, I, A.dtype, dev) for I in dims]
    Gbuf = torch.empty(math.prod(dims), dtype=A.dtype, device=dev)
    ranks = (C.c_int32 * N)()
    re = C.c_double(float("nan")) if want_rel_error else None
    o = make_opts(form, prec, 0.0, stream, None, re, None, 0)
    Uptrs = (C.c_void_p * N)(*[u.data_ptr() for u in Ubuf])
    _check("tucker_rsthosvd_adaptive",
           lib().tucker_rsthosvd_adaptive(A.data_ptr(), _dt(A), _i64(dims), N, float(eps), int(q), int(L0),
                                          C.c_uint64(int(seed) & (2**64 - 1)), Uptrs, Gbuf.data_ptr(), ranks,
                                          C.byref(o)))
    r = [int(x) for x in ranks]
    U = [u[:, :k] for u, k in zip(Ubuf, r)]
    G = Gbuf[:math.prod(r)]
    res = (U, G, r)
    return res + (re.value,) if want_rel_error else res


def gram(A, dims, mode, stream=None, prec="bf16"):
    """tucker_gram: G = A_(n) A_(n)^T (I_n x I_n) in one tensor-core pass (Strategy B)."""
    dims = _view(A, dims, mode)
    I = dims[mode]
    G = factor_tensor(I, I, A.dtype, A.device)
    o = make_opts(stream=stream, prec=prec)
    _check("tucker_gram", lib().tucker_gram(A.data_ptr(), _dt(A), _i64(dims), len(dims), mode, G.data_ptr(),
                                            C.byref(o)))
    return G


def check_wait_timeout(iters=1000, stream=None) -> int:
    """tucker_check_wait_timeout: the status (an int, not raised) of a bounded
    device wait that nothing completes; TUCKER_ERR_TIMEOUT (5) when the path works."""
    o = make_opts(stream=stream)
    return int(lib().tucker_check_wait_timeout(int(iters), C.byref(o)))


def last_device_status() -> int:
    return int(lib().tucker_last_device_status())


# ---------------------------------------------------------------- step entry points
def gaussian(rows, cols, seed, stream_id, dtype=torch.float32, device="cuda", stream=None):
    out = factor_tensor(rows, cols, dtype, device)
    o = make_opts(stream=stream)
    _check("tucker_gaussian", lib().tucker_gaussian(out.data_ptr(), _dt(out), rows, cols,
                                                    C.c_uint64(seed), C.c_uint32(stream_id), C.byref(o)))
    return out


def power_step(A, dims, mode, X, stream=None, prec="fp32"):
    """X_out = A_(n) (A_(n)^T X) (one power step of Strategy A); prec "tf32" /
    "bf16" run it on the tensor cores (see tucker_power_step)."""
    dims = _view(A, dims, mode)
    I = dims[mode]
    X = _colmajor_rows(X, I, A.dtype, "X")
    L = X.shape[1]
    out = factor_tensor(I, L, A.dtype, A.device)
    o = make_opts(stream=stream, prec=prec)
    _check("tucker_power_step", lib().tucker_power_step(A.data_ptr(), _dt(A), _i64(dims), len(dims), mode,
                                                        X.data_ptr(), L, out.data_ptr(), C.byref(o)))
    return out


def range_sketch(A, dims, mode, L, seed, stream=None, prec="fp32"):
    """Y = A_(n) Omega, Omega J_n x L Gaussian from the Philox stream; prec other
    than "fp32" runs it on the tensor cores (contiguous fibers)."""
    dims = _view(A, dims, mode)
    out = factor_tensor(dims[mode], L, A.dtype, A.device)
    o = make_opts(stream=stream, prec=prec)
    _check("tucker_range_sketch", lib().tucker_range_sketch(A.data_ptr(), _dt(A), _i64(dims), len(dims), mode, L,
                                                            C.c_uint64(seed), out.data_ptr(), C.byref(o)))
    return out


def fiber_norms(A, dims, mode, stream=None):
    dims = _view(A, dims, mode)
    J = 1
    for m, d in enumerate(dims):
        if m != mode:
            J *= d
    w = torch.empty(J, dtype=torch.float64, device=A.device)
    o = make_opts(stream=stream)
    _check("tucker_fiber_norms", lib().tucker_fiber_norms(A.data_ptr(), _dt(A), _i64(dims), len(dims), mode,
                                                          w.data_ptr(), C.byref(o)))
    return w


def fiber_norms12(A, dims, stream=None):
    """tucker_fiber_norms12: the mode-1 and mode-2 fiber norms from one pass over A."""
    dims = _view(A, dims, 1)
    E = 1
    for d in dims:
        E *= d
    w1 = torch.empty(E // dims[0], dtype=torch.float64, device=A.device)
    w2 = torch.empty(E // dims[1], dtype=torch.float64, device=A.device)
    o = make_opts(stream=stream)
    _check("tucker_fiber_norms12", lib().tucker_fiber_norms12(A.data_ptr(), _dt(A), _i64(dims), len(dims),
                                                              w1.data_ptr(), w2.data_ptr(), C.byref(o)))
    return w1, w2


def fiber_norms123(A, dims, stream=None, workspace=None):
    """tucker_fiber_norms123: the three modes' fiber norms of an order-3 tensor from one
    pass over A (the partials in ``workspace`` if given, else in a block the call
    allocates)."""
    dims = _view(A, dims, 2)
    if len(dims) != 3:
        raise ValueError("fiber_norms123 takes an order-3 tensor")
    I1, I2, I3 = dims
    w1 = torch.empty(I2 * I3, dtype=torch.float64, device=A.device)
    w2 = torch.empty(I1 * I3, dtype=torch.float64, device=A.device)
    w3 = torch.empty(I1 * I2, dtype=torch.float64, device=A.device)
    o = make_opts(stream=stream, workspace=workspace)
    _check("tucker_fiber_norms123", lib().tucker_fiber_norms123(A.data_ptr(), _dt(A), _i64(dims), 3, w1.data_ptr(),
                                                                w2.data_ptr(), w3.data_ptr(), C.byref(o)))
    return w1, w2, w3


def fiber_norms123_workspace_size(dims):
    n = C.c_size_t(0)
    _check("tucker_fiber_norms123_workspace_size",
           lib().tucker_fiber_norms123_workspace_size(_i64(dims), len(dims), C.byref(n)))
    return n.value


def quantize_weights(w, prob="nearly_optimal", stream=None):
    if w.dtype != torch.float64 or not w.is_contiguous():
        raise ValueError("w must be a contiguous float64 vector")
    W = torch.empty(w.numel(), dtype=torch.int64, device=w.device)   # uint64 bits
    o = make_opts(stream=stream)
    _check("tucker_quantize_weights", lib().tucker_quantize_weights(w.data_ptr(), w.numel(), PROB[prob],
                                                                    W.data_ptr(), C.byref(o)))
    return W


def sample_fibers(W, T, seed, mode, stream=None):
    if W.dtype != torch.int64 or not W.is_contiguous():
        raise ValueError("W must be a contiguous int64 vector (the uint64 weights' bits)")
    idx = torch.empty(max(T, 1), dtype=torch.int64, device=W.device)
    scale = torch.empty(max(T, 1), dtype=torch.float64, device=W.device)
    o = make_opts(stream=stream)
    _check("tucker_sample_fibers", lib().tucker_sample_fibers(W.data_ptr(), W.numel(), T, C.c_uint64(seed), mode,
                                                              idx.data_ptr(), scale.data_ptr(), C.byref(o)))
    return idx[:T], scale[:T]


def gather_fibers(A, dims, mode, idx, scale, stream=None):
    """C' = A_(n) S: column t is scale[t] times fiber idx[t]; every idx[t] must
    be below J_n (tucker_sample_fibers' indices always are)."""
    dims = _view(A, dims, mode)
    if idx.dtype != torch.int64 or scale.dtype != torch.float64 or idx.numel() != scale.numel() or \
            not idx.is_contiguous() or not scale.is_contiguous():
        raise ValueError("idx (int64) and scale (float64) must be contiguous vectors of equal length")
    T = idx.numel()
    out = factor_tensor(dims[mode], max(T, 1), A.dtype, A.device)
    o = make_opts(stream=stream)
    _check("tucker_gather_fibers", lib().tucker_gather_fibers(A.data_ptr(), _dt(A), _i64(dims), len(dims), mode,
                                                              idx.data_ptr(), scale.data_ptr(), T, out.data_ptr(),
                                                              C.byref(o)))
    return out[:, :T]


def quantize_weights_max(w, wmax, stream=None):
    """tucker_quantize_weights_max: integer weights against a given largest weight."""
    if w.dtype != torch.float64 or not w.is_contiguous():
        raise ValueError("w must be a contiguous float64 vector")
    W = torch.empty(w.numel(), dtype=torch.int64, device=w.device)   # uint64 bits
    o = make_opts(stream=stream)
    _check("tucker_quantize_weights_max", lib().tucker_quantize_weights_max(w.data_ptr(), w.numel(), float(wmax),
                                                                            W.data_ptr(), C.byref(o)))
    return W


def sample_fibers_slab(W, T, seed, mode, S_offset, S_total, fiber_offset, stream=None):
    """tucker_sample_fibers_slab: the draws of one slab (idx -1 / scale 0 elsewhere)."""
    if W.dtype != torch.int64 or not W.is_contiguous():
        raise ValueError("W must be a contiguous int64 vector (the uint64 weights' bits)")
    idx = torch.empty(max(T, 1), dtype=torch.int64, device=W.device)
    scale = torch.empty(max(T, 1), dtype=torch.float64, device=W.device)
    o = make_opts(stream=stream)
    _check("tucker_sample_fibers_slab", lib().tucker_sample_fibers_slab(
        W.data_ptr(), W.numel(), T, C.c_uint64(seed), mode, C.c_uint64(S_offset), C.c_uint64(S_total),
        int(fiber_offset), idx.data_ptr(), scale.data_ptr(), C.byref(o)))
    return idx[:T], scale[:T]


def cholqr(X, stream=None):
    """tucker_cholqr: (Q, F) with X = Q F, F the packed triangular factor (L*L doubles)."""
    I, L = X.shape
    if X.stride(0) != 1:
        X = X.t().contiguous().t()
    Q = factor_tensor(I, L, X.dtype, X.device)
    F = torch.empty(L * L, dtype=torch.float64, device=X.device)
    o = make_opts(stream=stream)
    _check("tucker_cholqr", lib().tucker_cholqr(X.data_ptr(), _dt(X), I, L, Q.data_ptr(), F.data_ptr(), C.byref(o)))
    return Q, F


def leading_factor_chain(X, R, factors, stream=None):
    """tucker_leading_factor_chain: U of C = X F_{k-1} ... F_0 (factors from cholqr, F_0 first)."""
    I, L = X.shape
    if X.stride(0) != 1:
        X = X.t().contiguous().t()
    U = factor_tensor(I, R, X.dtype, X.device)
    Fs = torch.cat([f.reshape(-1) for f in factors]) if factors else torch.empty(1, dtype=torch.float64,
                                                                                   device=X.device)
    o = make_opts(stream=stream)
    _check("tucker_leading_factor_chain", lib().tucker_leading_factor_chain(
        X.data_ptr(), _dt(X), I, L, R, Fs.data_ptr(), len(factors), U.data_ptr(), C.byref(o)))
    return U


def sample_factor(Cp, R, P, q, seed, mode, stream=None):
    """tucker_sample_factor: the factor of Algorithms 4/5 from a gathered sample C' (I x T)."""
    I, T = Cp.shape
    if Cp.stride(0) != 1:
        Cp = Cp.t().contiguous().t()
    U = factor_tensor(I, R, Cp.dtype, Cp.device)
    o = make_opts(stream=stream)
    _check("tucker_sample_factor", lib().tucker_sample_factor(Cp.data_ptr(), _dt(Cp), I, T, R, int(P), int(q),
                                                              C.c_uint64(int(seed) & (2**64 - 1)), int(mode),
                                                              U.data_ptr(), C.byref(o)))
    return U


def leading_factor(Cm, R, stream=None):
    I, L = Cm.shape
    if Cm.stride(0) != 1:
        Cm = Cm.t().contiguous().t()
    U = factor_tensor(I, R, Cm.dtype, Cm.device)
    o = make_opts(stream=stream)
    _check("tucker_leading_factor", lib().tucker_leading_factor(Cm.data_ptr(), _dt(Cm), I, L, R, U.data_ptr(),
                                                                C.byref(o)))
    return U


def ttm(A, dims, mode, M, transpose=False, stream=None, prec="fp32"):
    """A x_n M (transpose=False, M is K x I_n) or A x_n M^T (transpose=True, M is I_n x K);
    M must have column-major strides. prec "bf16"/"tf32": split-bf16 tensor cores
    (contiguous fibers only)."""
    dims = _view(A, dims, mode)
    if M.dim() != 2 or M.dtype != A.dtype or M.shape[0 if transpose else 1] != dims[mode]:
        raise ValueError("M must be I_n x K (transpose) or K x I_n, of A's dtype")
    K = M.shape[1] if transpose else M.shape[0]
    if M.stride(0) != 1:
        M = M.t().contiguous().t()
    out_dims = list(dims)
    out_dims[mode] = K
    n = 1
    for d in out_dims:
        n *= d
    out = torch.empty(n, dtype=A.dtype, device=A.device)
    o = make_opts(stream=stream, prec=prec)
    _check("tucker_ttm", lib().tucker_ttm(A.data_ptr(), _dt(A), _i64(dims), len(dims), mode, M.data_ptr(), K,
                                          int(transpose), out.data_ptr(), C.byref(o)))
    return out


def relative_error(A, dims, ranks, U, G, stream=None):
    dims, ranks = _problem("T", A, dims, ranks)
    U, G = _outputs((U, G), A, dims, ranks, A.device)
    re = C.c_double(0.0)
    o = make_opts(stream=stream)
    Up = (C.c_void_p * len(U))(*[u.data_ptr() for u in U])
    _check("tucker_relative_error", lib().tucker_relative_error(A.data_ptr(), _dt(A), _i64(dims), len(dims),
                                                                _i32(ranks), Up, G.data_ptr(), C.byref(re),
                                                                C.byref(o)))
    return re.value


# ---------------------------------------------------------------- measurement
def autotune_enable(on: bool = True):
    """Turn the library's autotuner on or off (tucker_autotune_enable)."""
    _check("tucker_autotune_enable", lib().tucker_autotune_enable(1 if on else 0))


def autotune_entries():
    """One line per tuned shape class: the class, its choice, the candidates' times."""
    L = lib()
    return [L.tucker_autotune_entry(k).decode() for k in range(L.tucker_autotune_count())]


def launch_count() -> int:
    """Kernel launches the library has made so far in this process."""
    return int(lib().tucker_launch_count())


def profile_enable(on: bool = True):
    _check("tucker_profile_enable", lib().tucker_profile_enable(int(bool(on))))


def profile_read(kernel: str):
    """(launches, total_ms, algorithmic bytes, flops) since profile_enable(True)."""
    n = C.c_int64(0)
    ms, b, f = C.c_double(0), C.c_double(0), C.c_double(0)
    _check("tucker_profile_read", lib().tucker_profile_read(KERNEL_CLASSES[kernel], C.byref(n), C.byref(ms),
                                                            C.byref(b), C.byref(f)))
    return int(n.value), ms.value, b.value, f.value


def power_step_noalloc(A, dims, mode, X, stream=None):
    """tucker_power_step_noalloc: the power step with the library's fixed scratch
    block instead of an allocation (see include/tucker.h)."""
    dims = _view(A, dims, mode)
    I = dims[mode]
    X = _colmajor_rows(X, I, A.dtype, "X")
    L = X.shape[1]
    out = factor_tensor(I, L, A.dtype, A.device)
    o = make_opts(stream=stream)
    _check("tucker_power_step_noalloc", lib().tucker_power_step_noalloc(A.data_ptr(), _dt(A), _i64(dims), len(dims),
                                                                        mode, X.data_ptr(), L, out.data_ptr(),
                                                                        C.byref(o)))
    return out


class Server:
    """Request loop of the C library (tucker_server_*): submit decompositions of
    any order, size and rank; they are admitted against ``budget_bytes`` of
    device memory and run concurrently on up to ``max_inflight`` streams.

    ``submit`` takes the tensor (device or host, pinned for overlap) and returns
    a ticket; the output tensors are created here on ``out_device`` unless given.
    The binding keeps every tensor of a request alive until ``wait`` has seen it
    complete. Requests overlap only as far as CUDA's hardware work queues allow:
    set ``CUDA_DEVICE_MAX_CONNECTIONS`` (8 by default) to at least
    ``max_inflight`` before the process first uses the GPU. ``tick_max`` > 1
    (paper form, FP32 arithmetic) admits up to that many consecutive requests
    of at most ``tick_elems`` tensor elements that the work list takes as one
    work-list batch on one stream; the library refuses ticks (unsupported), as
    the work-list path is not run."""

    def __init__(self, budget_bytes: int, max_inflight: int = 8, form="paper", prec="fp32", tick_max: int = 0,
                 tick_elems: int = 1 << 22):
        o = ServerOpts(C.sizeof(ServerOpts), int(max_inflight), int(budget_bytes), FORM[form], PREC[prec],
                       int(tick_max), int(tick_elems))
        h = C.c_void_p()
        _check("tucker_server_create", lib().tucker_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, which: str, A: torch.Tensor, dims, ranks, P=5, q=1, c=0, prob="uniform", seed=0,
               out=None, out_device=None):
        dims, ranks = _problem(which, A, dims, ranks)
        N = len(dims)
        dev = A.device if out_device is None else torch.device(out_device)
        U, G = _outputs(out, A, dims, ranks, dev)
        d64, r32 = _i64(dims), _i32(ranks)
        Up = (C.c_void_p * N)(*[u.data_ptr() for u in U])
        req = Request(C.sizeof(Request), 0 if which == "T" else 1, _dt(A), A.data_ptr(), d64, N, r32, int(P), int(q),
                      int(c), PROB[prob], int(seed) & (2**64 - 1), Up, G.data_ptr())
        t = C.c_uint64(0)
        _check("tucker_server_submit", lib().tucker_server_submit(self._h, C.byref(req), C.byref(t)))
        self._live[t.value] = (A, U, G)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(U, G) once the request has completed; raises on its failure, or
        TuckerError(status 5) if it has not completed within timeout_ms."""
        res = C.c_int(0)
        _check("tucker_server_wait", lib().tucker_server_wait(self._h, int(ticket), int(timeout_ms), C.byref(res)))
        A, U, G = self._live.pop(ticket)
        _check(f"request {ticket}", res.value)
        return U, G

    def stats(self) -> dict:
        st = ServerStats()
        _check("tucker_server_stats_get", lib().tucker_server_stats_get(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            _check("tucker_server_destroy", lib().tucker_server_destroy(self._h))
            self._h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent decompositions launched as one CUDA graph
    (tucker_batch_*). ``requests`` is a list of dicts with keys which ("T" or
    "ST"), A (device tensor), dims, ranks and optionally P, q, c, prob, seed.
    Outputs and the workspace are allocated here, once; ``run`` launches the
    whole batch (captured on the first run, replayed afterwards) and returns the
    list of (U, G). Inputs may be rewritten in place between runs. Each request
    runs on its own stream of the graph; with CUDA's default of 8 hardware work
    queues (``CUDA_DEVICE_MAX_CONNECTIONS``, read when the process first uses
    the GPU) streams sharing a queue wait on one another, so set it to 32 for
    batches of more than 8 requests. ``worklist=True`` asks for the work-list
    path (TUCKER_FLAG_WORKLIST), which the library plans but does not run: ``run``
    then raises TuckerError (unsupported); ``batch_describe`` shows its plan."""

    def __init__(self, requests, form="paper", prec="fp32", worklist=False):
        self._keep = []
        self.outputs = []
        self._offsets = []
        off = 0
        arr = (Request * len(requests))()
        for k, r in enumerate(requests):
            A = r["A"]
            dims, ranks = _problem(r["which"], A, r["dims"], r["ranks"])
            U, G = _outputs(None, A, dims, ranks, A.device)
            d64, r32 = _i64(dims), _i32(ranks)
            Up = (C.c_void_p * len(dims))(*[u.data_ptr() for u in U])
            arr[k] = Request(C.sizeof(Request), 0 if r["which"] == "T" else 1, _dt(A), A.data_ptr(), d64, len(dims),
                             r32, int(r.get("P", 5)), int(r.get("q", 1)), int(r.get("c", 0)),
                             PROB[r.get("prob", "uniform")], int(r.get("seed", 0)) & (2**64 - 1), Up, G.data_ptr())
            self._keep.append((A, d64, r32, Up))
            self.outputs.append((U, G))
            self._offsets.append(off)
            off += (workspace_size(r["which"], dims, ranks, P=int(r.get("P", 5)), q=int(r.get("q", 1)),
                                   c=int(r.get("c", 0)), dtype=A.dtype, form=form, prec=prec) + 255) // 256 * 256
        self._reqs = arr
        self._n = len(requests)
        self._form, self._prec = form, prec
        self._flags = FLAG_WORKLIST if worklist else 0
        n = C.c_size_t(0)
        o = make_opts(form=form, prec=prec, flags=self._flags)
        _check("tucker_batch_workspace_size",
               lib().tucker_batch_workspace_size(self._n, C.cast(arr, C.c_void_p), C.byref(o), C.byref(n)))
        self.workspace = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=requests[0]["A"].device)

    def run(self, stream=None, sync=True):
        o = make_opts(form=self._form, prec=self._prec, stream=stream, workspace=self.workspace,
                      flags=self._flags | (0 if sync else FLAG_ASYNC))
        _check("tucker_batch_run", lib().tucker_batch_run(self._n, C.cast(self._reqs, C.c_void_p), C.byref(o)))
        return self.outputs

    def status(self):
        """Each request's device status word (0 = success; bit 0 numerical
        failure, bit 1 a bounded wait timed out) as left by the last run; read
        once that run has completed."""
        w = self.workspace
        return [int(w[o:o + 4].view(torch.int32).item()) for o in self._offsets]
