"""Python binding of libdfs: the C-ABI entry points under the same names, on torch tensors.

Argument marshalling only (pointers, strides, dtypes, the current CUDA stream).  Every step of
the solve runs in libdfs's CUDA kernels; PyTorch provides device memory and streams.

Layouts (see include/dfs.h): S is (n, m) row-major, V and X are (k, m) with one right-hand
side per row, W/L are (n, n) lower-triangular, n-space vectors are (n, k).
"""

from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import (DFS_BF16, DFS_F32, DFS_F64, PRECISIONS, DfsError, NotConvergedError, dfs_info, dfs_options,
                   dfs_problem)

_DT = {torch.float64: DFS_F64, torch.float32: DFS_F32, torch.bfloat16: DFS_BF16}


def _dtype_code(t: torch.Tensor) -> int:
    try:
        return _DT[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported dtype {t.dtype} (float64, float32 or bfloat16)") from None


def _rows(t: torch.Tensor, name: str) -> int:
    """Leading dimension (row stride in elements) of a row-major 2-D tensor."""
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if t.stride(1) != 1:
        raise ValueError(f"{name} must have unit stride along its last dimension")
    return t.stride(0) if t.shape[0] > 1 else max(t.stride(0), t.shape[1])


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _opts(precision, max_iter, tol, timing=False, fp64_panel=False, center=False,
          two_kernel_gram=False, rhs_group=0) -> dfs_options:
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    flags = (_lib.DFS_FLAG_STEP_TIMING if timing else 0) | (_lib.DFS_FLAG_FP64_PANEL if fp64_panel else 0)
    flags |= _lib.DFS_FLAG_CENTER if center else 0
    flags |= _lib.DFS_FLAG_TWO_KERNEL_GRAM if two_kernel_gram else 0
    if rhs_group not in (0, 1, 2, 4, 8):
        raise ValueError("rhs_group must be 0 (auto), 1, 2, 4 or 8")
    flags |= (int(rhs_group) & 15) << 8
    return dfs_options(p, int(max_iter), float(tol), flags)


def _settle(lib, h, st: int, allow_not_converged: bool, **result):
    """Raise on a failed solve.  NOT_CONVERGED raises NotConvergedError (carrying the returned
    iterate and info) unless the caller allows it."""
    if st == _lib.DFS_OK:
        return
    if st == _lib.DFS_ERR_NOT_CONVERGED:
        if allow_not_converged:
            return
        msg = lib.dfs_last_error(h).decode() if h else ""
        e = NotConvergedError(st, f"{lib.dfs_status_string(st).decode()}: {msg}")
        for key, val in result.items():
            setattr(e, key, val)
        raise e
    _check(lib, h, st)


def _check(lib, h, status: int):
    if status != _lib.DFS_OK:
        msg = lib.dfs_last_error(h).decode() if h else ""
        raise DfsError(status, f"{lib.dfs_status_string(status).decode()}: {msg}")


def _info_dict(info: dfs_info) -> dict:
    return dict(status=info.status, precision=_lib.PRECISION_NAMES.get(info.precision_used, "?"),
                iters=info.iters, passes=info.passes, failed_pivot=info.failed_pivot,
                rel_correction=info.rel_correction,
                rel_residual_n=info.rel_residual_n, ms=[float(x) for x in info.ms])


class Handle:
    """Owns a dfs_handle (device workspace); one per device and host thread."""

    def __init__(self, device: int | None = None):
        self.lib = _lib.load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        st = self.lib.dfs_create(C.byref(h), self.device)
        if st != _lib.DFS_OK:
            raise DfsError(st, f"dfs_create failed: {self.lib.dfs_status_string(st).decode()}")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.dfs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default: dict[int, Handle] = {}


def default_handle(device: int | None = None) -> Handle:
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _default:
        _default[d] = Handle(d)
    return _default[d]


def dfs_kernel_launches() -> int:
    """Kernels libdfs has launched in this process."""
    return int(_lib.load().dfs_kernel_launches())


def dfs_reserve(n_max: int, m_max: int, k_max: int, precision="auto", handle: Handle | None = None):
    h = handle or default_handle()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(h.lib, h.h, h.lib.dfs_reserve(h.h, n_max, m_max, k_max, p))


def dfs_solve(S: torch.Tensor, V: torch.Tensor, lam: float, X: torch.Tensor | None = None, precision="auto",
              max_iter: int = -1, tol: float = 0.0, handle: Handle | None = None, stream=None,
              sync: bool = True, timing: bool = False, fp64_panel: bool = False, center: bool = False,
              two_kernel_gram: bool = False, allow_not_converged: bool = False, rhs_group: int = 0):
    """Solve (S^T S + lam I) X^T = V^T for the k rows of V (Eq. 1, Algorithm 1).

    center=True: S holds O and the system is Eq. 1 with Section 4's SR scores (O - O_bar)/sqrt(n).
    two_kernel_gram=True: the first pass over S and the BF16 Gram as two kernels instead of the
    fused one (for comparison).  rhs_group: right-hand sides per group of passes (0 = the
    library's choice).

    Returns (X, info) when sync is True (info = dict of dfs_info), else (X, None) with the work
    queued on the stream (read the status later with dfs_sync_info).  A solve whose refinement
    stops above tolerance raises NotConvergedError (with .X and .info) unless
    allow_not_converged is set.
    """
    h = handle or default_handle(S.device.index)
    n, m = S.shape
    k = V.shape[0]
    if V.shape[1] != m:
        raise ValueError("V must be (k, m)")
    vdt = torch.float64 if S.dtype == torch.float64 else torch.float32
    if V.dtype != vdt:
        raise TypeError(f"V must be {vdt} for S of dtype {S.dtype}")
    if X is None:
        X = torch.empty((k, m), device=S.device, dtype=vdt)
    opt = _opts(precision, max_iter, tol, timing, fp64_panel, center, two_kernel_gram, rhs_group)
    info = dfs_info()
    st = h.lib.dfs_solve(h.h, S.data_ptr(), _dtype_code(S), n, m, _rows(S, "S"), V.data_ptr(), k, _rows(V, "V"),
                         float(lam), X.data_ptr(), _rows(X, "X"), C.byref(opt), _stream(stream),
                         C.byref(info) if sync else None)
    if sync:
        d = _info_dict(info)
        _settle(h.lib, h.h, st, allow_not_converged, X=X, info=d)
        return X, d
    _check(h.lib, h.h, st)
    return X, None


def dfs_sync_info(handle: Handle | None = None, stream=None, allow_not_converged: bool = False) -> dict:
    h = handle or default_handle()
    info = dfs_info()
    st = h.lib.dfs_sync_info(h.h, _stream(stream), C.byref(info))
    d = _info_dict(info)
    _settle(h.lib, h.h, st, allow_not_converged, info=d)
    return d


def dfs_step_times(handle: Handle | None = None) -> tuple[list[float], int]:
    """Mean step times (ms) over recent timed solves: [gram, finalize+cholesky, first solve, rest,
    total, S v pass kernel, first refinement/x pass kernel, Cholesky kernel]."""
    h = handle or default_handle()
    out = (C.c_float * _lib.DFS_STEP_TIMES)()
    cnt = C.c_int(0)
    _check(h.lib, h.h, h.lib.dfs_step_times(h.h, out, C.byref(cnt)))
    return [float(x) for x in out], int(cnt.value)


def dfs_solve_host(S: torch.Tensor, V: torch.Tensor, lam: float, X: torch.Tensor | None = None, precision="auto",
                   max_iter: int = -1, tol: float = 0.0, handle: Handle | None = None, stream=None,
                   center: bool = False, allow_not_converged: bool = False):
    """Same solve with S, V, X in host memory (pinned for full copy speed); copies inside the call."""
    h = handle or default_handle()
    n, m = S.shape
    k = V.shape[0]
    if X is None:
        X = torch.empty((k, m), dtype=V.dtype, pin_memory=S.is_pinned())
    opt = _opts(precision, max_iter, tol, center=center)
    info = dfs_info()
    st = h.lib.dfs_solve_host(h.h, S.data_ptr(), _dtype_code(S), n, m, _rows(S, "S"), V.data_ptr(), k,
                              _rows(V, "V"), float(lam), X.data_ptr(), _rows(X, "X"), C.byref(opt),
                              _stream(stream), C.byref(info))
    d = _info_dict(info)
    _settle(h.lib, h.h, st, allow_not_converged, X=X, info=d)
    return X, d


def dfs_solve_host_async(S: torch.Tensor, V: torch.Tensor, lam: float, X: torch.Tensor, precision="auto",
                         max_iter: int = -1, tol: float = 0.0, handle: Handle | None = None, stream=None,
                         center: bool = False) -> torch.Tensor:
    """dfs_solve_host queued without waiting (pinned S, V, X): consecutive calls overlap one call's
    upload with the previous call's solve.  Read X, and the status (dfs_sync_info), after the stream
    has finished."""
    h = handle or default_handle()
    n, m = S.shape
    k = V.shape[0]
    if not (S.is_pinned() and V.is_pinned() and X.is_pinned()):
        raise ValueError("dfs_solve_host_async needs pinned host tensors")
    opt = _opts(precision, max_iter, tol, center=center)
    st = h.lib.dfs_solve_host_async(h.h, S.data_ptr(), _dtype_code(S), n, m, _rows(S, "S"), V.data_ptr(), k,
                                    _rows(V, "V"), float(lam), X.data_ptr(), _rows(X, "X"), C.byref(opt),
                                    _stream(stream))
    _check(h.lib, h.h, st)
    return X


def dfs_solve_complex(S_re: torch.Tensor, S_im: torch.Tensor, V_re: torch.Tensor, V_im: torch.Tensor, lam: float,
                      precision="auto", max_iter: int = -1, tol: float = 0.0, handle: Handle | None = None,
                      stream=None, allow_not_converged: bool = False, two_kernel_gram: bool = False):
    """Complex SR (Section 4, F = S^dagger S): solve (S^dagger S + lam I) X^T = V^T for S = S_re + i S_im
    (n x m planes) and the k rows of V = V_re + i V_im; returns (X_re, X_im, info)."""
    h = handle or default_handle(S_re.device.index)
    n, m = S_re.shape
    k = V_re.shape[0]
    if S_im.shape != S_re.shape or S_im.stride() != S_re.stride() or S_im.dtype != S_re.dtype:
        raise ValueError("S_re and S_im must share shape, strides and dtype")
    if V_im.shape != V_re.shape or V_im.stride() != V_re.stride() or V_re.shape[1] != m:
        raise ValueError("V_re and V_im must both be (k, m) with the same strides")
    X_re, X_im = torch.empty_like(V_re), torch.empty_like(V_re)
    opt = _opts(precision, max_iter, tol, two_kernel_gram=two_kernel_gram)
    info = dfs_info()
    st = h.lib.dfs_solve_complex(h.h, S_re.data_ptr(), S_im.data_ptr(), _dtype_code(S_re), n, m, _rows(S_re, "S"),
                                 V_re.data_ptr(), V_im.data_ptr(), k, _rows(V_re, "V"), float(lam), X_re.data_ptr(),
                                 X_im.data_ptr(), _rows(X_re, "X"), C.byref(opt), _stream(stream), C.byref(info))
    d = _info_dict(info)
    _settle(h.lib, h.h, st, allow_not_converged, X=(X_re, X_im), info=d)
    return X_re, X_im, d


def _batch_array(problems, alloc_x: bool):
    """The C problem array for [(S, V, lam[, X]), ...]: (array, outputs, S dtype code).  Without
    alloc_x a missing X is stood in for by V (planning reads only sizes and alignment)."""
    arr = (dfs_problem * len(problems))()
    outs = []
    dt = None
    for i, pr in enumerate(problems):
        S, V, lam = pr[0], pr[1], pr[2]
        X = pr[3] if len(pr) > 3 else (torch.empty_like(V) if alloc_x else V)
        dt = _dtype_code(S) if dt is None else dt
        if _dtype_code(S) != dt:
            raise TypeError("all S of a batch must share one dtype")
        arr[i] = dfs_problem(S.data_ptr(), S.shape[0], S.shape[1], _rows(S, "S"), V.data_ptr(), V.shape[0],
                             _rows(V, "V"), float(lam), X.data_ptr(), _rows(X, "X"))
        outs.append(X)
    return arr, outs, dt


def dfs_solve_batched(problems, precision="auto", max_iter: int = -1, tol: float = 0.0,
                      handle: Handle | None = None, stream=None, sync: bool = True, center: bool = False,
                      allow_not_converged: bool = False):
    """problems: list of (S, V, lam[, X]); returns (list of X, list of per-problem status or None).

    sync=False: no synchronization (the statuses stay on the device for dfs_batched_status);
    after dfs_plan_batched for the same shapes the call allocates nothing and can be captured.
    When a problem fails, the DfsError raised carries .outs (every X) and .statuses (per problem)."""
    h = handle or default_handle()
    arr, outs, dt = _batch_array(problems, alloc_x=True)
    opt = _opts(precision, max_iter, tol, center=center)
    status = (C.c_int * len(problems))() if sync else None
    st = h.lib.dfs_solve_batched(h.h, arr, len(problems), dt, C.byref(opt), _stream(stream), status)
    try:
        _settle(h.lib, h.h, st, allow_not_converged)
    except DfsError as e:
        e.outs = outs
        e.statuses = list(status) if sync else None
        raise
    return outs, (list(status) if sync else None)


def dfs_plan_batched(problems, precision="auto", max_iter: int = -1, tol: float = 0.0,
                     handle: Handle | None = None, center: bool = False) -> int:
    """Create the lanes and size the workspaces dfs_solve_batched needs for these problems
    ([(S, V, lam[, X]), ...]; only sizes and alignment are read).  Returns the device bytes held."""
    h = handle or default_handle()
    arr, _, dt = _batch_array(problems, alloc_x=False)
    opt = _opts(precision, max_iter, tol, center=center)
    nbytes = C.c_size_t(0)
    st = h.lib.dfs_plan_batched(h.h, arr, len(problems), dt, C.byref(opt), C.byref(nbytes))
    _check(h.lib, h.h, st)
    return nbytes.value


def dfs_batched_status(count: int, handle: Handle | None = None, stream=None,
                       allow_not_converged: bool = False) -> list:
    """Synchronize and return the device statuses of the last dfs_solve_batched (first `count`).
    Raises DfsError (with .statuses) on a failed problem; NOT_CONVERGED only raises
    (NotConvergedError) unless allow_not_converged is set."""
    h = handle or default_handle()
    status = (C.c_int * max(count, 1))()
    st = h.lib.dfs_batched_status(h.h, status, count, _stream(stream))
    out = list(status)[:count]
    try:
        _settle(h.lib, h.h, st, allow_not_converged)
    except DfsError as e:
        e.statuses = out
        raise
    return out


def dfs_set_batch_lanes(lanes: int, share: int = 1, handle: Handle | None = None) -> None:
    """Run dfs_solve_batched on up to `lanes` concurrent lanes, each lane's kernels sized for
    1/share of the SMs."""
    h = handle or default_handle()
    _check(h.lib, h.h, h.lib.dfs_set_batch_lanes(h.h, int(lanes), int(share)))


def dfs_get_batch_lanes(handle: Handle | None = None) -> tuple:
    """(lanes, share) dfs_solve_batched uses on this handle."""
    h = handle or default_handle()
    lanes, share = C.c_int(0), C.c_int(0)
    _check(h.lib, h.h, h.lib.dfs_get_batch_lanes(h.h, C.byref(lanes), C.byref(share)))
    return lanes.value, share.value


def dfs_autotune_batched(problems, precision="auto", max_iter: int = -1, tol: float = 0.0,
                         handle: Handle | None = None, stream=None, center: bool = False,
                         cache_path: str | None = None) -> dict:
    """Time dfs_solve_batched on `problems` ([(S, V, lam, X), ...]; X is overwritten) under each
    candidate (lanes, share), set the fastest on the handle and return
    {"lanes", "share", "ms"} (ms 0.0 when cache_path held a choice for this GPU and batch)."""
    h = handle or default_handle()
    arr, _, dt = _batch_array(problems, alloc_x=True)
    opt = _opts(precision, max_iter, tol, center=center)
    lanes, share, ms = C.c_int(0), C.c_int(0), C.c_float(0.0)
    path = cache_path.encode() if cache_path else None
    st = h.lib.dfs_autotune_batched(h.h, arr, len(problems), dt, C.byref(opt), path, _stream(stream),
                                    C.byref(lanes), C.byref(share), C.byref(ms))
    _check(h.lib, h.h, st)
    return {"lanes": lanes.value, "share": share.value, "ms": ms.value}


def dfs_gram(S: torch.Tensor, lam: float, precision="auto", W: torch.Tensor | None = None,
             handle: Handle | None = None, stream=None) -> torch.Tensor:
    """Algorithm 1, Gram: lower triangle of W = S S^T + lam I (upper triangle untouched)."""
    h = handle or default_handle(S.device.index)
    n, m = S.shape
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    wdt = torch.float64 if (p == PRECISIONS["fp64"] or (p == 0 and S.dtype == torch.float64)) else torch.float32
    if W is None:
        W = torch.zeros((n, n), device=S.device, dtype=wdt)
    st = h.lib.dfs_gram(h.h, S.data_ptr(), _dtype_code(S), n, m, _rows(S, "S"), float(lam), p, W.data_ptr(),
                        _rows(W, "W"), _stream(stream))
    _check(h.lib, h.h, st)
    return W


def dfs_cholesky(W: torch.Tensor, handle: Handle | None = None, stream=None) -> tuple[torch.Tensor, int]:
    """Algorithm 1's Cholesky, in place on the lower triangle of W; returns (L, failed_pivot or -1)."""
    h = handle or default_handle(W.device.index)
    n = W.shape[0]
    piv = C.c_int64(-1)
    st = h.lib.dfs_cholesky(h.h, W.data_ptr(), _dtype_code(W), n, _rows(W, "W"), _stream(stream), C.byref(piv))
    if st != _lib.DFS_OK:
        msg = h.lib.dfs_last_error(h.h).decode()
        raise DfsError(st, f"{h.lib.dfs_status_string(st).decode()}: {msg} (pivot {piv.value})")
    return W, piv.value


def dfs_trsm(L: torch.Tensor, B: torch.Tensor, trans: bool = False, handle: Handle | None = None,
             stream=None) -> torch.Tensor:
    """In place on B (n, k): solves L A = B (trans False) or L^T Y = B (trans True)."""
    h = handle or default_handle(L.device.index)
    n = L.shape[0]
    k = B.shape[1]
    st = h.lib.dfs_trsm(h.h, L.data_ptr(), _dtype_code(L), n, _rows(L, "L"), B.data_ptr(), k, _rows(B, "B"),
                        1 if trans else 0, _stream(stream))
    _check(h.lib, h.h, st)
    return B


def dfs_fisher_pass(S: torch.Tensor, V: torch.Tensor, lam: float, Y: torch.Tensor | None = None,
                    want_x: bool = True, want_r: bool = True, handle: Handle | None = None, stream=None):
    """One read of S: X = (V - S^T Y)/lam and R = S (V - S^T Y) - lam Y (Y (n, k) FP64 or None = 0)."""
    h = handle or default_handle(S.device.index)
    n, m = S.shape
    k = V.shape[0]
    X = torch.empty_like(V) if want_x else None
    R = torch.empty((n, k), device=S.device, dtype=torch.float64) if want_r else None
    st = h.lib.dfs_fisher_pass(h.h, S.data_ptr(), _dtype_code(S), n, m, _rows(S, "S"), V.data_ptr(), k,
                               _rows(V, "V"), Y.data_ptr() if Y is not None else None,
                               _rows(Y, "Y") if Y is not None else k, float(lam),
                               X.data_ptr() if X is not None else None, _rows(X, "X") if X is not None else m,
                               R.data_ptr() if R is not None else None, k, _stream(stream))
    _check(h.lib, h.h, st)
    return X, R


def dfs_fisher_pass_noalloc(S: torch.Tensor, V: torch.Tensor, lam: float, Y: torch.Tensor | None = None,
                            X: torch.Tensor | None = None, R: torch.Tensor | None = None, stream=None):
    """dfs_fisher_pass without a handle or any device allocation inside the library call.

    Writes X = (V - S^T Y)/lam into X and R = S (V - S^T Y) - lam Y into R (n x k FP64) when
    they are given; the caller owns (and allocates) both.  Scratch is the library's fixed
    per-device array of DFS_NOALLOC_SCRATCH_BYTES, shared by all calls on the device: calls
    that overlap on the device race.  Runs on the current device.
    """
    lib = _lib.load()
    n, m = S.shape
    k = V.shape[0]
    need = C.c_int64(0)
    st = lib.dfs_fisher_pass_noalloc(S.data_ptr(), _dtype_code(S), n, m, _rows(S, "S"), V.data_ptr(), k,
                                     _rows(V, "V"), Y.data_ptr() if Y is not None else None,
                                     _rows(Y, "Y") if Y is not None else k, float(lam),
                                     X.data_ptr() if X is not None else None, _rows(X, "X") if X is not None else m,
                                     R.data_ptr() if R is not None else None, _rows(R, "R") if R is not None else k,
                                     _stream(stream), C.byref(need))
    if st != _lib.DFS_OK:
        detail = ""
        if st == _lib.DFS_ERR_NO_MEMORY:
            detail = (f": needs {need.value} bytes of scratch, the fixed array holds "
                      f"{_lib.DFS_NOALLOC_SCRATCH_BYTES}")
        raise DfsError(st, lib.dfs_status_string(st).decode() + detail)
    return X, R


def dfs_fisher_pass_noalloc_status(stream=None) -> int:
    """Wait for `stream` and return the device status of the last dfs_fisher_pass_noalloc on the
    current device (0 = DFS_OK, 5 = DFS_ERR_TIMEOUT, ...).  Allocates nothing."""
    lib = _lib.load()
    out = C.c_int(-1)
    st = lib.dfs_fisher_pass_noalloc_status(C.byref(out), _stream(stream))
    if st != _lib.DFS_OK:
        raise DfsError(st, lib.dfs_status_string(st).decode())
    return int(out.value)


def dfs_set_test_fault(fault: int, wait_limit_ns: int = 0, handle: Handle | None = None):
    """Test hook: following calls on the handle withhold the signal `fault` names
    (DFS_TEST_FAULT_*), so that the bounded device waits for it run out after wait_limit_ns
    (<= 0: the 2 s default).  DFS_TEST_FAULT_NONE switches it off."""
    h = handle or default_handle()
    _check(h.lib, h.h, h.lib.dfs_set_test_fault(h.h, int(fault), int(wait_limit_ns)))


def dfs_fisher_pass_noalloc_test_fault(fault: int, wait_limit_ns: int = 0):
    """The test hook of dfs_set_test_fault for the no-allocation calls on the current device."""
    lib = _lib.load()
    st = lib.dfs_fisher_pass_noalloc_test_fault(int(fault), int(wait_limit_ns))
    if st != _lib.DFS_OK:
        raise DfsError(st, lib.dfs_status_string(st).decode())


def dfs_measure_peak(kind: str) -> float:
    """Measured peak flop/s of the current device's SIMT fused multiply-add: kind "ffma32" or
    "dfma64" (the roofline denominators of the FP32-path Gram and of FP64 arithmetic)."""
    lib = _lib.load()
    code = {"ffma32": _lib.DFS_PEAK_FFMA32, "dfma64": _lib.DFS_PEAK_DFMA64}[kind]
    out = C.c_double(0.0)
    st = lib.dfs_measure_peak(code, C.byref(out))
    if st != _lib.DFS_OK:
        raise DfsError(st, lib.dfs_status_string(st).decode())
    return float(out.value)
