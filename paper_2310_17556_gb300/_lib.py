"""ctypes view of libdfs.so (the C ABI declared in include/dfs.h).

Loading fails loudly when the library has not been built: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdfs.so")
LIB_DEBUG_PATH = os.path.join(PKG, "libdfs_debug.so")  # device index checks (-DDFS_DEBUG_BOUNDS)

# enums of include/dfs.h
DFS_OK = 0
DFS_ERR_INVALID_ARG = 1
DFS_ERR_NOT_SPD = 2
DFS_ERR_NOT_CONVERGED = 3
DFS_ERR_NONFINITE = 4
DFS_ERR_TIMEOUT = 5
DFS_ERR_NO_MEMORY = 6
DFS_ERR_CUDA = 7
DFS_ERR_UNSUPPORTED = 8
DFS_ERR_BOUNDS = 9

DFS_F64, DFS_F32, DFS_BF16 = 0, 1, 2
PRECISIONS = {"auto": 0, "fp64": 1, "fp32": 2, "bf16": 3, "tf32": 4, "bf16x3": 5, "fp8": 6}
PRECISION_NAMES = {v: k for k, v in PRECISIONS.items()}

# every entry point include/dfs.h declares
EXPORTS = (
    "dfs_create", "dfs_destroy", "dfs_status_string", "dfs_last_error", "dfs_reserve", "dfs_kernel_launches",
    "dfs_solve", "dfs_solve_host", "dfs_solve_host_async", "dfs_solve_complex", "dfs_sync_info", "dfs_step_times", "dfs_solve_batched",
    "dfs_plan_batched", "dfs_batched_status", "dfs_set_batch_lanes", "dfs_get_batch_lanes", "dfs_autotune_batched",
    "dfs_gram", "dfs_cholesky", "dfs_trsm", "dfs_fisher_pass", "dfs_fisher_pass_noalloc",
    "dfs_fisher_pass_noalloc_status", "dfs_fisher_pass_noalloc_test_fault", "dfs_set_test_fault",
    "dfs_measure_peak",
)


class dfs_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_iter", C.c_int), ("tol", C.c_double), ("flags", C.c_int)]


class dfs_info(C.Structure):
    _fields_ = [("status", C.c_int), ("precision_used", C.c_int), ("iters", C.c_int),
                ("failed_pivot", C.c_int), ("passes", C.c_int), ("rel_correction", C.c_double),
                ("rel_residual_n", C.c_double), ("ms", C.c_float * 9)]


DFS_STEP_TIMES = 9
DFS_FLAG_STEP_TIMING = 1
DFS_FLAG_FP64_PANEL = 2
DFS_FLAG_CENTER = 4
DFS_FLAG_TWO_KERNEL_GRAM = 8
DFS_PEAK_FFMA32 = 1
DFS_PEAK_DFMA64 = 2
DFS_TEST_FAULT_NONE = 0
DFS_TEST_FAULT_CHOLESKY = 1
DFS_TEST_FAULT_CLUSTER_PASS = 2
DFS_TEST_FAULT_FUSED_GRAM = 3
DFS_NOALLOC_SCRATCH_BYTES = 8 << 20


class dfs_problem(C.Structure):
    _fields_ = [("S", C.c_void_p), ("n", C.c_int64), ("m", C.c_int64), ("lds", C.c_int64),
                ("V", C.c_void_p), ("k", C.c_int64), ("ldv", C.c_int64),
                ("lam", C.c_double), ("X", C.c_void_p), ("ldx", C.c_int64)]


_I64 = C.c_int64
_VP = C.c_void_p
_SIGS = {
    "dfs_create": (C.c_int, [C.POINTER(_VP), C.c_int]),
    "dfs_destroy": (C.c_int, [_VP]),
    "dfs_status_string": (C.c_char_p, [C.c_int]),
    "dfs_kernel_launches": (C.c_int64, []),
    "dfs_last_error": (C.c_char_p, [_VP]),
    "dfs_reserve": (C.c_int, [_VP, _I64, _I64, _I64, C.c_int]),
    "dfs_solve": (C.c_int, [_VP, _VP, C.c_int, _I64, _I64, _I64, _VP, _I64, _I64, C.c_double, _VP, _I64,
                            C.POINTER(dfs_options), _VP, C.POINTER(dfs_info)]),
    "dfs_solve_host": (C.c_int, [_VP, _VP, C.c_int, _I64, _I64, _I64, _VP, _I64, _I64, C.c_double, _VP, _I64,
                                 C.POINTER(dfs_options), _VP, C.POINTER(dfs_info)]),
    "dfs_solve_host_async": (C.c_int, [_VP, _VP, C.c_int, _I64, _I64, _I64, _VP, _I64, _I64, C.c_double, _VP,
                                       _I64, C.POINTER(dfs_options), _VP]),
    "dfs_solve_complex": (C.c_int, [_VP, _VP, _VP, C.c_int, _I64, _I64, _I64, _VP, _VP, _I64, _I64, C.c_double,
                                    _VP, _VP, _I64, C.POINTER(dfs_options), _VP, C.POINTER(dfs_info)]),
    "dfs_sync_info": (C.c_int, [_VP, _VP, C.POINTER(dfs_info)]),
    "dfs_step_times": (C.c_int, [_VP, C.POINTER(C.c_float), C.POINTER(C.c_int)]),
    "dfs_solve_batched": (C.c_int, [_VP, C.POINTER(dfs_problem), C.c_int, C.c_int, C.POINTER(dfs_options), _VP,
                                    C.POINTER(C.c_int)]),
    "dfs_plan_batched": (C.c_int, [_VP, C.POINTER(dfs_problem), C.c_int, C.c_int, C.POINTER(dfs_options),
                                   C.POINTER(C.c_size_t)]),
    "dfs_batched_status": (C.c_int, [_VP, C.POINTER(C.c_int), C.c_int, _VP]),
    "dfs_set_batch_lanes": (C.c_int, [_VP, C.c_int, C.c_int]),
    "dfs_get_batch_lanes": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "dfs_autotune_batched": (C.c_int, [_VP, C.POINTER(dfs_problem), C.c_int, C.c_int, C.POINTER(dfs_options), C.c_char_p,
                                       _VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "dfs_gram": (C.c_int, [_VP, _VP, C.c_int, _I64, _I64, _I64, C.c_double, C.c_int, _VP, _I64, _VP]),
    "dfs_cholesky": (C.c_int, [_VP, _VP, C.c_int, _I64, _I64, _VP, C.POINTER(_I64)]),
    "dfs_trsm": (C.c_int, [_VP, _VP, C.c_int, _I64, _I64, _VP, _I64, _I64, C.c_int, _VP]),
    "dfs_fisher_pass": (C.c_int, [_VP, _VP, C.c_int, _I64, _I64, _I64, _VP, _I64, _I64, _VP, _I64, C.c_double,
                                  _VP, _I64, _VP, _I64, _VP]),
    "dfs_fisher_pass_noalloc": (C.c_int, [_VP, C.c_int, _I64, _I64, _I64, _VP, _I64, _I64, _VP, _I64, C.c_double,
                                          _VP, _I64, _VP, _I64, _VP, C.POINTER(_I64)]),
    "dfs_fisher_pass_noalloc_status": (C.c_int, [C.POINTER(C.c_int), _VP]),
    "dfs_fisher_pass_noalloc_test_fault": (C.c_int, [C.c_int, _I64]),
    "dfs_set_test_fault": (C.c_int, [_VP, C.c_int, _I64]),
    "dfs_measure_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
}

_lib = None


def lib_path() -> str:
    """The library this process uses: libdfs_debug.so when DFS_DEBUG_BOUNDS=1, else libdfs.so."""
    return LIB_DEBUG_PATH if os.environ.get("DFS_DEBUG_BOUNDS", "0") == "1" else LIB_PATH


def load() -> C.CDLL:
    """Load the library from the package folder (RuntimeError if it was never built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        flag = " --debug-bounds" if path == LIB_DEBUG_PATH else ""
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2310_17556_gb300.build{flag}` "
                           "(the CUDA path has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DfsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class NotConvergedError(DfsError):
    """Refinement stopped above its tolerance (DFS_ERR_NOT_CONVERGED).  .X (or .outs) holds the
    best iterate the solve returned and .info its dfs_info fields."""
