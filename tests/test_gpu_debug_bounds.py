"""The debug build's device index checks (libdfs_debug.so, -DDFS_DEBUG_BOUNDS), the stand-in for a
memory checker: small cases through every instrumented kernel (the fused first pass, the tensor
and SIMT Grams, the Cholesky, the n-space solve, the cluster and tile-correction passes, the tile
packing) run in a child process on the debug library.  No check may fire (no DFS_ERR_BOUNDS, every
status 0), and each result must equal the release library's up to summation order.

The checks turn a bad index into a recorded status and a skipped access; this test runs valid
inputs only (nothing here is meant to go out of bounds)."""

import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2310_17556_gb300 import workloads as wl

from test_gpu_parity import aligned, dev, np64

pytestmark = pytest.mark.gpu

dfs = pytest.importorskip("paper_2310_17556_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (kind, n, m, k, precision, lambda): the cases both libraries run
CASES = [
    ("real", 257, 33336, 1, "bf16", 1e-3),   # fused first pass, cluster pass, tile correction, n-space
    ("real", 300, 20000, 8, "bf16", 1e-2),   # S v pass with tiles, tensor Gram, eight right-hand sides
    ("real", 200, 9000, 2, "fp32", 1e-2),    # SIMT Gram, plain x pass
    ("real", 2100, 12000, 1, "bf16", 1e-2),  # n above 2048: non-cluster n-space sizes, wider Cholesky
    ("complex", 300, 20004, 3, "bf16", 1e-2),
    ("batch", 0, 0, 2, "bf16", 0.0),
]


def run_cases():
    """Every case's outputs, in CASES order (device tensors moved to the host)."""
    out = []
    for j, (kind, n, m, k, prec, lam) in enumerate(CASES):
        if kind == "real":
            S = aligned(wl.gaussian(n, m, seed=2100 + j, device=dev()))
            V = wl.rhs(m, k, seed=2200 + j, device=dev())
            X, info = dfs.dfs_solve(S, V, lam, precision=prec)
            out.append(([X.cpu()], info["status"]))
        elif kind == "complex":
            Z = wl.gaussian(2 * n, m, seed=2100 + j, device=dev())
            Vr, Vi = wl.rhs(m, k, seed=2200 + j, device=dev()), wl.rhs(m, k, seed=2300 + j, device=dev())
            Xr, Xi, info = dfs.dfs_solve_complex(Z[:n], Z[n:], Vr, Vi, lam, precision=prec)
            out.append(([Xr.cpu(), Xi.cpu()], info["status"]))
        else:
            probs = [(wl.gaussian(nn, mm, seed=2400 + q, device=dev()), wl.rhs(mm, k, seed=2500 + q, device=dev()), ll)
                     for q, (nn, mm, ll) in enumerate([(130, 8000, 1e-2), (64, 20000, 1e-3), (400, 5000, 1e-1)])]
            outs, statuses = dfs.dfs_solve_batched(probs, precision=prec)
            out.append(([x.cpu() for x in outs], max(statuses)))
    torch.cuda.synchronize()
    return out


CHILD = (
    "import sys, torch\n"
    "sys.path.insert(0, {tests!r})\n"
    "import test_gpu_debug_bounds as t\n"
    "from paper_2310_17556_gb300 import _lib\n"
    "assert _lib.lib_path() == _lib.LIB_DEBUG_PATH\n"
    "torch.save(t.run_cases(), {out!r})\n"
)


@pytest.fixture(scope="module")
def debug_lib():
    from paper_2310_17556_gb300 import build

    return build.build(debug_bounds=True)


def test_debug_library_runs_every_instrumented_kernel_without_a_bounds_fault(debug_lib, tmp_path):
    out = tmp_path / "debug.pt"
    env = dict(os.environ, DFS_DEBUG_BOUNDS="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD.format(tests=os.path.join(ROOT, "tests"), out=str(out))],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    dbg = torch.load(out)
    rel = run_cases()
    assert len(dbg) == len(rel) == len(CASES)
    for case, (xd, sd), (xr, sr) in zip(CASES, dbg, rel):
        assert sd == 0 and sr == 0, (case, sd, sr)
        for a, b in zip(xd, xr):
            a64, b64 = np64(a), np64(b)
            err = np.linalg.norm(a64 - b64) / np.linalg.norm(b64)
            assert err <= 1e-6, (case, err)
