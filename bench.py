#!/usr/bin/env python3
"""Throughput of the damped-Fisher Cholesky solve (arXiv 2310.17556, Algorithm 1) on GB300.

Workload: one solve of (S^T S + lambda I) x = v at n = 1024 samples, m = 2^20 parameters, k = 1,
S stored in FP32 and SVD-structured (S = U diag(sigma) V^T / sqrt(n), U Haar, V orthonormal from
the QR of a Gaussian, sigma log-spaced 1 .. 1e-3), v ~ N(0, 1), lambda = 1e-4 (and 1e-2 reported
beside it).  Synthetic data: the paper measures on no public dataset.

A "step" is one complete dfs_solve: tensor-core Gram, Cholesky, the S v pass, the triangular
solves and the refinement passes that write x (all of Algorithm 1), with S resident in HBM
(4.3 GB, larger than L2, so no L2 flush is needed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun; every rank solves its own independent problem (weak scaling,
no collective on the data path).  Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SAMPLES = 1024
M_PARAMS = 1 << 20
LAMBDA = 1e-4
LAMBDA_ALT = 1e-2
SIGMA_MIN = 1e-3
METRIC = "damped-Fisher solves/s at n=1024,m=2^20 (mixed vs FP32 path, rel err≤1e-6)"
UNIT = "solves/s"
# TF32 dense tensor rate relative to BF16 (nominal 1.1 vs 2.25 PFLOP/s per GPU)
TF32_OVER_BF16 = 1.1 / 2.25


def workload_config(lam=LAMBDA):
    return {
        "workload": f"SVD-structured FP32 score matrix n={N_SAMPLES} m={M_PARAMS} k=1 lambda={lam:g} "
                    f"(sigma log-spaced 1..{SIGMA_MIN:g})",
        "n": N_SAMPLES, "m": M_PARAMS, "k": 1, "lambda": lam,
        "mixed_path": "TF32 tcgen05 Gram + n-space refinement to est. err <= 1e-7",
        "cache": "inputs larger than L2 (S is 4.3 GB; L2 is 129 MB), no flush between steps",
        "parallelism": "replicas (one independent solve per GPU)",
    }


# ----------------------------------------------------------------------------- helpers


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _clock_sampler(gpu_index: int):
    fields = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={fields}",
                                 "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=10)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 7:
            continue
        try:
            sm.append(float(parts[0]))
            mx.append(float(parts[1]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[3:7]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "samples": len(sm), "reasons": sorted(reasons)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _kernel_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, or None if the kernel changed since."""
    p = os.path.join(ROOT, "profiles", "roofline_counters.json")
    try:
        with open(p) as f:
            doc = json.load(f)
    except (OSError, ValueError):
        return None
    ent = doc.get(kernel)
    if not ent:
        return None
    h = hashlib.sha256()
    for rel in ent.get("sources", []):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != ent.get("sha256"):
        return None
    return ent.get("dram_bytes_per_launch")


def _make_inputs(torch, wl, dev, seed):
    S, U, s, V = wl.svd_structured(N_SAMPLES, M_PARAMS, seed=seed, sigma_min=SIGMA_MIN, device=dev,
                                   dtype=torch.float32, factor_dtype=torch.float64)
    del U, V
    v = wl.rhs(M_PARAMS, 1, seed=seed + 7, device=dev)
    torch.cuda.synchronize()
    return S, v, float(s[0])


def _residual_bound(torch, S, v, x, lam, smax):
    """FP64 residual of Eq. 1 and the error bound it gives: e_rel <= cond(A) * res with
    cond(A) = (sigma_max^2 + lambda) / lambda (A = S^T S + lambda I)."""
    Sd = S.double()
    xd = x.double().reshape(-1)
    r = Sd.T @ (Sd @ xd) + lam * xd - v.double().reshape(-1)
    res = float(torch.linalg.norm(r) / torch.linalg.norm(v.double()))
    del Sd
    cond = (smax * smax + lam) / lam
    return res, cond * res


# ----------------------------------------------------------------------------- CPU (oracle) arm


def _oracle_sample_solves_per_s(S_np, v_np, lam, m_sample):
    """Time the FP64 oracle on the first m_sample columns; scale to the full m (cost ~ n^2 m)."""
    import oracle

    Ss = S_np[:, :m_sample]
    vs = v_np[:m_sample]
    t0 = time.perf_counter()
    oracle.solve(Ss, vs, lam)
    dt = time.perf_counter() - t0
    return (1.0 / dt) * (m_sample / M_PARAMS), dt


def _host_inputs(seed):
    import torch

    from paper_2310_17556_gb300 import workloads as wl

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    m_gen = M_PARAMS
    S, v, smax = _make_inputs(torch, wl, dev, seed) if dev == "cuda" else (None, None, None)
    if S is None:  # no GPU: generate a reduced sample directly on the host
        m_gen = 1 << 17
        S, _, s, _ = wl.svd_structured(N_SAMPLES, m_gen, seed=seed, sigma_min=SIGMA_MIN)
        v = wl.rhs(m_gen, 1, seed=seed + 7)
    return S.cpu().double().numpy(), v.cpu().double().numpy()[0], m_gen


def cpu_baseline(S_np, v_np, target_s=12.0):
    """The oracle (FP64 numpy, all host cores) on a bounded column sample of the workload."""
    m_avail = S_np.shape[1]
    m_s = min(1 << 14, m_avail)
    rate, dt = _oracle_sample_solves_per_s(S_np, v_np, LAMBDA, m_s)
    while dt * 2 < target_s and m_s * 2 <= m_avail and m_s < (1 << 18):
        m_s *= 2
        rate, dt = _oracle_sample_solves_per_s(S_np, v_np, LAMBDA, m_s)
    return {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 oracle (numpy, {os.cpu_count()} threads) on the first {m_s} of {M_PARAMS} columns "
                      f"(n={N_SAMPLES}, k=1) in {dt:.2f} s, scaled by {m_s}/{M_PARAMS} (cost linear in m)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    S_np, v_np, m_avail = _host_inputs(231017556 + 1)
    # size the per-step sample so that warmup + steps take a few minutes at most
    m_s = min(1 << 14, m_avail)
    _, dt = _oracle_sample_solves_per_s(S_np, v_np, LAMBDA, m_s)
    budget = 150.0 / max(1, args.steps + args.warmup)
    while dt * 2 < budget and m_s * 2 <= m_avail and m_s < (1 << 18):
        m_s *= 2
        _, dt = _oracle_sample_solves_per_s(S_np, v_np, LAMBDA, m_s)
    for _ in range(args.warmup):
        _oracle_sample_solves_per_s(S_np, v_np, LAMBDA, m_s)
    times = []
    for _ in range(args.steps):
        _, dt = _oracle_sample_solves_per_s(S_np, v_np, LAMBDA, m_s)
        times.append(dt)
    per_full = statistics.mean(times) * (M_PARAMS / m_s)
    value = 1.0 / per_full
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_full * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"each step: FP64 oracle on the first {m_s} of {M_PARAMS} columns, "
                                   f"scaled by {m_s}/{M_PARAMS}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    barrier()
    import paper_2310_17556_gb300 as dfs
    from paper_2310_17556_gb300 import workloads as wl

    S, v, smax = _make_inputs(torch, wl, dev, 231017556 + 1 + rank)
    X = torch.empty_like(v)
    stream = torch.cuda.current_stream()
    h = dfs.default_handle()

    # ---------------- mixed path (headline) ----------------
    for _ in range(args.warmup):
        dfs.dfs_solve(S, v, LAMBDA, X=X, precision="tf32", sync=False)
    info = dfs.dfs_sync_info()
    if info["status"] != 0:
        raise RuntimeError(f"mixed solve failed: {info}")
    dfs.dfs_step_times()  # reset the timing ring
    clocks_proc = _clock_sampler(local)
    time.sleep(0.3)
    barrier()
    launches0 = dfs.dfs_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        dfs.dfs_solve(S, v, LAMBDA, X=X, precision="tf32", sync=False, timing=True)
    e1.record(stream)
    barrier()
    launches = dfs.dfs_kernel_launches() - launches0
    clocks = _clock_summary(clocks_proc)
    elapsed_ms = e0.elapsed_time(e1)
    info = dfs.dfs_sync_info()
    step_ms, nsteps_timed = dfs.dfs_step_times()
    if dist is not None:
        t = torch.tensor([elapsed_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    value = ws * args.steps / (elapsed_ms / 1e3)
    res, err_bound = _residual_bound(torch, S, v, X, LAMBDA, smax)

    # same solve at lambda = 1e-2 (fewer passes are needed there), a few steps
    X2 = torch.empty_like(v)
    dfs.dfs_solve(S, v, LAMBDA_ALT, X=X2, precision="tf32", sync=False)
    torch.cuda.synchronize()
    k2 = max(3, args.steps // 4)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(k2):
        dfs.dfs_solve(S, v, LAMBDA_ALT, X=X2, precision="tf32", sync=False)
    a1.record(stream)
    torch.cuda.synchronize()
    info_alt = dfs.dfs_sync_info()
    alt_value = k2 / (a0.elapsed_time(a1) / 1e3)
    res_alt, bound_alt = _residual_bound(torch, S, v, X2, LAMBDA_ALT, smax)

    # ---------------- plain FP32 path (comparison) ----------------
    Xf = torch.empty_like(v)
    dfs.dfs_solve(S, v, LAMBDA, X=Xf, precision="fp32", sync=False)
    torch.cuda.synchronize()
    kf = max(3, args.steps // 10)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(kf):
        dfs.dfs_solve(S, v, LAMBDA, X=Xf, precision="fp32", sync=False)
    f1.record(stream)
    torch.cuda.synchronize()
    fp32_value = kf / (f0.elapsed_time(f1) / 1e3)
    res_f, bound_f = _residual_bound(torch, S, v, Xf, LAMBDA, smax)

    # ---------------- end to end through the host-memory entry point ----------------
    S_h = torch.empty(S.shape, dtype=S.dtype, pin_memory=True)
    S_h.copy_(S)
    v_h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
    v_h.copy_(v)
    X_h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
    del S
    torch.cuda.empty_cache()
    dfs.dfs_solve_host(S_h, v_h, LAMBDA, X=X_h, precision="tf32")
    ke = max(3, args.steps // 10)
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        dfs.dfs_solve_host(S_h, v_h, LAMBDA, X=X_h, precision="tf32")
    barrier()
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = ws * ke / e2e_s

    # ---------------- roofline of the dominant kernel (tensor-core Gram) ----------------
    peaks, peak_kind = _peaks()
    gram_ms = step_ms[0]
    flops = float(N_SAMPLES) * (N_SAMPLES + 1) * M_PARAMS  # lower triangle incl. diagonal, 2 flop/MAC
    peak_tf = peaks["bf16_tflops_sustained"] * TF32_OVER_BF16
    achieved_tf = flops / (gram_ms / 1e3) / 1e12 if gram_ms > 0 else None
    roofline = {
        "kernel": "gram_tc_kernel<TF32>", "bound": "tensor", "achieved": achieved_tf, "peak": peak_tf,
        "unit": "TFLOP/s", "frac": (achieved_tf / peak_tf) if achieved_tf else None,
        "traffic": _kernel_traffic("gram_tc_kernel<TF32>"),
        "peak_source": f"{peak_kind} bf16_tflops_sustained x {TF32_OVER_BF16:.3f} (TF32/BF16 nominal)",
        "algorithmic_flop_per_launch": flops, "avg_launch_ms": gram_ms, "launches_averaged": nsteps_timed,
        "hbm_alt": {"bytes_per_launch": 4.0 * N_SAMPLES * M_PARAMS,
                    "achieved_gbs": 4.0 * N_SAMPLES * M_PARAMS / (gram_ms / 1e3) / 1e9 if gram_ms > 0 else None,
                    "peak_gbs": peaks["hbm_gbs"]},
    }

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32", "data": "synthetic", "config": workload_config(),
        "accuracy": {"res_fp64": res, "e_rel_bound": err_bound, "iters": info["iters"],
                     "est_err": info["rel_correction"], "status": info["status"]},
        "step_ms": {"gram": step_ms[0], "finalize_cholesky": step_ms[1], "first_solve": step_ms[2],
                    "refinement": step_ms[3], "total": step_ms[4]},
        "fp32_path": {"value": fp32_value, "unit": UNIT, "res_fp64": res_f, "e_rel_bound": bound_f,
                      "steps": kf},
        "lambda_1e-2": {"value": alt_value, "unit": UNIT, "res_fp64": res_alt, "e_rel_bound": bound_alt,
                        "iters": info_alt["iters"], "steps": k2},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N_SAMPLES * M_PARAMS + 4 * M_PARAMS,
                "d2h_bytes_per_step": 4 * M_PARAMS, "steps": ke, "api": "dfs_solve_host (pinned host S, v, x)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline,
    }
    if rank == 0 and not args.no_cpu_baseline:
        S_np = S_h[:, : 1 << 18].double().numpy()
        v_np = v_h[0, : 1 << 18].double().numpy()
        line["cpu_baseline"] = cpu_baseline(S_np, v_np)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
