#!/usr/bin/env python3
"""Throughput of the damped-Fisher Cholesky solve (arXiv 2310.17556, Algorithm 1) on GB300.

Workload: solves of (S^T S + lambda I) x = v at n = 1024 samples, m = 2^20 parameters, k = 1,
S stored in FP32 and SVD-structured (S = U diag(sigma) V^T / sqrt(n), U Haar, V orthonormal from
the QR of a Gaussian, sigma log-spaced 1 .. 1e-3), v ~ N(0, 1), lambda = 1e-4 (1e-2 reported
beside it).  Synthetic data: the paper measures on no public dataset.

A "step" is one complete dfs_solve on the mixed path: the S v pass that also packs S into BF16
tensor-core tiles, the tcgen05 Gram, the Cholesky, the triangular solves and the n-space
refinement passes that write x (all of Algorithm 1), with S resident in HBM (4.3 GB, larger
than L2, so no L2 flush is needed between steps).  The plain FP32 path is timed beside it, and
every reported solution is compared with the FP64 oracle's on the full problem.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload precision|batch|stress|complex     (the other configurations, one GPU)

N > 1 runs under torchrun; every rank solves its own independent problem (weak scaling, no
collective on the data path).  Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import hashlib
import json
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
SEED = 231017556 + 1
METRIC = "damped-Fisher solves/s at n=1024,m=2^20 (mixed vs FP32 path, rel err≤1e-6)"
UNIT = "solves/s"
PRECISION = "bf16"


def workload_config(lam=LAMBDA):
    return {
        "workload": f"SVD-structured FP32 score matrix n={N_SAMPLES} m={M_PARAMS} k=1 lambda={lam:g} "
                    f"(sigma log-spaced 1..{SIGMA_MIN:g})",
        "n": N_SAMPLES, "m": M_PARAMS, "k": 1, "lambda": lam,
        "mixed_path": "fused first pass (b = S v, BF16 tiles and the tcgen05 Gram in one kernel), "
                      "Cholesky, n-space refinement (FP32 passes over S with FP64 accumulation) to "
                      "est. rel. error <= 1e-7",
        "cache": "inputs larger than L2 (S is 4.3 GB; L2 is 129 MB), no flush between steps",
        "launch": "one dfs_solve captured into a CUDA graph, replayed once per step",
        "parallelism": "replicas (one independent solve per GPU)",
    }


# ----------------------------------------------------------------------------- helpers


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(value: float, dist, device) -> float:
    """The largest value over the ranks (a job's time is its slowest rank's); the value itself
    when there is no process group."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(world_size: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank solves `steps` problems of its own (weak scaling)."""
    return world_size * steps / seconds


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
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _live_peaks(torch, dfs):
    """Peaks MEASURED_PEAKS.json does not carry, measured here: the SIMT fused multiply-add rates
    (this library's own probe kernels) and cuBLAS TF32 and FP8 GEMM rates (8192^3, best of 3),
    in TFLOP/s.  None where a probe is not available."""
    out = {}
    for kind in ("ffma32", "dfma64"):
        try:
            out[kind + "_tflops"] = dfs.dfs_measure_peak(kind) / 1e12
        except Exception:  # noqa: BLE001 - a probe that cannot run reports nothing
            out[kind + "_tflops"] = None
    N = 8192

    def best(fn, flop):
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        return flop / (min(t) / 1e3) / 1e12

    try:
        a = torch.randn((N, N), device="cuda", dtype=torch.float32)
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        out["tf32_tflops_cublas"] = best(lambda: a @ a, 2.0 * N ** 3)
        torch.backends.cuda.matmul.allow_tf32 = prev
        a8 = a.to(torch.float8_e4m3fn)
        one = torch.ones((), device="cuda", dtype=torch.float32)
        out["fp8_tflops_cublas"] = best(lambda: torch._scaled_mm(a8, a8.t(), scale_a=one, scale_b=one,
                                                                  out_dtype=torch.bfloat16), 2.0 * N ** 3)
        del a, a8
        torch.cuda.empty_cache()
    except Exception:  # noqa: BLE001
        out.setdefault("tf32_tflops_cublas", None)
        out.setdefault("fp8_tflops_cublas", None)
    return out


def _kernel_traffic(kernel: str):
    """DRAM bytes per full-size launch from the committed ncu summary, or None when the kernel's
    sources changed since the counters were taken."""
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
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        except OSError:
            return None
    if h.hexdigest() != ent.get("sha256"):
        return None
    return ent.get("dram_bytes_per_launch")


def _make_inputs(torch, wl, dev, seed):
    S, U, s, V = wl.svd_structured(N_SAMPLES, M_PARAMS, seed=seed, sigma_min=SIGMA_MIN, device=dev,
                                   dtype=torch.float32, factor_dtype=torch.float64)
    del U, V
    v = wl.rhs(M_PARAMS, 1, seed=seed + 7, device=dev)
    torch.cuda.synchronize()
    return S, v


def _timed(torch, stream, fn, steps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


# ----------------------------------------------------------------------------- oracle (CPU) side


def _oracle_solve(S64, v64, lam):
    import oracle

    t0 = time.perf_counter()
    x = oracle.solve(S64, v64, lam)
    return x, time.perf_counter() - t0


def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


_CONFIG1_PROBE = (
    "import sys, time; sys.path.insert(0, %r); import numpy as np; import oracle\n"
    "from paper_2310_17556_gb300 import workloads as wl\n"
    "S = wl.gaussian(256, 16384, seed=231017556, dtype=__import__('torch').float64).numpy()\n"
    "v = wl.rhs(16384, 1, seed=231017557, dtype=__import__('torch').float64).numpy()[0]\n"
    "oracle.solve(S, v, 1e-3); t0 = time.perf_counter(); [oracle.solve(S, v, 1e-3) for _ in range(5)]\n"
    "print((time.perf_counter() - t0) / 5)\n")


def _oracle_config1_times():
    """The oracle's time for the small FP64 configuration (n=256, m=16384, k=1, lambda=1e-3) on all
    host cores and on one core (BLAS threads pinned to 1), each in a fresh interpreter."""
    out = {}
    for label, threads in (("all_cores", None), ("one_core", "1")):
        env = dict(os.environ)
        if threads:
            for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
                env[k] = threads
        try:
            r = subprocess.run([sys.executable, "-c", _CONFIG1_PROBE % ROOT], capture_output=True, text=True,
                               timeout=300, env=env)
            out[label + "_s"] = float(r.stdout.strip().splitlines()[-1])
        except (OSError, subprocess.SubprocessError, ValueError, IndexError):
            out[label + "_s"] = None
    return out


def _errors(S64, v64, lam, x, x_ref):
    import oracle

    e = oracle.errors(S64, v64, lam, x, x_ref)
    return {k: float(v) for k, v in e.items()}


def _host_inputs(seed):
    import torch

    from paper_2310_17556_gb300 import workloads as wl

    if torch.cuda.is_available():
        S, v = _make_inputs(torch, wl, "cuda", seed)
        m_avail = M_PARAMS
    else:  # no GPU: a reduced problem generated on the host
        m_avail = 1 << 17
        S, _, _, _ = wl.svd_structured(N_SAMPLES, m_avail, seed=seed, sigma_min=SIGMA_MIN)
        v = wl.rhs(m_avail, 1, seed=seed + 7)
    return S.cpu().double().numpy(), v.cpu().double().numpy()[0], m_avail


def run_reference(args):
    """The FP64 oracle (numpy, host cores) as the reference arm, on a bounded column sample of the
    workload per step (cost is linear in m), scaled to the full m."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    S_np, v_np, m_avail = _host_inputs(SEED)

    def sample(m_s):
        t0 = time.perf_counter()
        oracle.solve(S_np[:, :m_s], v_np[:m_s], LAMBDA)
        return time.perf_counter() - t0

    m_s = min(1 << 14, m_avail)
    dt = sample(m_s)
    budget = 150.0 / max(1, args.steps + args.warmup)
    while dt * 2 < budget and m_s * 2 <= m_avail:
        m_s *= 2
        dt = sample(m_s)
    for _ in range(args.warmup):
        sample(m_s)
    times = [sample(m_s) for _ in range(args.steps)]
    per_full = statistics.mean(times) * (M_PARAMS / m_s)
    value = 1.0 / per_full
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_full * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"each step: FP64 oracle on the first {m_s} of {M_PARAMS} columns, "
                                   f"scaled by {m_s}/{M_PARAMS} (cost linear in m)"},
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

    S, v = _make_inputs(torch, wl, dev, SEED + rank)
    n, m = S.shape
    X = torch.empty_like(v)
    stream = torch.cuda.current_stream()

    def solve(lam=LAMBDA, prec=PRECISION, out=X, timing=False):
        dfs.dfs_solve(S, v, lam, X=out, precision=prec, sync=False, timing=timing)

    # ---------------- mixed path (headline), per-kernel CUDA events inside the timed region ----
    # The solve's launch sequence is fixed (no host round trip), so it is captured once into a CUDA
    # graph and the timed steps replay it: every kernel of the solve runs each step, without the
    # per-launch host overhead.  The step events are part of the graph.
    for _ in range(args.warmup):
        solve()
    info = dfs.dfs_sync_info()
    if info["status"] != 0:
        raise RuntimeError(f"mixed solve failed: {info}")
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    launches_cap0 = dfs.dfs_kernel_launches()
    with torch.cuda.graph(graph, stream=cap):
        solve(timing=True)
    per_solve_launches = dfs.dfs_kernel_launches() - launches_cap0
    stream.wait_stream(cap)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    info = dfs.dfs_sync_info()
    if info["status"] != 0:
        raise RuntimeError(f"mixed solve (graph replay) failed: {info}")
    # (no dfs_step_times reset here: the captured solve left one timed slot pending, and every
    # replay re-records that slot's events, so after the timed replays it holds the last one's)
    clocks_proc = _clock_sampler(local)
    time.sleep(0.3)
    barrier()
    elapsed_ms = _timed(torch, stream, graph.replay, args.steps)
    barrier()
    launches = per_solve_launches * args.steps
    clocks = _clock_summary(clocks_proc)
    info = dfs.dfs_sync_info()
    step_ms, nsteps_timed = dfs.dfs_step_times()
    nsteps_timed = args.steps  # the graph's events are re-recorded by every replay
    elapsed_ms = _max_over_ranks(elapsed_ms, dist, dev)
    value = _job_rate(ws, args.steps, elapsed_ms / 1e3)
    X_mixed = X.clone()

    # ---------------- same workload at lambda = 1e-2 ----------------
    X2 = torch.empty_like(v)
    solve(LAMBDA_ALT, out=X2)
    k2 = max(3, args.steps // 4)
    alt_ms = _timed(torch, stream, lambda: solve(LAMBDA_ALT, out=X2), k2)
    info_alt = dfs.dfs_sync_info()

    # ---------------- plain FP32 path ----------------
    Xf = torch.empty_like(v)
    solve(prec="fp32", out=Xf)
    kf = max(3, args.steps // 10)
    dfs.dfs_step_times()
    fp32_ms = _timed(torch, stream, lambda: solve(prec="fp32", out=Xf, timing=True), kf)
    info_f = dfs.dfs_sync_info()
    fp32_steps, _ = dfs.dfs_step_times()

    # ---------------- end to end through the host-memory entry point ----------------
    S_h = torch.empty(S.shape, dtype=S.dtype, pin_memory=True)
    S_h.copy_(S)
    v_h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
    v_h.copy_(v)
    X_h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
    del S
    torch.cuda.empty_cache()
    # every step uploads S and v from pinned host memory and downloads x; consecutive steps overlap
    # one step's upload with the previous step's solve (dfs_solve_host_async)
    for _ in range(2):
        dfs.dfs_solve_host_async(S_h, v_h, LAMBDA, X_h, precision=PRECISION)
    torch.cuda.synchronize()
    # the host -> device link rate of this machine (plain uploads of S, the best of three: the first
    # touches fresh device memory), which bounds the e2e value
    S_probe = torch.empty(S_h.shape, dtype=S_h.dtype, device=dev)
    best_s = None
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S_probe.copy_(S_h, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        best_s = dt if best_s is None else min(best_s, dt)
    link_gbs = S_h.numel() * S_h.element_size() / best_s / 1e9
    del S_probe
    torch.cuda.empty_cache()
    ke = max(3, args.steps // 10)
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        dfs.dfs_solve_host_async(S_h, v_h, LAMBDA, X_h, precision=PRECISION)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    info_e2e = dfs.dfs_sync_info()
    if info_e2e["status"] != 0:
        raise RuntimeError(f"host-path solve failed: {info_e2e}")
    e2e_s = _max_over_ranks(e2e_s, dist, dev)
    e2e_value = _job_rate(ws, ke, e2e_s)

    peaks_live = _live_peaks(torch, dfs)

    # ---------------- rooflines from the live per-kernel events ----------------
    # Algorithmic work is the method's own (Algorithm 1 with Q inlined): S and the vectors it reads
    # and writes, and the n (n + 1) m flops of the symmetric Gram.  Bytes the design adds (the
    # BF16 tiles it writes and re-reads) are not counted there; they show in `traffic` (ncu) and
    # in traffic / algorithmic.  A kernel timed inside a milliseconds-long step takes the burst peaks.
    peaks, peak_kind = _peaks()
    hbm = peaks["hbm_gbs"]
    bf16 = peaks["bf16_tflops"]
    gram_ms, svp_ms, pass_ms, chol_ms = step_ms[0], step_ms[5], step_ms[6], step_ms[7]
    # the fused first pass has no separate S v pass: its two marks are adjacent (a few us apart)
    fused = svp_ms < 0.05 * gram_ms
    pass_bytes = 4.0 * n * m + 8.0 * m            # S, v read; x written (first refinement pass)
    sv_bytes = 4.0 * n * m + 4.0 * m              # S, v read (b = S v; the Gram reads S once with it)
    gram_flop = float(n) * (n + 1) * m            # lower triangle incl. diagonal, 2 flop / MAC
    passes = max(1, info["passes"])  # full passes over S; a final correction reads the BF16 tiles

    def hbm_line(name, nbytes, ms, launches_per_step, extra=None):
        ach = nbytes / (ms / 1e3) / 1e9 if ms > 0 else None
        traffic = _kernel_traffic(name)
        d = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
             "frac": ach / hbm if ach else None, "traffic": traffic,
             "traffic_over_algorithmic": traffic / nbytes if traffic else None,
             "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": ms,
             "launches_per_step": launches_per_step, "ms_per_step": ms * launches_per_step}
        if extra:
            d.update(extra)
        return d

    pass_line = hbm_line("fisher_pass_cluster_kernel", pass_bytes, pass_ms, passes)
    kernels = [pass_line]
    gram_tf = gram_flop / (gram_ms / 1e3) / 1e12 if gram_ms > 0 else None
    if fused:
        # one kernel streams S (HBM) and runs the Gram (tensor cores): its bound is the larger of
        # the two times at peak, 4 n m / HBM against n (n + 1) m / BF16
        t_hbm, t_tc = sv_bytes / (hbm * 1e9), gram_flop / (bf16 * 1e12)
        kernels.append(hbm_line("gram_fused_kernel", sv_bytes, gram_ms, 1, {
            "tensor_achieved_tflops": gram_tf, "tensor_peak_tflops": bf16,
            "tensor_frac": gram_tf / bf16 if gram_tf else None, "algorithmic_flop_per_launch": gram_flop,
            "bound_ms_at_peak": max(t_hbm, t_tc) * 1e3, "bound_frac": max(t_hbm, t_tc) * 1e3 / gram_ms if gram_ms else None}))
    else:
        svp_name = "sv_ring_kernel" if n <= 1024 else "sv_pack_kernel"
        kernels.append(hbm_line(svp_name, sv_bytes, svp_ms, 1))
        kernels.append({"kernel": "gram_tc_kernel", "bound": "tensor", "achieved": gram_tf, "peak": bf16,
                        "unit": "TFLOP/s", "frac": gram_tf / bf16 if gram_tf else None,
                        "traffic": _kernel_traffic("gram_tc_kernel"), "algorithmic_flop_per_launch": gram_flop,
                        "avg_launch_ms": gram_ms, "launches_per_step": 1, "ms_per_step": gram_ms})
    corr_ms = step_ms[8]
    if corr_ms > 0:
        # x -= S_bf16^T dy / lambda: the refinement's last correction, reading the BF16 tiles the
        # design keeps (2 bytes an entry of S) and x read and written
        n_rows = -(-n // 256) * 256
        corr_bytes = 2.0 * n_rows * (-(-m // 64) * 64) + 8.0 * m
        kernels.append(hbm_line("tile_correct_kernel", corr_bytes, corr_ms, 1))
    kernels.append({"kernel": "chol_coop_kernel", "bound": "latency", "avg_launch_ms": chol_ms,
                    "launches_per_step": 1, "ms_per_step": chol_ms,
                    "note": "31 dependent 32-wide block steps; n^3/3 = %.2e flop" % (n ** 3 / 3.0)})
    roofline = dict(max((k for k in kernels if k["bound"] != "latency"), key=lambda d: d["ms_per_step"]))
    # the plain FP32 path's Gram (SIMT, FP32 fused multiply-adds) against the measured FFMA rate
    ffma = peaks_live.get("ffma32_tflops")
    fp32_gram_tf = gram_flop / (fp32_steps[0] / 1e3) / 1e12 if fp32_steps[0] > 0 else None
    fp32_gram_line = {"kernel": "gram_simt_kernel (plain FP32 path)", "bound": "ffma", "achieved": fp32_gram_tf,
                      "peak": ffma, "unit": "TFLOP/s",
                      "frac": fp32_gram_tf / ffma if (fp32_gram_tf and ffma) else None,
                      "avg_launch_ms": fp32_steps[0], "peak_source": "live dfs_measure_peak(ffma32)"}
    roofline["peak_source"] = f"{peak_kind} MEASURED_PEAKS (hbm_gbs; bf16_tflops burst for the tensor side)"
    roofline["launches_averaged"] = nsteps_timed
    # the whole step against Algorithm 1's own work: S read twice (Gram + b, then x), v read twice,
    # x written; the Gram's flops
    step_s = (elapsed_ms / args.steps) / 1e3
    alg_bytes = 2 * 4.0 * n * m + 12.0 * m
    step_roofline = {"algorithmic_bytes": alg_bytes, "algorithmic_flop": gram_flop,
                     "achieved_gbs": alg_bytes / step_s / 1e9, "frac_hbm": alg_bytes / step_s / 1e9 / hbm,
                     "achieved_tflops": gram_flop / step_s / 1e12, "frac_tensor": gram_flop / step_s / 1e12 / bf16,
                     "bound_ms_at_peak": alg_bytes / (hbm * 1e9) * 1e3 + 0.0,
                     "note": "Algorithm 1 reads S twice; the refinement's extra pass and the tile "
                             "correction are the design's"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic", "config": workload_config(),
        "step_ms": {"gram" if not fused else "fused_first_pass": step_ms[0], "finalize_cholesky": step_ms[1],
                    "first_solve": step_ms[2], "refinement": step_ms[3], "total": step_ms[4],
                    "sv_kernel": step_ms[5], "first_refinement_pass_kernel": step_ms[6],
                    "cholesky_kernel": step_ms[7], "tile_correct_kernel": step_ms[8]},
        "fp32_path": {"value": kf / (fp32_ms / 1e3), "unit": UNIT, "steps": kf, "status": info_f["status"],
                      "gram_roofline": fp32_gram_line,
                      "mixed_over_fp32": (args.steps / (elapsed_ms / 1e3)) / (kf / (fp32_ms / 1e3))},
        "peaks_live": peaks_live,
        "lambda_1e-2": {"value": k2 / (alt_ms / 1e3), "unit": UNIT, "iters": info_alt["iters"], "steps": k2},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n * m + 4 * m,
                "d2h_bytes_per_step": 4 * m, "steps": ke,
                "api": "dfs_solve_host_async (pinned host S, v, x; upload of step i+1 overlaps the solve of step i)",
                "h2d_link_gbs": link_gbs,
                "upload_bound_value": link_gbs * 1e9 / (4.0 * n * m + 4.0 * m)},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline,
        "step_roofline": step_roofline,
        "kernels": kernels,
        "mixed_info": {"iters": info["iters"], "full_passes": info["passes"], "est_rel_err": info["rel_correction"],
                       "status": info["status"]},
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the FP64 oracle on the full problem: accuracy of every reported solution, and its own
        # time on the host cores as the CPU baseline
        S64 = S_h.double().numpy()
        v64 = v_h[0].double().numpy()
        x_ref, t_ref = _oracle_solve(S64, v64, LAMBDA)
        acc = {"mixed": _errors(S64, v64, LAMBDA, X_mixed.cpu().double().numpy()[0], x_ref),
               "fp32_path": _errors(S64, v64, LAMBDA, Xf.cpu().double().numpy()[0], x_ref)}
        x_ref2, _ = _oracle_solve(S64, v64, LAMBDA_ALT)
        acc["mixed_lambda_1e-2"] = _errors(S64, v64, LAMBDA_ALT, X2.cpu().double().numpy()[0], x_ref2)
        line["accuracy_vs_fp64_oracle"] = acc
        line["accuracy_ok"] = acc["mixed"]["e_rel"] <= 1e-6 and acc["fp32_path"]["e_rel"] <= 1e-5
        line["cpu_baseline"] = {"value": 1.0 / t_ref, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "cpu_model": _cpu_model(),
                                "sample": f"one full FP64 oracle solve of this workload (n={n}, m={m}, k=1, "
                                          f"lambda={LAMBDA:g}) in {t_ref:.2f} s, numpy with its default "
                                          f"BLAS threads on {os.cpu_count()} host cores",
                                "small_config_fp64_n256_m16384": _oracle_config1_times()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _residual_fp64(torch, S, X, V, lam, chunk=1 << 18):
    """||S^T S x + lam x - v|| / ||v|| per RHS in FP64 (torch, column chunks of S)."""
    n, m = S.shape
    k = V.shape[0]
    Sx = torch.zeros((n, k), device=S.device, dtype=torch.float64)
    for c0 in range(0, m, chunk):
        Sx += S[:, c0:c0 + chunk].double() @ X[:, c0:c0 + chunk].double().T
    num = torch.zeros(k, device=S.device, dtype=torch.float64)
    for c0 in range(0, m, chunk):
        r = (S[:, c0:c0 + chunk].double().T @ Sx).T + lam * X[:, c0:c0 + chunk].double() - V[:, c0:c0 + chunk].double()
        num += (r * r).sum(dim=1)
    return (num.sqrt() / V.double().norm(dim=1)).cpu().tolist()


def run_workload(args):
    """The other configurations, on one GPU, one JSON line per path:
      precision  n=4096, m=2^22, k=4, FP32 S with singular values log-spaced 1/sqrt(n) .. 1e-4/sqrt(n),
                 lambda=1e-4; BF16 and FP8 Gram.  cond(A) ~ 3.4, so the FP64 residual bounds e_rel.
      batch      64 independent problems, n ~ U{64..1024}, m log-uniform in [1e4, 5e5], lambda log-uniform
                 in [1e-5, 1e-1], k=8; dfs_solve_batched (concurrency from dfs_autotune_batched) against
                 one dfs_solve after another and against the plain FP32 path on the same batch.
      complex    n=512, m=2^18, k=1 complex SR: dfs_solve_complex on stacked planes against dfs_solve on
                 the real 2n x 2m representation of the same problem.
      stress     n=8192, m=2^22, BF16 S with Student-t entries and log-normal column scales,
                 lambda=1e-5, k=1; the FP64 residual against the FP32-storage floor of x.
    Each timed region holds the solves only (inputs resident in HBM and larger than L2)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2310_17556_gb300 as dfs
    from paper_2310_17556_gb300 import workloads as wl

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = 231017556
    steps, warmup = max(1, min(args.steps, 5)), 3

    def timed(fn, k_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(k_steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k_steps

    def emit(line):
        line.update({"n_gpus": 1, "steps": steps, "warmup": warmup, "higher_is_better": True, "scaling": "weak",
                     "vs_baseline": None, "data": "synthetic"})
        print(json.dumps(line), flush=True)

    if args.workload == "precision":
        n, m, k, lam = 4096, 1 << 22, 4, 1e-4
        S = wl.svd_structured_lowmem(n, m, seed=base + 3, sigma_min=1e-4, device=dev)
        V = wl.rhs(m, k, seed=base + 10, device=dev)
        cond = (1.0 / n + lam) / lam
        for prec in ("bf16", "fp8"):
            X = torch.empty_like(V)
            fn = lambda: dfs.dfs_solve(S, V, lam, X=X, precision=prec, sync=False, timing=True)
            for _ in range(warmup):
                fn()
            dfs.dfs_step_times()
            clk = _clock_sampler(0)
            ms = timed(fn, steps)
            clocks = _clock_summary(clk)
            info = dfs.dfs_sync_info()
            st, _ = dfs.dfs_step_times()
            res = _residual_fp64(torch, S, X, V, lam)
            emit({"workload": "precision", "metric": "solves/s, n=4096 m=2^22 k=4", "value": 1e3 / ms,
                  "unit": "solves/s", "ms_per_step": ms, "dtype": prec, "clocks": clocks,
                  "config": {"n": n, "m": m, "k": k, "lambda": lam, "S": "FP32, sigma log-spaced 1..1e-4 (/sqrt n)"},
                  "info": {"status": info["status"], "iters": info["iters"], "full_passes": info["passes"]},
                  "step_ms": {"gram": st[0], "finalize_cholesky": st[1], "first_solve": st[2], "rest": st[3],
                              "sv_kernel": st[5], "first_refinement_pass_kernel": st[6], "cholesky_kernel": st[7],
                              "tile_correct_kernel": st[8]},
                  "accuracy": {"fp64_residual_max": max(res), "bound_e_rel": cond * max(res),
                               "ok": cond * max(res) <= 1e-6}})
    elif args.workload == "batch":
        shapes = wl.ragged_batch_shapes(64, seed=base + 4)
        probs = []
        for j, (n, m, lam) in enumerate(shapes):
            m = (m + 3) // 4 * 4
            S = wl.gaussian(n, m, seed=base + 400 + j, device=dev)
            V = wl.rhs(m, 8, seed=base + 700 + j, device=dev)
            probs.append((S, V, lam, torch.empty_like(V)))
        # concurrency chosen by the library's autotuner on this batch (lanes x SM share)
        tune = dfs.dfs_autotune_batched(probs, precision="bf16")
        batch = lambda: dfs.dfs_solve_batched(probs, precision="bf16", sync=False)
        loop = lambda: [dfs.dfs_solve(S, V, lam, X=X, precision="bf16", sync=False) for S, V, lam, X in probs]
        for fn in (batch, loop):
            for _ in range(warmup):
                fn()
        clk = _clock_sampler(0)
        ms_b = timed(batch, steps)
        clocks = _clock_summary(clk)
        ms_l = timed(loop, steps)
        _, status = dfs.dfs_solve_batched(probs, precision="bf16")
        X_mixed = [X.clone() for _, _, _, X in probs]
        # the plain FP32 path (SIMT Gram, no refinement) on the same batch
        fp32 = lambda: dfs.dfs_solve_batched(probs, precision="fp32", sync=False)
        fp32()
        ms_f = timed(fp32, max(1, min(steps, 3)))
        _, status_f = dfs.dfs_solve_batched(probs, precision="fp32")
        X_fp32 = [X.clone() for _, _, _, X in probs]
        import oracle

        import numpy as np

        # the oracle on a spread of the batch: the smallest, the median and the largest problem by
        # cost n^2 m + 4 n m k; the batch's CPU time from a fit t = a + b cost over the three
        cost = lambda p: p[0].shape[0] ** 2 * p[0].shape[1] + 4 * p[0].shape[0] * p[0].shape[1] * p[1].shape[0]
        by_cost = sorted(range(len(probs)), key=lambda j: cost(probs[j]))
        sample = [by_cost[0], by_cost[len(by_cost) // 2], by_cost[-1]]
        samples, err_mixed, err_fp32 = [], [], []
        for j in sample:
            S, V, lam, _ = probs[j]
            s64, v64 = S.double().cpu().numpy(), V.double().cpu().numpy().T
            t0 = time.perf_counter()
            ref = oracle.solve(s64, v64, lam).T
            dt = time.perf_counter() - t0
            rel = lambda X: float(np.max(np.linalg.norm(X.double().cpu().numpy() - ref, axis=1) /
                                         np.linalg.norm(ref, axis=1)))
            err_mixed.append(rel(X_mixed[j]))
            err_fp32.append(rel(X_fp32[j]))
            samples.append({"n": S.shape[0], "m": S.shape[1], "k": V.shape[0], "s": round(dt, 3)})
            del s64, v64, ref
        cs = np.array([float(cost(probs[j])) for j in sample])
        ts = np.array([x["s"] for x in samples])
        b_fit, a_fit = np.polyfit(cs, ts, 1)
        a_fit = max(float(a_fit), 0.0)
        t_all = sum(a_fit + float(b_fit) * cost(p) for p in probs)
        ok = all(x == 0 for x in status) and max(err_mixed) <= 1e-6
        emit({"workload": "batch", "metric": "problems/s, 64 ragged problems, k=8", "value": 64e3 / ms_b,
              "unit": "problems/s", "ms_per_step": ms_b, "dtype": "bf16", "clocks": clocks,
              "autotune": {"lanes": tune["lanes"], "share": tune["share"], "ms": tune["ms"]},
              "sequential": {"value": 64e3 / ms_l, "ms_per_step": ms_l, "api": "one dfs_solve after another"},
              "fp32_path": {"value": 64e3 / ms_f, "ms_per_step": ms_f, "statuses_ok": all(x == 0 for x in status_f),
                            "e_rel_sampled_vs_oracle": err_fp32,
                            "note": "the plain FP32 path (FFMA Gram, no refinement) on the same batch"},
              "config": {"problems": 64, "n": "U{64..1024}", "m": "log-uniform [1e4, 5e5]",
                         "lambda": "log-uniform [1e-5, 1e-1]", "k": 8,
                         "S_bytes": sum(p[0].numel() * 4 for p in probs)},
              "accuracy": {"statuses_ok": all(x == 0 for x in status), "e_rel_sampled_vs_oracle": err_mixed,
                           "ok": ok},
              "cpu_baseline": {"value": len(probs) / t_all, "unit": "problems/s", "cores": os.cpu_count(),
                               "kind": "oracle", "samples": samples,
                               "fit": {"a_s": a_fit, "b_s_per_cost": float(b_fit)},
                               "sample": "FP64 oracle on the smallest, median and largest problem by cost "
                                         "n^2 m + 4 n m k; batch time from the fit t = a + b cost"}})
    elif args.workload == "complex":
        # complex SR (Section 4): the native route on the stacked planes against the real 2n x 2m
        # representation [[A, -B], [B, A]] solved by dfs_solve (the same Eq. 1), n=512, m=2^18
        n, m, k, lam = 512, 1 << 18, 1, 1e-3
        Z = torch.cat([wl.gaussian(n, m, seed=base + 20, device=dev), wl.gaussian(n, m, seed=base + 21, device=dev)],
                      dim=0) / 2 ** 0.5
        A, B = Z[:n], Z[n:]
        Vr, Vi = wl.rhs(m, k, seed=base + 22, device=dev), wl.rhs(m, k, seed=base + 23, device=dev)
        RS = torch.cat([torch.cat([A, -B], dim=1), torch.cat([B, A], dim=1)], dim=0)
        V2 = torch.cat([Vr, Vi], dim=1)
        native = lambda: dfs.dfs_solve_complex(A, B, Vr, Vi, lam, precision="bf16")
        real2 = lambda: dfs.dfs_solve(RS, V2, lam, precision="bf16")
        for fn in (native, real2):
            for _ in range(warmup):
                fn()
        clk = _clock_sampler(0)
        ms_c = timed(native, steps)
        clocks = _clock_summary(clk)
        ms_r = timed(real2, steps)
        Xr, Xi, info = native()
        X2, _ = real2()
        import oracle

        import numpy as np

        S64 = (A.double() + 1j * B.double()).cpu().numpy()
        ref = oracle.solve_complex(S64, (Vr.double() + 1j * Vi.double()).cpu().numpy().T, lam).T
        rel = lambda X: float(np.max(np.linalg.norm(X - ref, axis=1) / np.linalg.norm(ref, axis=1)))
        e_native = rel((Xr.double() + 1j * Xi.double()).cpu().numpy())
        x2 = X2.double().cpu().numpy()
        e_real2 = rel(x2[:, :m] + 1j * x2[:, m:])
        emit({"workload": "complex", "metric": "complex solves/s, n=512 m=2^18 k=1", "value": 1e3 / ms_c,
              "unit": "solves/s", "ms_per_step": ms_c, "dtype": "bf16", "clocks": clocks,
              "real_representation": {"ms_per_step": ms_r, "ratio_native_over_real": ms_c / ms_r,
                                      "api": "dfs_solve on [[A, -B], [B, A]] (2n x 2m, formed beforehand)"},
              "config": {"n": n, "m": m, "k": k, "lambda": lam, "S": "complex Gaussian, planes stacked in one array"},
              "accuracy": {"status": info["status"], "e_rel_native_vs_oracle": e_native,
                           "e_rel_real_representation_vs_oracle": e_real2, "ok": e_native <= 1e-6}})
    elif args.workload == "stress":
        n, m, lam = 8192, 1 << 22, 1e-5
        S = wl.heavy_tailed(n, m, seed=base + 5, device=dev, dtype=torch.bfloat16)
        V = wl.rhs(m, 1, seed=base + 12, device=dev)
        X = torch.empty_like(V)
        fn = lambda: dfs.dfs_solve(S, V, lam, X=X, precision="bf16", max_iter=12, sync=False, timing=True)
        for _ in range(warmup):
            fn()
        dfs.dfs_step_times()
        clk = _clock_sampler(0)
        ms = timed(fn, steps)
        clocks = _clock_summary(clk)
        info = dfs.dfs_sync_info()
        st, _ = dfs.dfs_step_times()
        res = _residual_fp64(torch, S, X, V, lam)
        # ||S||_2^2 by power iteration, for the FP32-storage floor 2^-24 (||S||^2 + lambda) ||x|| / ||v||
        u = torch.randn(n, device=dev, generator=torch.Generator(device=dev).manual_seed(7))
        u /= u.norm()
        s2 = 0.0
        for _ in range(30):
            w = torch.zeros(n, device=dev)
            for c0 in range(0, m, 1 << 18):
                Sc = S[:, c0:c0 + (1 << 18)].float()
                w += Sc @ (Sc.T @ u)
            s2 = float(torch.dot(u, w))
            u = w / w.norm()
        floor = 2.0 ** -24 * (s2 + lam) * float(X.double().norm() / V.double().norm())
        emit({"workload": "stress", "metric": "solves/s, n=8192 m=2^22 BF16 S heavy-tailed", "value": 1e3 / ms,
              "unit": "solves/s", "ms_per_step": ms, "dtype": "bf16", "clocks": clocks,
              "config": {"n": n, "m": m, "k": 1, "lambda": lam, "S": "BF16, Student-t(3) x log-normal columns / sqrt n"},
              "info": {"status": info["status"], "iters": info["iters"], "full_passes": info["passes"]},
              "step_ms": {"gram": st[0], "finalize_cholesky": st[1], "first_solve": st[2], "rest": st[3],
                          "sv_kernel": st[5], "first_refinement_pass_kernel": st[6], "cholesky_kernel": st[7],
                          "tile_correct_kernel": st[8]},
              "accuracy": {"fp64_residual": res[0], "fp32_storage_floor": floor, "sigma_max_sq": s2,
                           "ok": res[0] <= 2 * floor}})
    return 0


def run_profile_solve(args):
    """One small BF16 solve for an ncu capture (--profile-solve M): Gaussian S of n x M
    (--profile-n, default 1024; FP32, or BF16 with --profile-bf16; seed 1), V (--profile-k right-hand
    sides, default 1) seed 2, lambda 1e-4,
    after --warmup solves.  Prints the device status."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2310_17556_gb300 as dfs
    from paper_2310_17556_gb300 import workloads as wl

    torch.cuda.set_device(0)
    n = args.profile_n or N_SAMPLES
    S = wl.gaussian(n, args.profile_solve, seed=1, device="cuda",
                    dtype=torch.bfloat16 if args.profile_bf16 else torch.float32)
    v = wl.rhs(args.profile_solve, args.profile_k or 1, seed=2, device="cuda")
    X = torch.empty_like(v)
    for _ in range(args.warmup + 1):
        dfs.dfs_solve(S, v, LAMBDA, X=X, precision=PRECISION, sync=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": {"n": n, "m": args.profile_solve, "s_dtype": str(S.dtype),
                                        **dfs.dfs_sync_info()}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["headline", "precision", "batch", "stress", "complex"], default="headline",
                    help="headline (default): the metric's workload; the others: one GPU, one line per path")
    ap.add_argument("--profile-solve", type=int, default=0, metavar="M",
                    help="run one small solve (n=1024, m=M) after --warmup solves, for ncu captures")
    ap.add_argument("--profile-n", type=int, default=0, metavar="N", help="rows of S for --profile-solve")
    ap.add_argument("--profile-bf16", action="store_true", help="BF16 S for --profile-solve")
    ap.add_argument("--profile-k", type=int, default=0, metavar="K", help="right-hand sides for --profile-solve")
    args = ap.parse_args()
    if args.profile_solve:
        return run_profile_solve(args)
    if args.workload != "headline" and args.impl == "ours":
        return run_workload(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
