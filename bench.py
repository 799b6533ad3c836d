#!/usr/bin/env python3
"""ANLS-BPP NMF benchmark: iterations per second of the whole per-iteration hot
path (Gram H H^T, A H^T, BPP for W, Gram W^T W, W^T A, BPP for H, objective)
on one GB300, with roofline, clocks, end-to-end and CPU-oracle numbers.

Default workload: the dense 96000 x 64000, k = 50 recipe (A = W0 H0 +
|N(0, 0.05^2)|, 24.6 GB FP32, inputs larger than L2), warm-started BPP.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16x3]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

With N > 1 (torchrun), every rank runs an independent replica of the workload
(the method has no exchange step on one GPU: replicas only); value counts the
iterations of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (m, n, k, sigma, description)
    "dense-large": (96000, 64000, 50, 0.05,
                    "dense A=W0*H0+|N(0,0.05^2)| 96000x64000 k=50 fp32 (24.6 GB)"),
    "dense-medium": (24000, 16000, 50, 0.05,
                     "dense A=W0*H0+|N(0,0.05^2)| 24000x16000 k=50 fp32 (1.5 GB)"),
    "dense-small": (2000, 1000, 10, 0.01,
                    "dense A=W0*H0+|N(0,0.01^2)| 2000x1000 k=10 fp32"),
    "dense-video": (1013400, 2400, 50, 0.05,
                    "dense A=W0*H0+|N(0,0.05^2)| 1013400x2400 k=50 fp32 (9.7 GB; the shape of the "
                    "paper's Video matrix, synthetic)"),
    "sparse-large": (2000000, 1000000, 50, None,
                     "sparse CSR 2000000x1000000, 20M uniform draws, values U(0,1], k=50"),
    "sparse-medium": (200000, 100000, 50, None,
                      "sparse CSR 200000x100000, 2M uniform draws, values U(0,1], k=50"),
}
# Sparse workloads: number of uniform position draws (duplicates merged).
SPARSE_DRAWS = {"sparse-large": 20000000, "sparse-medium": 2000000}
# The batched-NLS stress workload: one step is one nmf_nls_bpp call on the
# whole batch (its metric is right-hand sides per second, not iterations).
STRESS = "bpp-stress"
STRESS_ROWS, STRESS_K, STRESS_NRHS = 200000, 100, 1000000
# name: (mean of a, description). With a uniform in [0, 1) every solution is
# positive (the all-passive group); a = u - 0.45 gives solutions of mixed
# signs (about 71 of 100 indices passive, 3-4 exchange rounds per
# right-hand side).
STRESS_WORKLOADS = {
    STRESS: (0.5, "batched NLS: 1000000 right-hand sides, k=100; G = W^T W of W 200000x100 "
                  "U[0,1) with 30% zeros; b drawn as W^T a for a U[0,1)^200000 (CLT form)"),
    "bpp-stress-mixed": (0.05, "batched NLS: 1000000 right-hand sides, k=100; the same G; b "
                               "drawn as W^T a for a = u - 0.45, u U[0,1)^200000 (CLT form): "
                               "solutions of mixed signs"),
}
STRESS_METRIC = "BPP right-hand sides/s"
STRESS_CPU_SAMPLE = 300000
STRESS_CHECK = 10000      # right-hand sides of the oracle check (cpu_baseline leg)
SEED = 1509
METRIC = "ANLS-BPP iterations/s"


def metric_name(solver: str) -> str:
    """BPP is the paper's local solver and the headline; MU (Eq. 5) and HALS
    (Eq. 6) run the same iteration with the other update."""
    return METRIC if solver == "bpp" else f"ANLS-{solver.upper()} iterations/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic per launch (read + write bytes) of the dominant kernel from one
# ncu capture, keyed by (kernel, workload, precision); None until captured or
# when the kernel changed since. dense-large: the two mm_tc_kernel launches of
# an iteration captured on the 24000 x 16000 case (A H^T with the objective,
# from the pre-split A: 1.5545 GB read + 7.3 MB written; A^T W from the
# pre-split A^T: 1.5464 GB + 18.8 MB in 6 splits), reads scaled by the element
# ratio 16, writes by the rows (A H^T 96000 x 50 out; A^T W 3 splits of
# 64000 x 50 there), averaged: 24.84 GB per launch against 24.61 GB of
# algorithmic bytes.
MLP_HIDDEN = 256     # width of the proposal network (3k -> 256 -> 256 -> k)

NCU_TRAFFIC = {
    ("mm_tc_kernel", "dense-large", "bf16x3"): 24.84e9,
    ("mm_tc_kernel", "dense-medium", "bf16x3"): 1.5635e9,
}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks: a timed region counts at its slowest
    rank's time. One rank returns x unchanged."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def peaks():
    try:
        with open(MEASURED_PEAKS) as fh:
            p = json.load(fh)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def fp32_peak_probe(nmf, gpu_index: int) -> dict:
    """The FP32 FMA rate this GPU sustains, measured in-process by the
    library's probe (eight independent chains per thread on every SM, scalar
    FFMA and packed FFMA2; CUDA events), with the SM clock sampled while it
    ran. No GPU setting is touched."""
    sampler = ClockSampler(gpu_index)
    sampler.start()
    ffma = nmf.nmf_probe_fp32_fma(packed=False, launches=120) / 1e12
    ffma2 = nmf.nmf_probe_fp32_fma(packed=True, launches=120) / 1e12
    clocks = sampler.stop()
    return {"tflops": max(ffma, ffma2), "ffma_tflops": ffma, "ffma2_tflops": ffma2,
            "sm_mhz": clocks["sm_mhz"] if clocks else None}


def alu_peak(probe: dict, clocks) -> tuple[float, str]:
    """The probe's FP32 rate at the timed region's median SM clock."""
    scale, how = 1.0, "probe clock not sampled"
    if clocks and clocks.get("sm_mhz") and probe.get("sm_mhz"):
        scale = clocks["sm_mhz"] / probe["sm_mhz"]
        how = f"x {clocks['sm_mhz']:.0f} / {probe['sm_mhz']:.0f} MHz (timed / probe median)"
    peak = probe["tflops"] * scale
    src = (f"measured: FP32 FMA probe {probe['tflops']:.1f} TFLOP/s (FFMA {probe['ffma_tflops']:.1f}, "
           f"FFMA2 {probe['ffma2_tflops']:.1f}) {how}")
    return peak, src


def oracle_sample(m, n, k, sigma, steps, warm: bool, solver="bpp"):
    """Time the FP64 oracle (as it stands) on a crop of the workload and scale
    to the full size by m*n (the products and objective dominate; they scale
    with m*n, the NLS work with m+n). Returns (iter/s full-size, sample text,
    threads, seconds per sample step)."""
    import oracle
    import synth
    ms, ns = (min(m, 6000), min(n, 4000)) if m * n > 6000 * 4000 else (m, n)
    A = synth.dense_planted(ms, ns, k, sigma, seed=SEED, n_full=n)
    W0, Ht0 = synth.init_factors(ms, ns, k, seed=SEED)
    orc = oracle.default()
    r = orc.anls(A, W0, Ht0, iters=1, warm=warm, solver=solver)   # warm-up (first iteration)
    t0 = time.perf_counter()
    orc.anls(A, r["W"].astype("float32"), r["Ht"].astype("float32"), iters=steps, warm=warm,
             solver=solver)
    dt = (time.perf_counter() - t0) / steps
    scale = (m * n) / (ms * ns)
    sample = (f"oracle ANLS iterations on the {ms}x{ns} crop of the same recipe (k={k}), "
              f"{steps} iterations, time per iteration x {scale:.1f} (m*n ratio)")
    return 1.0 / (dt * scale), sample, orc.num_threads(), dt


def oracle_sample_sparse(m, n, k, draws, steps, warm: bool, csr, solver="bpp"):
    """Time the FP64 oracle on the top-left (m/20) x (n/20) block of the same
    CSR matrix and scale by the row-plus-column ratio (the NLS work, one solve
    per row and per column, dominates the sparse iteration)."""
    import numpy as np
    import oracle
    import synth
    rowptr, colidx, vals = csr
    ms, ns = max(1, m // 20), max(1, n // 20)
    keep_r = np.zeros(len(colidx), dtype=bool)
    keep_r[:rowptr[ms]] = True
    keep = keep_r & (colidx < ns)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rowptr))
    r_c, c_c, v_c = rows[keep], colidx[keep], vals[keep]
    rp = np.zeros(ms + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(r_c, minlength=ms))
    W0, Ht0 = synth.init_factors(ms, ns, k, seed=SEED)
    orc = oracle.default()
    crop = (rp, np.ascontiguousarray(c_c), np.ascontiguousarray(v_c))
    r = orc.anls(None, W0, Ht0, iters=1, warm=warm, csr=crop, shape=(ms, ns), solver=solver)
    t0 = time.perf_counter()
    orc.anls(None, r["W"].astype("float32"), r["Ht"].astype("float32"), iters=steps, warm=warm,
             csr=crop, shape=(ms, ns), solver=solver)
    dt = (time.perf_counter() - t0) / steps
    scale = (m + n) / (ms + ns)
    sample = (f"oracle ANLS iterations on the top-left {ms}x{ns} block of the same CSR "
              f"({len(c_c)} nonzeros, k={k}), {steps} iterations, time per iteration x "
              f"{scale:.1f} (rows+columns ratio)")
    return 1.0 / (dt * scale), sample, orc.num_threads(), dt


def stress_oracle_sample(G, B, n, keep=0):
    """The FP64 oracle (as it stands) on the first n right-hand sides of the
    stress batch. Returns (right-hand sides per second, sample text, threads,
    seconds, the oracle's (X, passive, rounds) of the first `keep`)."""
    import oracle
    Gh = G.cpu().numpy()
    Bs = B[:n].double().cpu().numpy()
    oracle.bpp(Gh, Bs[:100])                    # warm-up
    t0 = time.perf_counter()
    Xo, Po, Ro, _, _ = oracle.bpp(Gh, Bs)
    dt = time.perf_counter() - t0
    return (n / dt, f"oracle BPP on the first {n} right-hand sides of the same batch",
            oracle.num_threads(), dt, (Xo[:keep], Po[:keep], Ro[:keep]))


def stress_oracle_check(nmf, G, B, r, kept, k, margin):
    """The GPU's solutions of the first right-hand sides against the oracle's
    (kept from the timed oracle sample): relative error against the FP32
    bound 20 cond(G) 6e-8, and passive sets and round counts on the
    right-hand sides whose KKT margin is clear (every passive x_i at least
    margin max|x|, every active y_i at least margin max|b|)."""
    import numpy as np
    Xo, Po, Ro = kept
    n = Xo.shape[0]
    Gh = G.cpu().numpy()
    Bs = B[:n].double().cpu().numpy()
    X = r["X"][:n].double().cpu().numpy()
    P = nmf.passive_to_bool(r["passive"][:n], k).cpu().numpy()
    R = r["rounds"][:n].cpu().numpy()
    Pb = Po.astype(bool)
    cond = float(np.linalg.cond(Gh))
    err = float(np.linalg.norm(X - Xo) / np.linalg.norm(Xo))
    Y = Xo @ Gh - Bs
    xm = np.where(Pb, Xo, np.inf).min(axis=1) / np.maximum(np.abs(Xo).max(axis=1), 1e-300)
    ym = np.where(~Pb, Y, np.inf).min(axis=1) / np.maximum(np.abs(Bs).max(axis=1), 1e-300)
    ok = np.minimum(xm, ym) >= margin
    return {"rhs": int(n), "rel_err": err, "bound": 20 * cond * 6e-8, "cond": cond,
            "margin": margin, "margin_clear": float(ok.mean()),
            "passive_equal_margin_clear": float((P[ok] == Pb[ok]).all(axis=1).mean())
            if ok.any() else None,
            "rounds_equal_margin_clear": float((R[ok] == Ro[ok]).mean()) if ok.any() else None,
            "passive_equal_all": float((P == Pb).all(axis=1).mean())}


def run_stress_reference(args, world):
    import torch

    from synth import torch_gen
    mean_a, desc = STRESS_WORKLOADS[args.workload]
    G, B = torch_gen.stress_batch_device(torch.device("cpu"), STRESS_ROWS, STRESS_K,
                                         max(STRESS_CPU_SAMPLE // 10, 1000), mean_a=mean_a)
    steps = max(1, args.steps)
    total_n, total_s = 0, 0.0
    for _ in range(steps):
        v, sample, cores, dt, _ = stress_oracle_sample(G, B, B.shape[0])
        total_n += B.shape[0]
        total_s += dt
    value = total_n / total_s
    line = {"impl": "reference", "metric": STRESS_METRIC, "value": value, "unit": "RHS/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * STRESS_NRHS / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                             "sample": sample + f", {steps} times"},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_stress(args, rank, world, local_rank):
    """Times K nmf_nls_bpp calls on the stress batch (one call = one step)."""
    import torch
    import torch.distributed as dist

    import paper_1509_09313_gb300 as nmf
    from synth import torch_gen

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    k, nrhs = STRESS_K, STRESS_NRHS
    mean_a, desc = STRESS_WORKLOADS[args.workload]
    t_gen = time.perf_counter()
    G, B = torch_gen.stress_batch_device(dev, STRESS_ROWS, k, nrhs, mean_a=mean_a)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen

    def barrier():
        if world > 1:
            dist.barrier()

    r = None
    for _ in range(args.warmup):
        r = nmf.nmf_nls_bpp(G, B, max_rounds=args.max_rounds)
    probe = fp32_peak_probe(nmf, local_rank)
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = nmf.nmf_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx is not None:
        nvtx.range_push("timed")    # lets ncu select exactly the timed launches
    for _ in range(args.steps):
        r = nmf.nmf_nls_bpp(G, B, max_rounds=args.max_rounds)
    if nvtx is not None:
        nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = nmf.nmf_kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world, dev)
    value = world * nrhs * args.steps / (ms / 1000.0)

    # Algorithmic work of the last call: per right-hand side and exchange
    # round, 2|F|^2 + 2|F|(k - |F|) flops (a solve through a factor of G_FF
    # and y = G x - g off F), |F| taken from the final passive set. Bytes: B
    # in, X, passive sets, rounds and statuses out.
    rounds = r["rounds"].double()
    f = nmf.passive_to_bool(r["passive"], k).double().sum(dim=1)
    flops = float((rounds * (2 * f * f + 2 * f * (k - f))).sum().item())
    nbytes = 4.0 * nrhs * k * 2 + (8 + 4 + 1) * nrhs
    step_s = ms / 1000.0 / args.steps
    # Rounds per right-hand side, and the share the group-tile pass can take:
    # right-hand sides whose first candidate (every index passive) was final.
    rh = torch.bincount(r["rounds"].long().clamp(min=0)).cpu().tolist()
    group_share = float(((r["rounds"] == 1) & (f == k)).double().mean().item())
    pk, pk_kind = peaks()
    fp32_peak, peak_src = alu_peak(probe, clocks)
    achieved = flops / step_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak,
            "kernel": ("bpp_group_tc_kernel" if nmf.nmf_nls_bpp_get_shape(k)[2] == 2
                       else "bpp_group_kernel") if group_share >= 0.5 else "bpp_solve32_kernel",
            "timed": "the whole nmf_nls_bpp call (all its kernels)",
            "peak_source": peak_src,
            "achieved_gbs": nbytes / step_s / 1e9, "hbm_frac": nbytes / step_s / 1e9 / pk["hbm_gbs"],
            "traffic": None}

    e2e = None
    if not args.no_e2e:
        B_host = torch.empty((nrhs, k), dtype=torch.float32, pin_memory=True)
        B_host.copy_(B)
        X_host = torch.empty((nrhs, k), dtype=torch.float32, pin_memory=True)
        B_dev = torch.empty_like(B)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            B_dev.copy_(B_host, non_blocking=True)
            r2 = nmf.nmf_nls_bpp(G, B_dev, max_rounds=args.max_rounds)
            X_host.copy_(r2["X"], non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        barrier()
        dt = max_over_ranks(dt, world, dev)
        e2e = {"value": world * nrhs * args.steps / dt, "unit": "RHS/s",
               "h2d_bytes_per_step": 4 * nrhs * k, "d2h_bytes_per_step": 4 * nrhs * k,
               "note": "upload B, nmf_nls_bpp, download X, every step"}

    cpu, check = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample_n = STRESS_CPU_SAMPLE if mean_a >= 0.5 else STRESS_CPU_SAMPLE // 2
        v, sample, cores, _, kept = stress_oracle_sample(G, B, sample_n, keep=STRESS_CHECK)
        cpu = {"value": v, "unit": "RHS/s", "cores": cores, "kind": "oracle", "sample": sample}
        # Mixed partitions have ~30 active indices of 100, so few right-hand
        # sides clear 1e-3; 3e-4 is still ~40 cond(G) 6e-8 (cond ~117).
        check = stress_oracle_check(nmf, G, B, r, kept, k, 1e-3 if mean_a >= 0.5 else 3e-4)

    if rank == 0:
        line = {"metric": STRESS_METRIC, "value": value, "unit": "RHS/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": desc, "seed": SEED, "mean_a": mean_a,
                           "launch_shape": list(nmf.nmf_nls_bpp_get_shape(k)),
                           "l2": f"inputs larger than L2 (B = {4 * nrhs * k / 1e9:.1f} GB)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches,
                "bpp": {"rounds_per_rhs": float(rounds.mean().item()),
                        "rounds_histogram": rh,
                        "passive_per_rhs": float(f.mean().item()),
                        "group_share": group_share, "per_warp_share": 1.0 - group_share,
                        "status": nmf.nmf_status_str(r["worst"])},
                "oracle_check": check,
                "setup_s": {"generate": t_gen}}
        print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload in STRESS_WORKLOADS:
        import oracle
        oracle.build()
        run_stress_reference(args, world)
        return
    m, n, k, sigma, desc = WORKLOADS[args.workload]
    import oracle
    oracle.build()
    steps = max(1, args.steps)
    if args.workload in SPARSE_DRAWS:
        import synth
        csr = synth.csr_uniform(m, n, SPARSE_DRAWS[args.workload], seed=SEED)
        value, sample, cores, dt = oracle_sample_sparse(m, n, k, SPARSE_DRAWS[args.workload],
                                                        steps, args.start == "warm", csr,
                                                        args.solver)
    else:
        value, sample, cores, dt = oracle_sample(m, n, k, sigma, steps, args.start == "warm",
                                                 args.solver)
    line = {"impl": "reference", "metric": metric_name(args.solver), "value": value,
            "unit": "iter/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "start": args.start, "solver": args.solver},
            "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1509_09313_gb300 as nmf
    import synth
    from synth import torch_gen

    m, n, k, sigma, desc = WORKLOADS[args.workload]
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    sparse = args.workload in SPARSE_DRAWS
    if sparse:
        args.precision = "fp32"     # SpMM and the sparse objective have one precision
    t_gen = time.perf_counter()
    csr_host = None
    if sparse:
        csr_host = synth.csr_uniform(m, n, SPARSE_DRAWS[args.workload], seed=SEED)
        A = tuple(torch.from_numpy(x).to(dev) for x in csr_host)
        nnz = int(csr_host[1].size)
    else:
        A = torch_gen.dense_planted_device(m, n, k, sigma, SEED, dev)
    W0h, Ht0h = synth.init_factors(m, n, k, seed=SEED)
    W0 = torch.from_numpy(W0h).to(dev)
    Ht0 = torch.from_numpy(Ht0h).to(dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen

    learned = args.start == "learned"
    h = nmf.nmf_init(A, W0, Ht0, precision=args.precision,
                     start="cold" if learned else args.start,
                     max_bpp_rounds=args.max_rounds, objective_every=True,
                     shape=(m, n) if sparse else None, solver=args.solver,
                     fused_products=not args.no_fused_products)
    net = None
    if learned:
        # Learned starting partitions: the proposal network trains on every
        # warm-up half-step's (features, final passive sets), then proposes
        # the starting partition of every timed solve.
        net = nmf.nmf_mlp_create(k, MLP_HIDDEN, torch.from_numpy(synth.mlp_init(k, MLP_HIDDEN,
                                                                               seed=SEED)).to(dev))
        h.nmf_set_proposal(net, "train", epochs=1, batch=8192, lr=1e-3)
    if args.pgrad:
        h.nmf_set_pgrad(True)   # record the stopping measure of every iterate
    h.nmf_iterate(args.warmup)
    if learned:
        h.nmf_set_proposal(net, "use")
    warm_status = h.nmf_sync()
    # The FP32 SIMT forms (plain FP32 products, sparse BPP) are quoted against
    # the measured FP32 FMA rate.
    probe = fp32_peak_probe(nmf, local_rank) if (sparse or args.precision == "fp32") else None
    st0 = h.nmf_get_stats()
    h.nmf_set_timing(True)

    def barrier():
        if world > 1:
            dist.barrier()

    sampler = ClockSampler(local_rank)
    torch.cuda.synchronize()
    barrier()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx is not None:
        nvtx.range_push("timed")    # lets ncu select exactly the timed launches
    h.nmf_iterate(args.steps)
    if nvtx is not None:
        nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    status = h.nmf_sync()
    st1 = h.nmf_get_stats()
    f_hist = h.nmf_objective_history()
    pg_ratio = None
    if args.pgrad:
        pg = h.nmf_pgrad_history()
        pg_ratio = pg[-1] / pg[0] if pg and pg[0] > 0 else None
    ms = max_over_ranks(ms, world, dev)
    value = world * args.steps / (ms / 1000.0)

    # Roofline of the dominant kernel (the two m*n*k products), from the
    # handle's per-phase CUDA events over the timed region.
    launches_mm = 2 * args.steps
    mm_ms = (st1["ms_mm"] - st0["ms_mm"]) / launches_mm
    nls_ms = (st1["ms_nls"] - st0["ms_nls"]) / launches_mm
    gram_ms = (st1["ms_gram"] - st0["ms_gram"]) / launches_mm
    obj_ms = (st1["ms_objective"] - st0["ms_objective"]) / args.steps
    prop_ms = (st1["ms_proposal"] - st0["ms_proposal"]) / launches_mm
    pk, pk_kind = peaks()
    bytes_mm = 4.0 * m * n + 4.0 * (m + n) * k     # A once + factor in + product out
    flops_mm = 2.0 * m * n * k
    if sparse:
        # Compulsory bytes of one SpMM, averaged over A H^T and A^T W: CSR
        # (4-byte index + 4-byte value per nonzero, 8-byte row pointers), the
        # dense operand read once, the product written once.
        bytes_mm = 8.0 * nnz + 4.0 * (m + n) + 4.0 * (m + n) * k
        flops_mm = 2.0 * nnz * k
        if mm_ms > 0:
            achieved = bytes_mm / (mm_ms / 1000.0) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "kernel": "spmm_kernel",
                    "peak_source": f"{pk_kind} hbm_gbs", "bytes": "compulsory",
                    "achieved_with_gathers_gbs":
                        (bytes_mm + 4.0 * nnz * k) / (mm_ms / 1000.0) / 1e9}
        else:   # the products are formed inside the BPP solves
            roof = {"bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": None, "kernel": "spmm_kernel",
                    "note": "no separate product pass: each right-hand side is gathered "
                            "inside the FP32 BPP solves"}
    elif args.precision == "fp32":
        # The products' pass: A H^T with the objective's W H (2mnk more) and
        # A^T W, averaged over the two launches of an iteration.
        fp32_peak, peak_src = alu_peak(probe, clocks)
        flops_f32 = 1.5 * flops_mm
        achieved = flops_f32 / (mm_ms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "kernel": "mm_f32_kernel, mm_f32_t_kernel",
                "peak_source": peak_src, "flops": "2mnk per product + 2mnk for W H",
                "achieved_gbs": bytes_mm / (mm_ms / 1000.0) / 1e9}
    else:
        achieved = bytes_mm / (mm_ms / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "kernel": "mm_tc_kernel",
                "peak_source": f"{pk_kind} hbm_gbs",
                "achieved_tflops": flops_mm / (mm_ms / 1000.0) / 1e12}
    roof["traffic"] = NCU_TRAFFIC.get((roof["kernel"], args.workload, args.precision))
    roof_products = None
    if sparse and args.solver == "bpp":
        # On the sparse workload the FP32 BPP solves, not the products, hold
        # most of the step: they get the "roofline" entry. Work of the method
        # per solve with final passive set size f: 2f^2 + 2f(k - f) flops for
        # the solution and y = Gx - g, plus f^3/3 for the factor; solves per
        # right-hand side = 1 + exchange rounds (every round re-solves; the
        # final f stands in for the intermediate ones). Bytes: b in, x out,
        # passive set in and out.
        pW, pH = h.nmf_get_passive()
        fsum = 0.0
        for P_ in (pW, pH):
            fv = nmf.passive_to_bool(P_, k).double().sum(dim=1)
            fsum += float((2 * fv * fv + 2 * fv * (k - fv) + fv ** 3 / 3).sum().item())
        rounds_per = (st1["bpp_rounds"] - st0["bpp_rounds"]) / max(st1["bpp_rhs"] - st0["bpp_rhs"], 1)
        flops_bpp = fsum * (1.0 + rounds_per)
        bytes_bpp = (m + n) * (8.0 * k + 16.0)
        t_bpp = 2 * nls_ms / 1000.0                   # both half-steps of one iteration
        fp32_peak, peak_src = alu_peak(probe, clocks)
        roof_products = roof
        roof = {"bound": "alu", "achieved": flops_bpp / t_bpp / 1e12, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": flops_bpp / t_bpp / 1e12 / fp32_peak,
                "kernel": "bpp_solve32_kernel",
                "peak_source": peak_src,
                "flops_per_iteration": flops_bpp,
                "achieved_gbs": bytes_bpp / t_bpp / 1e9,
                "hbm_frac": bytes_bpp / t_bpp / 1e9 / pk["hbm_gbs"],
                "note": "small dependent systems (mean |F| below k/2): bound by instruction "
                        "issue, not by the FP32 pipes or HBM",
                "traffic": None}

    # End to end through the public API from pinned host memory: upload A and the
    # starting point, nmf_init, K iterations, download W, H^T and the objective.
    e2e = None
    if not args.no_e2e:
        if sparse:
            A_host = tuple(torch.from_numpy(x).pin_memory() for x in csr_host)
        else:
            A_host = torch.empty((m, n), dtype=torch.float32, pin_memory=True)
            A_host.copy_(A)
        W0_host = torch.from_numpy(W0h).pin_memory()
        Ht0_host = torch.from_numpy(Ht0h).pin_memory()
        W_out = torch.empty((m, k), dtype=torch.float32, pin_memory=True)
        Ht_out = torch.empty((n, k), dtype=torch.float32, pin_memory=True)
        h.nmf_destroy()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        if sparse:
            for dst, src in zip(A, A_host):
                dst.copy_(src, non_blocking=True)
        else:
            A.copy_(A_host, non_blocking=True)
        W0.copy_(W0_host, non_blocking=True)
        Ht0.copy_(Ht0_host, non_blocking=True)
        h2 = nmf.nmf_init(A, W0, Ht0, precision=args.precision,
                          start="cold" if learned else args.start,
                          max_bpp_rounds=args.max_rounds, objective_every=True,
                          shape=(m, n) if sparse else None, solver=args.solver,
                          fused_products=not args.no_fused_products)
        if learned:
            h2.nmf_set_proposal(net, "use")    # the network trained above
        h2.nmf_iterate(args.steps)
        Wd, Htd = h2.nmf_get_factors()
        W_out.copy_(Wd, non_blocking=True)
        Ht_out.copy_(Htd, non_blocking=True)
        f_e2e = h2.nmf_objective_history()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        barrier()
        dt = max_over_ranks(dt, world, dev)
        h2.nmf_destroy()
        h2d = (sum(x.numel() * x.element_size() for x in A_host) if sparse else 4 * m * n) + \
            4 * (m + n) * k
        d2h = 4 * (m + n) * k + 8 * len(f_e2e)
        e2e = {"value": world * args.steps / dt, "unit": "iter/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "upload A + start, nmf_init, K iterations, download W, H^T, objective"}
    else:
        h.nmf_destroy()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if sparse:   # ~7 s per crop iteration on 16 cores: keep the sample near 20 s
            v, sample, cores, _ = oracle_sample_sparse(m, n, k, SPARSE_DRAWS[args.workload],
                                                       min(args.cpu_steps, 3),
                                                       args.start == "warm", csr_host,
                                                       args.solver)
        else:
            v, sample, cores, _ = oracle_sample(m, n, k, sigma, args.cpu_steps,
                                                args.start == "warm", args.solver)
        cpu = {"value": v, "unit": "iter/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        rounds = st1["bpp_rounds"] - st0["bpp_rounds"]
        rhs = st1["bpp_rhs"] - st0["bpp_rhs"]
        line = {"metric": metric_name(args.solver), "value": value, "unit": "iter/s",
                "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else "bf16x3/f32",
                "data": "synthetic",
                "config": {"workload": desc, "precision": args.precision, "start": args.start,
                           "solver": args.solver,
                           **({"fused_products": not args.no_fused_products} if sparse else {}),
                           "seed": SEED,
                           "l2": "small input (L2-resident)" if args.workload == "dense-small"
                           else (f"CSR {8 * nnz / 1e9:.2f} GB + factors {8 * (m + n) * k / 1e9:.2f} GB, "
                                 "larger than L2" if sparse
                                 else f"inputs larger than L2 (A = {4 * m * n / 1e9:.1f} GB)"),
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"],
                **({"roofline_products": roof_products} if roof_products else {}),
                # "gram_prep_side": Gram + BPP preparation on the handle's side
                # stream, fork to finish; it overlaps the products (so it also
                # counts time queued behind them) and is not part of the step sum.
                "phase_ms_per_launch": {"mm": mm_ms, "nls": nls_ms, "gram_prep_side": gram_ms,
                                        "objective": obj_ms, "proposal": prop_ms},
                "bpp": {"rounds_per_rhs": rounds / max(rhs, 1),
                        "fp64_solves": st1["bpp_fp64_solves"] - st0["bpp_fp64_solves"],
                        "fp64_halfsteps": st1["bpp_fp64_halfsteps"] - st0["bpp_fp64_halfsteps"],
                        "status": nmf.nmf_status_str(status),
                        "warmup_status": nmf.nmf_status_str(warm_status)},
                "objective_last": f_hist[-1] if f_hist else None,
                "pgrad_ratio_last": pg_ratio,
                "setup_s": {"generate": t_gen}}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16x3"], default="bf16x3")
    ap.add_argument("--start", choices=["cold", "warm", "learned"], default="warm",
                    help="BPP starting partitions: empty, the previous iteration's, or the "
                         "proposal network's (trained during the warm-up iterations)")
    ap.add_argument("--workload", choices=sorted(list(WORKLOADS) + list(STRESS_WORKLOADS)),
                    default="dense-large")
    ap.add_argument("--pgrad", action="store_true",
                    help="record the projected-gradient stopping measure in every iteration")
    ap.add_argument("--solver", choices=["bpp", "mu", "hals"], default="bpp",
                    help="local update: BPP (Sec. 4.2), MU (Eq. 5) or HALS (Eq. 6)")
    ap.add_argument("--max-rounds", type=int, default=100)
    ap.add_argument("--no-fused-products", action="store_true",
                    help="sparse BPP: run the SpMM pass before the solves instead of gathering "
                         "each right-hand side inside them (same results)")
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.solver != "bpp" and args.start == "learned":
        ap.error("--start learned proposes BPP partitions; it needs --solver bpp")
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload in STRESS_WORKLOADS:
        run_stress(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
