#!/usr/bin/env python3
"""Benchmark of the RBGS QR hot path (Balabanov & Grigori, arXiv 2111.14641).

One step = one full RBGS QR factorization (Alg. 2: every column block sketched,
projected, orthonormalised and re-sketched) of a synthetic matrix already
resident in HBM, through the C ABI of librbgs.

Default workload (mixed precision): n = 1,000,000 rows, m = 1000 columns,
block size m_p = 50, SRHT sketch k = 2000, W in FP32 with singular values
log-spaced from 1 to 1e-6 (W = U diag(sigma) V^T with U random signs scaled by
a power of two and V Sylvester-Hadamard, a product that is exact in FP64, so
the CPU oracle can be given the very matrix the GPU factors).
W and Q are stored in FP32; the tall products run on the tcgen05 tensor cores
with FP16 hi/lo split operands (three products, about 2^-22 relative; the
basis is kept pre-split in the workspace), the sketches in FP32; the
sketch-space steps (least squares, block Cholesky QR, R) run in FP64
(--fine 0 runs them in FP32; the line reports the other choice as a variant).  Step 2 takes one Richardson iteration per pass; every block
after the first takes a second projection pass (--reorth 1).

`value` is GFLOP/s of the method's own work per factorization (the cost model
of Sec. 3: step 3's products, the triangular solve and the sketches of W and
Q); the Richardson products and the second pass are reported apart under
`reorth_overhead`.  `roofline` is the dominant kernel (the tall update)
against the measured HBM copy bandwidth; `step_roofline` is the whole step's
minimum HBM bytes at that bandwidth over the measured step time.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (n, m, mb, sketch, k, cond, seed_W, seed_theta, description)
    "c2": dict(n=1_000_000, m=1000, mb=50, sketch="srht", k=2000, cond=1e6, seed_w=7, seed_theta=1,
               recipe="hadamard",
               desc="RBGS QR n=1e6 m=1000 mb=50 SRHT k=2000, W fp32 cond 1e6 (log-spaced sigma; "
                    "W = 2^-15 (signs x diag(sigma) x Hadamard), exact on CPU and GPU)"),
    "c1": dict(n=10_000, m=100, mb=10, sketch="gauss", k=200, cond=1e8, seed_w=7, seed_theta=1,
               desc="RBGS QR n=1e4 m=100 mb=10 Gaussian k=200, W fp64 cond 1e8"),
}
CPU_SAMPLE_ROWS = 16384
CPU_SAMPLE_COLS = 500
METRIC = "RBGS QR GFLOP/s & roofline frac, mixed vs FP64 on GB300 at stated orthogonality"
SKETCH_SPACE = {0: "fp32", 1: "fp64", 2: "fp64 storage, double-fp32 products"}
SKETCH_SPACE_KEY = {0: "fp32", 1: "fp64", 2: "fp64_dfloat"}
FINE_MIXED = 2  # the sketch-space mode of the mixed runs beside the headline (C3, C4, C5); set from --fine
TALL_KERNEL = {"f16x3": "tall_h3_kernel", "tf32x3": "tall_tc_kernel"}
TALL_SOURCE = {"f16x3": "tall_h3.cu", "tf32x3": "tall_tc.cu"}


def sketch_flops_per_col(n, k, sketch):
    """SRHT: n' log2 n' additions per column (n' = 2^ceil(log2 n)); a dense
    Gaussian or Rademacher sketch: 2 k n per column."""
    npad = 1 << max(0, math.ceil(math.log2(n)))
    return npad * math.log2(npad) if sketch == "srht" else 2.0 * k * n


def algorithmic_flops(n, m, mb, k, sketch):
    """Work the method must do in one factorization (the cost model of the
    discussion after Alg. 2, Sec. 3): step 3's tall products,
    sum_i 2 n (i-1) m_p m_p = n m (m - m_p), the triangular solve with R_ii,
    n m m_p, and the sketches of W and Q (step 1 and step 5), 2 m columns.
    The sketch-space steps (least squares and block QR, O(k m^2)) are not
    counted, nor anything a second pass repeats."""
    return float(n) * m * (m - mb) + float(n) * m * mb + 2.0 * m * sketch_flops_per_col(n, k, sketch)


def overhead_flops(n, m, mb, k, sketch, ls_iters, reorth_blocks):
    """Work done beyond the method's count: the Richardson products of step 2
    (2 l k m (m - m_p)), and for each block that takes the second projection
    pass (an extension for the orthogonality targets) its projection,
    triangular update, sketch and least squares once more."""
    psk = sketch_flops_per_col(n, k, sketch)
    f = 2.0 * ls_iters * k * m * (m - mb)
    if reorth_blocks:
        c_avg = (m - mb) / 2.0 + mb / 2.0  # mean c over the blocks that take it
        f += reorth_blocks * (2.0 * n * c_avg * mb + n * mb * mb + mb * psk + 4.0 * ls_iters * k * c_avg * mb)
    return f


def algorithmic_bytes(n, m, mb, elem):
    """Minimum HBM traffic of one factorization: step 3 reads the basis
    Q_{1:i-1} for every block (elem n m_p p (p - 1) / 2 bytes), and W is read
    and Q written once (2 n m elem)."""
    p = m // mb
    return elem * (float(n) * mb * p * (p - 1) / 2.0 + 2.0 * n * m)


def two_pass_bytes(n, m, mb, elem, reorth_blocks):
    """The same with the second projection pass on reorth_blocks blocks: each
    reads the basis and its own block again and writes it (the tall kernel's
    bytes, 4 n (c + 2 m_p) per launch in FP32)."""
    p = m // mb
    c_avg = (m - mb) / 2.0 + mb / 2.0
    return algorithmic_bytes(n, m, mb, elem) + reorth_blocks * elem * float(n) * (c_avg + 2 * mb) * (
        1.0 if p > 1 else 0.0)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def aggregate_over_ranks(ms_local: float, flops: float, world: int, device):
    """Replicas only: every rank factors its own copy of the workload.  The
    step time is the slowest rank's (max over ranks) and the whole-job
    throughput counts every rank's work: world * flops / max time (GFLOP/s)."""
    import torch

    ms_all = ms_local
    if world > 1:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_all = float(t.item())
    return ms_all, world * flops / (ms_all * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_w(cfg, device, dtype):
    import torch
    import synth

    if cfg.get("recipe") == "hadamard":
        W = synth.hadamard_svd_matrix_torch(cfg["n"], cfg["m"], cfg["cond"], cfg["seed_w"], device=device,
                                            dtype=dtype)
    else:
        W = synth.svd_matrix_torch(cfg["n"], cfg["m"], cfg["cond"], cfg["seed_w"], device=device, dtype=dtype)
    torch.cuda.synchronize()
    return W


def quality(rb, W, Q, R, cfg):
    """||W - QR||_F/||W||_F (FP64 products on the device), and sketched
    orthogonality ||I - (Theta Q)^T (Theta Q)|| in the Frobenius and 2-norm
    with Theta applied to Q in FP64 by librbgs, cond(Q) from the FP64 Gram."""
    import torch

    n, m = W.shape
    num, den = 0.0, 0.0
    R64 = R.double()
    chunk = 1 << 17
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        Wc = W[r0:r1].double()
        E = Wc - Q[r0:r1].double() @ R64
        num += float((E * E).sum())
        den += float((Wc * Wc).sum())
    Q64 = rb.colmajor(Q.double())
    S = rb.sketch_apply(Q64, cfg["sketch"], cfg["k"], cfg["seed_theta"], prec="fp64")
    import numpy as np

    # m x m spectral quantities on the host (numpy LAPACK)
    Ei = np.eye(m) - (S.t() @ S).cpu().numpy()
    d_fro = float(np.linalg.norm(Ei))
    d_two = float(np.linalg.norm(Ei, 2))
    ev = np.linalg.eigvalsh((Q64.t() @ Q64).cpu().numpy())
    condq = float(np.sqrt(ev.max() / ev.min()))
    del Q64, S
    return {"rel_factorization_error": math.sqrt(num / den), "sketched_orthogonality_fro": d_fro,
            "sketched_orthogonality_2": d_two, "cond_Q": condq}


def tall_traffic(prec, bytes_per_launch):
    """DRAM bytes per tall-update launch: the ratio of ncu's measured
    dram__bytes_read + dram__bytes_write to the algorithmic bytes of one
    captured launch (profiles/tall_tc_kernel_*.md), scaled to the average
    launch here; None unless that capture was taken from the kernel source
    as it is now."""
    import glob
    import hashlib

    if prec not in TALL_KERNEL:
        return None
    kernel = TALL_KERNEL[prec]
    src = os.path.join(ROOT, "paper_2111_14641_gb300", "csrc", TALL_SOURCE[prec])
    try:
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_*.md"))):
        fields = {}
        with open(path) as f:
            for ln in f:
                if ":" in ln and not ln.startswith(("|", " ", "#", "-")):
                    key, _, val = ln.partition(":")
                    fields[key.strip()] = val.strip()
        ratio = fields.get("traffic_over_algorithmic")
        prefix = fields.get("kernel_source_sha256_prefix")
        if ratio and prefix and digest.startswith(prefix):
            return float(ratio) * bytes_per_launch
    return None


def cpu_baseline(cfg, ls_iters, reorth, one_core=False):
    """The CPU oracle (plain FP64 C, all host cores) on a bounded sample of the
    workload: a CPU_SAMPLE_ROWS x CPU_SAMPLE_COLS matrix of the same recipe
    (same m_p, k, sketch and conditioning), i.e. the first blocks of a
    shorter factorization."""
    import numpy as np

    import oracle
    import synth

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    ns = min(cfg["n"], CPU_SAMPLE_ROWS)
    ms = min(cfg["m"], CPU_SAMPLE_COLS)
    if cfg.get("recipe") == "hadamard":
        W = synth.hadamard_svd_matrix(ns, ms, cfg["cond"], cfg["seed_w"]).astype(np.float64)
    else:
        W = synth.svd_matrix(ns, ms, cfg["cond"], cfg["seed_w"])
    t0 = time.perf_counter()
    out = oracle.rbgs(W, cfg["mb"], cfg["sketch"], cfg["k"], cfg["seed_theta"], variant=5, ls="richardson",
                      ls_iters=ls_iters, reorth=bool(reorth), ls_iters_first=1)
    dt = time.perf_counter() - t0
    flops = algorithmic_flops(ns, ms, cfg["mb"], cfg["k"], cfg["sketch"])
    res = {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
           "sample": f"oracle RBGS (Alg. 2, Alg. 5, Richardson l={ls_iters}, reorth={int(bool(reorth))}) on "
                     f"n={ns} rows x m={ms} (m_p={cfg['mb']}, {cfg['sketch']} k={cfg['k']}, same recipe), "
                     f"{dt:.1f} s", "seconds": dt, "delta": float(out["delta"]), "cpu": cpu_model()}
    if one_core:
        # the same sample's first quarter of the rows on one thread
        n1 = max(cfg["mb"], ns // 4)
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.rbgs(np.asfortranarray(W[:n1]), cfg["mb"], cfg["sketch"], min(cfg["k"], n1), cfg["seed_theta"],
                    variant=5, ls="richardson", ls_iters=ls_iters, reorth=bool(reorth), ls_iters_first=1)
        d1 = time.perf_counter() - t0
        oracle.set_threads(cores)
        res["one_core"] = {"value": algorithmic_flops(n1, ms, cfg["mb"], min(cfg["k"], n1), cfg["sketch"]) / d1 / 1e9,
                           "unit": "GFLOP/s", "sample": f"n={n1} rows x m={ms}, 1 thread, {d1:.1f} s"}
    del W
    return res


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo; on Arm the part is named by
    the implementer and part fields, given as they are)."""
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
    except OSError:
        return "unknown"
    for ln in txt.splitlines():
        if ln.lower().startswith(("model name", "cpu model")):
            return ln.split(":", 1)[1].strip()
    impl = [ln.split(":", 1)[1].strip() for ln in txt.splitlines() if ln.startswith("CPU implementer")]
    part = [ln.split(":", 1)[1].strip() for ln in txt.splitlines() if ln.startswith("CPU part")]
    if impl and part:
        name = " (Neoverse V2)" if impl[0].lower() == "0x41" and part[0].lower() == "0xd4f" else ""
        return f"Arm implementer {impl[0]} part {part[0]}{name}"
    return "unknown"


def run_reference(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    ls_iters, reorth = args.ls_iters, args.reorth
    for _ in range(args.warmup):
        pass  # the oracle has no caches to warm; warm-up steps would only repeat the timed work
    vals = []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(cfg, ls_iters, reorth)
        vals.append(cb["seconds"])
    ms = 1e3 * sum(vals) / len(vals)
    value = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"] + f" (oracle sample: {CPU_SAMPLE_ROWS} x {CPU_SAMPLE_COLS})",
                       "sample_rows": CPU_SAMPLE_ROWS, "sample_cols": CPU_SAMPLE_COLS},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args, cfg):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import paper_2111_14641_gb300 as rb

    rb.load()
    prec = args.prec
    dtype = torch.float64 if prec == "fp64" else torch.float32
    n, m, mb, k = cfg["n"], cfg["m"], cfg["mb"], cfg["k"]
    W = make_w(cfg, dev, dtype)
    Q = torch.empty((m, n), dtype=dtype, device=dev).t()
    R = torch.empty((m, m), dtype=torch.float64, device=dev).t()

    def step(timing=False):
        return rb.rbgs_qr(W, mb, cfg["sketch"], k, cfg["seed_theta"], prec=prec, ls_iters=args.ls_iters,
                          reorth=args.reorth, reorth_tol=args.reorth_tol, Q=Q, R=R, sync=True, timing=timing,
                          fine=args.fine)[2]

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = rb.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tall_ms = tall_bytes = 0.0
    tall_launches = passes2 = 0
    for _ in range(args.steps):
        st = step(timing=True)
        tall_ms += st.tall_ms
        tall_bytes += st.tall_bytes
        tall_launches += st.tall_launches
        passes2 = st.passes2
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = rb.launch_count() - l0
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    flops = algorithmic_flops(n, m, mb, k, cfg["sketch"])
    ms_all, value = aggregate_over_ranks(ms, flops, world, dev)
    extra = overhead_flops(n, m, mb, k, cfg["sketch"], args.ls_iters, passes2)

    # ---- roofline of the dominant kernel (tall update), from its own CUDA events
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured"
    if peak is None:
        peak, peak_src = 6800.0, "fallback"
    achieved = tall_bytes / (tall_ms * 1e-3) / 1e9 if tall_ms > 0 else None
    traffic = tall_traffic(prec, tall_bytes / max(tall_launches, 1))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "kernel": TALL_KERNEL.get(prec, "tall_simt_kernel"),
                "peak_source": peak_src, "launch_ms_avg": tall_ms / max(tall_launches, 1),
                "bytes_per_launch_avg": tall_bytes / max(tall_launches, 1)}

    # ---- the whole step against the HBM roofline: the minimum bytes of one
    # factorization (the basis read once per block, W read and Q written once)
    # at the measured copy bandwidth, over the measured step time; and the
    # same with the second pass's bytes
    elem = 8 if prec == "fp64" else 4
    b1 = algorithmic_bytes(n, m, mb, elem)
    b2 = two_pass_bytes(n, m, mb, elem, passes2)
    step_roofline = {"bound": "hbm", "bytes_single_pass": b1, "bytes_two_pass": b2, "peak_gbs": peak,
                     "roofline_ms_single_pass": b1 / (peak * 1e9) * 1e3,
                     "roofline_ms_two_pass": b2 / (peak * 1e9) * 1e3, "ms_per_step": ms_all,
                     "frac": b1 / (peak * 1e9) * 1e3 / ms_all, "frac_two_pass": b2 / (peak * 1e9) * 1e3 / ms_all,
                     "peak_source": peak_src}

    # ---- end to end: the host-buffer entry point (rbgs_qr_host) on pinned host
    # W, Q, R; its copies of W up and of Q, R down are inside the timed region
    # (they overlap the factorization block by block)
    e2e = None
    if not args.no_e2e:
        W_h = torch.empty((m, n), dtype=dtype, pin_memory=True).t()
        W_h.copy_(W)
        Q_h = torch.empty((m, n), dtype=dtype, pin_memory=True).t()
        R_h = torch.empty((m, m), dtype=torch.float64, pin_memory=True).t()
        torch.cuda.synchronize()

        def step_host():
            return rb.rbgs_qr_host(W_h, mb, cfg["sketch"], k, cfg["seed_theta"], prec=prec, ls_iters=args.ls_iters,
                                   reorth=args.reorth, reorth_tol=args.reorth_tol, Q=Q_h, R=R_h, fine=args.fine)

        def step_host_timed():
            return rb.rbgs_qr_host(W_h, mb, cfg["sketch"], k, cfg["seed_theta"], prec=prec, ls_iters=args.ls_iters,
                                   reorth=args.reorth, reorth_tol=args.reorth_tol, Q=Q_h, R=R_h, fine=args.fine,
                                   timing=True)

        # the plain copy rates of the same pinned buffers, alone and both ways at once
        rates = copy_rates(W_h, Q_h, W, Q)
        step_host()  # allocates the library's device copies
        torch.cuda.synchronize()
        # three warm-up calls in all; a longer warm-up (1.5 s of calls) was tried and did
        # not remove the occasional stalled copies, which come and go at random
        warm_e2e = 1
        while warm_e2e < 3:
            step_host()
            warm_e2e += 1
        torch.cuda.synchronize()
        steps_e2e = max(1, min(args.steps, 10))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tls = []
        a.record()
        for _ in range(steps_e2e):
            tls.append(step_host_timed()[2])  # each call's copy / compute timeline from the library's events
        b.record()
        torch.cuda.synchronize()
        ms_e2e = a.elapsed_time(b) / steps_e2e
        diff_q = float((Q_h.double() - Q.cpu().double()).abs().max())
        h2d = W_h.element_size() * n * m
        d2h = Q_h.element_size() * n * m + 8 * m * m
        e2e = {"value": world * flops / (ms_e2e * 1e-3) / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e, "api": "rbgs_qr_host (pinned host buffers)",
               "max_abs_diff_Q_vs_device_path": diff_q,
               "median_call_ms": statistics.median(t.host_total_ms for t in tls), "warmup_calls": warm_e2e,
               "timeline_ms": {"W_on_device": [t.host_up_ms for t in tls],
                               "Q_final_on_device": [t.host_compute_ms for t in tls],
                               "Q_R_on_host": [t.host_total_ms for t in tls]},
               "copy_rates_gbs": rates}
        del W_h, Q_h, R_h

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"f16x3": "f32 (3x FP16-split tensor products)",
                                           "tf32x3": "f32 (3xTF32 tensor products)", "fp32": "f32",
                                           "fp64": "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": cfg["desc"], "n": n, "m": m, "mb": mb, "sketch": cfg["sketch"], "k": k,
                       "prec": prec, "sketch_space": SKETCH_SPACE[args.fine if prec != "fp64" else 1],
                       "ls_iters": args.ls_iters, "reorth": args.reorth,
                       "reorth_tol": args.reorth_tol, "passes2": passes2,
                       "l2": "inputs larger than L2 (W and Q are GBs; no flush needed)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "step_roofline": step_roofline, "clocks": clocks, "gpu_launches": launches,
            "e2e": e2e, "algorithmic_gflop_per_step": flops / 1e9,
            "reorth_overhead": {"gflop_per_step": extra / 1e9, "passes2": passes2,
                                "value_counting_it": world * (flops + extra) / (ms_all * 1e-3) / 1e9,
                                "note": "step-2 Richardson products, and the second projection pass (projection, "
                                        "triangular update, sketch, least squares) on passes2 blocks: work done to "
                                        "meet the orthogonality target, not counted in value"}}

    if rank == 0 and not args.no_quality:
        line["quality"] = quality(rb, W if args.no_e2e else _refill(W, cfg, dev, dtype), Q, R, cfg)

    if rank == 0 and world == 1 and not args.no_variant and prec != "fp64":
        for other in (0, 1, 2):
            if other != args.fine:
                line[f"variant_sketch_space_{SKETCH_SPACE_KEY[other]}"] = sketch_space_variant(
                    rb, W, Q, R, cfg, args, prec, other, flops)

    if rank == 0 and world == 1 and not args.no_fp64_compare and prec != "fp64":
        line["fp64_path"] = fp64_compare(rb, cfg, args, dev)

    if rank == 0 and world == 1 and not args.no_krylov:
        line["krylov_c4"] = krylov_c4(rb, dev, prec if prec != "fp64" else "f16x3")
    if rank == 0 and world == 1 and not args.no_batched:
        line["batched_c3"] = batched_c3(rb, dev, prec if prec != "fp64" else "f16x3")
    if rank == 0 and world == 1 and not args.no_learned:
        line["learned_c5"] = learned_c5(rb, dev, C5_FULL if args.c5_full else C5_SHORT if args.c5_short else C5_DEFAULT)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(cfg, args.ls_iters, args.reorth, one_core=True)
        line["cpu_baseline"] = {k2: cb[k2] for k2 in ("value", "unit", "cores", "kind", "sample", "cpu", "one_core")}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def sketch_space_variant(rb, W, Q, R, cfg, args, prec, fine, flops_ref):
    """The same factorization with the other precision of the sketch-space
    steps (FP32 or FP64), 3 warm-up and up to 5 timed steps, with its quality."""
    import torch

    def step():
        return rb.rbgs_qr(W, cfg["mb"], cfg["sketch"], cfg["k"], cfg["seed_theta"], prec=prec,
                          ls_iters=args.ls_iters, reorth=args.reorth, reorth_tol=args.reorth_tol, Q=Q, R=R,
                          sync=True, fine=int(fine))[2]

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        st = step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    out = {"ms_per_step": ms, "steps": steps, "sketch_space": SKETCH_SPACE[fine],
           "value": algorithmic_flops(cfg["n"], cfg["m"], cfg["mb"], cfg["k"], cfg["sketch"]) / (ms * 1e-3) / 1e9,
           "unit": "GFLOP/s", "passes2": st.passes2}
    if not args.no_quality:
        out["quality"] = quality(rb, W, Q, R, cfg)
    return out


def stencil_eigs_smallest(nx, ny, bx, by, count):
    """The count smallest eigenvalues of the 5-point convection-diffusion
    operator in closed form: with h = 1/(nx+1) (= 1/(ny+1)) and cell Peclet
    numbers P = b h / 2 < 1, lambda_jl = (2/h^2) [2 - sqrt(1 - Px^2) cos(j pi h)
    - sqrt(1 - Py^2) cos(l pi h)] (real: the operator is similar to a
    symmetric one by a diagonal scaling)."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    px, py = bx * hx / 2.0, by * hy / 2.0
    jm = int(math.ceil(math.sqrt(count))) + 4
    lam = []
    for j in range(1, jm + 1):
        for l in range(1, jm + 1):
            lam.append(2.0 * (1.0 - math.sqrt(1 - px * px) * math.cos(j * math.pi * hx)) / hx ** 2 +
                       2.0 * (1.0 - math.sqrt(1 - py * py) * math.cos(l * math.pi * hy)) / hy ** 2)
    return sorted(lam)[:count]


def eigvec_condition_log10(nx, ny, bx, by):
    """log10 of the condition number of the diagonal scaling D that makes the
    operator symmetric (D^-1 A D), ((1+P)/(1-P))^(n/2) per direction: a bound
    for the eigenvector matrix's condition, i.e. how far rounding can move the
    eigenvalues of this non-normal operator."""
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    px, py = bx * hx / 2.0, by * hy / 2.0
    return (nx / 2.0) * math.log10((1 + px) / (1 - px)) + (ny / 2.0) * math.log10((1 + py) / (1 - py))


def ritz_smallest(rb, nx, ny, bx, by, mb, p, iters, prec, fine, dev, nev=20, tol=None, interblock=4, trsm=True):
    """Alg. 8 with which = smallest real part on the stencil operator, restarted
    one iteration at a time from the previous X (the restart block of step 4),
    stopping after `iters` iterations or when every one of the nev smallest
    values has a residual estimate below tol |mu|.  Returns the nev smallest
    Ritz values with their estimates and their errors against the closed-form
    spectrum."""
    import torch

    n = nx * ny
    op = rb.stencil_op(nx, ny, bx, by)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    B = torch.randn((mb, n), generator=g, device=dev, dtype=torch.float64).t()
    k = 4 * p * mb
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    for it in range(iters):
        vals, X, res = rb.rayleigh_ritz(op, B, p=p, n_iter=1, which="SR", sketch="srht", k=k, seed=1, prec=prec,
                                        ls_iters=1, reorth=1, fine=fine, interblock=interblock, trsm=trsm)
        B = X
        done = it + 1
        order = sorted(range(mb), key=lambda j: vals[j].real)[:nev]
        if tol is not None and all(res[j] <= tol * abs(vals[j]) for j in order):
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    exact = stencil_eigs_smallest(nx, ny, bx, by, nev)
    order = sorted(range(mb), key=lambda j: vals[j].real)[:nev]
    got = [vals[j] for j in order]
    rel = [abs(v - e) / abs(e) for v, e in zip(got, exact)]
    return {"grid": [nx, ny], "b": [bx, by], "block": mb, "blocks_per_iteration": p, "k": k, "prec": prec,
            "interblock": interblock, "trsm": trsm,
            "iterations": done, "s_per_iteration": dt / done,
            "ritz_values": [[v.real, v.imag] for v in got], "exact": exact,
            "rel_error": rel, "max_rel_error": max(rel),
            "rel_resid_estimate": [res[j] / abs(vals[j]) for j in order],
            "log10_eigvec_condition_bound": eigvec_condition_log10(nx, ny, bx, by)}


def krylov_c4(rb, dev, prec):
    """Restarted randomized block GMRES (Sec. 5.2) on the 2-D convection-
    diffusion operator: 1024 x 1024 interior points, b = (100, 50), 8 right
    sides N(0,1), 40 blocks per cycle, SRHT with k = 4 x 320.  The mixed basis
    and the FP64 path run the same number of cycles, one call per cycle
    (restarted from the previous X), so the line carries both residual
    histories.  Unpreconditioned restarted GMRES converges slowly on this
    operator: the line reports the time per cycle and the history.

    Then Alg. 8 for the 20 smallest-real-part eigenvalues (block of 24, 10
    blocks per iteration, restarted) on the same operator, with each Ritz
    value's error against the closed-form spectrum; and the same on a 64 x 64
    grid with b = (10, 5), where the eigenproblem is well conditioned enough
    for the Ritz values to converge to the closed form.  Alg. 8 runs the
    Arnoldi steps with Alg. 4 and the row-wise triangular solve: once Ritz
    vectors converge, the restart block spans a nearly invariant subspace, the
    next Krylov block is numerically rank deficient, and the explicit
    R_ii^{-1} of Alg. 5 then loses the basis."""
    import torch

    nx = ny = 1024
    n, mb, restart = nx * ny, 8, 40
    p, k = restart + 1, 4 * restart * mb
    cycles = 5
    op = rb.stencil_op(nx, ny, 100.0, 50.0)
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    B = torch.randn((mb, n), generator=g, device=dev, dtype=torch.float64).t()
    out = {"workload": "block GMRES(40 blocks), 5-point convection-diffusion 1024^2, b=(100,50), 8 RHS, SRHT k=1280",
           "n": n, "rhs": mb, "blocks_per_cycle": restart}
    for label, pr, fine in (("mixed", prec, FINE_MIXED), ("fp64", "fp64", 0)):
        rb.block_gmres(op, B, None, p=p, rtol=0.0, max_cycles=1, sketch="srht", k=k, seed=1, prec=pr, ls_iters=1,
                       reorth=1, fine=fine)  # warm-up cycle
        X = torch.zeros((mb, n), device=dev, dtype=torch.float64).t()
        torch.cuda.synchronize()
        hist = []
        t0 = time.perf_counter()
        for _ in range(cycles):
            X, cyc, rel = rb.block_gmres(op, B, X, p=p, rtol=0.0, max_cycles=1, sketch="srht", k=k, seed=1,
                                         prec=pr, ls_iters=1, reorth=1, fine=fine)
            hist.append(max(rel))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[label] = {"prec": pr, "sketch_space": SKETCH_SPACE[fine if pr != "fp64" else 1], "cycles": cycles, "s_per_cycle": dt / cycles,
                      "relres_max_history": hist, "relres_max": hist[-1]}
    out["fp64_over_mixed_time_per_cycle"] = out["fp64"]["s_per_cycle"] / out["mixed"]["s_per_cycle"]
    out["note"] = ("1e-8 is not reached without a preconditioner (the paper's GMRES experiment uses ILU(0)); "
                   f"residual after {cycles} cycles of 40 blocks reported for both paths")
    rr = {"workload": "randomized Rayleigh-Ritz (Alg. 8), 20 smallest-real-part values, block 24, 10 blocks per "
                      "iteration, SRHT k = 4 x 240, restarted"}
    def guarded(*a, **kw):
        try:
            return ritz_smallest(*a, **kw)
        except rb.RbgsError as e:  # the small eigenproblem's QR iteration did not converge
            return {"error": str(e)}

    rr["mixed"] = guarded(rb, 1024, 1024, 100.0, 50.0, 24, 11, 6, prec, FINE_MIXED, dev)
    rr["fp64"] = guarded(rb, 1024, 1024, 100.0, 50.0, 24, 11, 2, "fp64", 0, dev)
    if "error" not in rr["mixed"] and "error" not in rr["fp64"]:
        rr["fp64_over_mixed_time_per_iteration"] = rr["fp64"]["s_per_iteration"] / rr["mixed"]["s_per_iteration"]
    rr["note"] = ("at 1024^2 the eigenvector matrix of this non-normal operator has condition up to "
                  f"1e{eigvec_condition_log10(1024, 1024, 100.0, 50.0):.0f}, and the 20 smallest eigenvalues are "
                  "3.5e-6 of the spectral range apart, so restarted Ritz values approach them slowly")
    rr["converged_64x64_b10_5"] = guarded(rb, 64, 64, 10.0, 5.0, 24, 11, 60, prec, FINE_MIXED, dev, tol=1e-8)
    rr["converged_64x64_b10_5_fp64"] = guarded(rb, 64, 64, 10.0, 5.0, 24, 11, 60, "fp64", 0, dev, tol=1e-10)
    out["rayleigh_ritz"] = rr
    return out


def batched_c3(rb, dev, prec, count=32, sample=8):
    """Many independent factorizations in one call (rbgs_qr_batched): the first
    `count` problems of the 256-problem workload (n ~ U[2e4, 2e5], m in
    {64..256}, m_p in {16, 32}, Gaussian k = 2m, near-duplicate columns).

    The near-duplicates are perturbed at the FP32 rounding level, so in FP32
    storage a block that holds a column and its near-copy is numerically rank
    deficient: cond(R_ii) ~ 1/u_32.  Multiplying by the explicit inverse
    R_ii^{-1} (the fused update of Alg. 5, or Alg. 4's in-place scaling, the
    option the remark after Alg. 4 allows) then has an error of u_32
    cond(R_ii) = O(1), and both W = QR and cond(Q) are lost.  A row-wise
    triangular solve is backward stable whatever cond(R_ii), and with Alg. 4's
    explicit sketch and the second pass it keeps cond(Q) = O(1) (the regime of
    the paper's first experiment).  The mixed path therefore runs Alg. 4 with
    the triangular solve (opts.trsm); Alg. 4 and Alg. 5 with the explicit
    inverse are shown beside it, and the FP64 path both ways.

    Each configuration is timed on 8 internal streams (the mixed Alg. 4 also
    on 1, and as one captured CUDA graph replayed with a single launch);
    quality on `sample` problems: ||W - QR|| / ||W||, cond(Q),
    Delta = ||I - S^T S||_F and Delta~ = ||P - S R||_F / ||P||_F with S =
    Theta Q and P = Theta W (step 6 of Alg. 2, Theta applied in FP64).
    problems_per_s_at_quality counts the batch only when every sampled problem
    has cond(Q) <= 10 and ||W - QR|| / ||W|| <= 1e-5."""
    import torch
    import synth

    specs = synth.batch_specs(count)
    out = {"workload": f"{count} problems of the 256-problem batch: n~U[2e4,2e5], m in {{64..256}}, "
                       "m_p in {16,32}, Gaussian k=2m, every 8th column a 1e-7-perturbed duplicate",
           "problems": count}
    runs = (("mixed_alg4_trsm", prec, torch.float32, 4, (1, 8), True),
            ("mixed_alg4", prec, torch.float32, 4, (8,), False), ("mixed_alg5", prec, torch.float32, 5, (8,), False),
            ("fp64", "fp64", torch.float64, 5, (8,), False), ("fp64_alg4_trsm", "fp64", torch.float64, 4, (8,), True))
    for label, pr, dt, ib, stream_counts, trsm in runs:
        Ws = [synth.near_duplicate_matrix_torch(n, m, 11 + i, device=dev, dtype=dt) for i, (n, m, _) in enumerate(specs)]
        mbs = [mp for _, _, mp in specs]
        ks = [2 * m for _, m, _ in specs]
        seeds = [7 + i for i in range(count)]
        kw = dict(ls_iters=1, reorth=1, fine=FINE_MIXED if pr != "fp64" else 0, interblock=ib, trsm=trsm)
        res = {"prec": pr, "interblock": ib, "trsm": trsm}
        for ns in stream_counts:
            rb.rbgs_qr_batched(Ws[:2], mbs[:2], ks[:2], seeds[:2], "gauss", prec=pr, nstreams=ns, **kw)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Qs, Rs, status, _ = rb.rbgs_qr_batched(Ws, mbs, ks, seeds, "gauss", prec=pr, nstreams=ns, **kw)
            torch.cuda.synchronize()
            dts = time.perf_counter() - t0
            res[f"streams_{ns}"] = {"s": dts, "problems_per_s": count / dts,
                                    "statuses_ok": sum(1 for x in status if x == 0)}
        if label == "mixed_alg4_trsm":
            # the same batch captured once as one CUDA graph, replayed with one launch
            g = rb.BatchedQRGraph(Ws, mbs, ks, seeds, "gauss", prec=pr, nstreams=8, **kw)
            g.launch()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = 2
            for _ in range(reps):
                _, _, gst, _ = g.launch()
            torch.cuda.synchronize()
            dtg = (time.perf_counter() - t0) / reps
            res["graph_streams_8"] = {"s": dtg, "problems_per_s": count / dtg,
                                      "statuses_ok": sum(1 for x in gst if x == 0)}
            g.destroy()
            del g
        qual = []
        for i in range(min(sample, count)):
            Q, W = Qs[i].double(), Ws[i].double()
            fe = float(torch.linalg.norm(W - Q @ Rs[i]) / torch.linalg.norm(W))
            sv = torch.linalg.svdvals(Q)
            S = rb.sketch_apply(rb.colmajor(Q), "gauss", ks[i], seeds[i], prec="fp64")
            P = rb.sketch_apply(rb.colmajor(W), "gauss", ks[i], seeds[i], prec="fp64")
            m = Q.shape[1]
            delta = float(torch.linalg.norm(torch.eye(m, device=dev, dtype=torch.float64) - S.t() @ S))
            delta_t = float(torch.linalg.norm(P - S @ Rs[i]) / torch.linalg.norm(P))
            qual.append({"n": W.shape[0], "m": m, "mb": mbs[i], "rel_factorization_error": fe,
                         "cond_Q": float(sv[0] / sv[-1]), "delta": delta, "delta_tilde": delta_t,
                         "certified": delta <= 0.1 and delta_t <= 0.1})
        res["quality_sample"] = qual
        ok = all(q["cond_Q"] <= 10.0 and q["rel_factorization_error"] <= 1e-5 for q in qual)
        res["quality_holds"] = ok
        res["problems_per_s_at_quality"] = res["streams_8"]["problems_per_s"] if ok else None
        out[label] = res
        del Ws, Qs, Rs
        torch.cuda.empty_cache()
    return out


C5_FULL = dict(N=512, mb=4, widths=(16, 32, 64, 64), train_fields=200, pairs_per_field=100, steps=12000,
               test_fields=50, p=40, kfac=4, max_cycles=200, batch=16, lr=1e-3, basis="f16x3")
C5_DEFAULT = dict(C5_FULL, train_fields=24, steps=2500, test_fields=3, max_cycles=60)
# a few training steps and one short solve: the kernels at the configured sizes, for profiler captures
C5_SHORT = dict(C5_FULL, train_fields=1, pairs_per_field=8, steps=20, test_fields=1, max_cycles=2)


def learned_c5(rb, dev, cfg):
    """The learned right preconditioner on random diffusion problems
    -div(a grad u) = f, a = exp(g) with g a Gaussian random field (correlation
    0.05, variance 1) on an N x N grid, mb right-hand sides.

    Training inputs (the vectors M sees inside flexible GMRES, scaled to unit
    RMS by the library): per training field, (A) pairs_per_field columns of
    the Arnoldi basis of a plain randomized block Arnoldi run from a seeded
    N(0,1) block; (S) pairs_per_field residuals r_k = b - A x_k of plain
    randomized block GMRES (restart 20 blocks) at cycles 0, 1, 2, 4, 8, 14,
    20 and 30 of solves with b = A x*, x* smooth Gaussian random fields
    (correlation lengths 0.02 .. 0.8): the (residual, correction) pairs
    (r_k, x* - x_k) of the plain solver, whose later residuals are dominated
    by the low modes the plain solver cannot remove.  Training: Adam on the
    residual-norm loss ||B (y - B^{-1} x)|| (the correction enters through
    B^{-1} x, so it needs no solve), `steps` batches of `batch` pairs drawn
    at random, half from (A) and half from (S), all on the GPU by the
    library's forward, backward, loss and Adam kernels.
    Evaluation on unseen fields: randomized block flexible GMRES with the
    network (plain GMRES as the fallback, accept 0.9) to relative residual
    1e-8 against plain randomized block GMRES with the same restart (p
    blocks), sketch (SRHT, k = kfac p mb) and basis precision, both capped at
    max_cycles; wall times on the host clock around each synchronous solve."""
    import torch
    import synth

    N, mb, widths, p = cfg["N"], cfg["mb"], cfg["widths"], cfg["p"]
    n = N * N
    k = cfg["kfac"] * p * mb
    basis = cfg["basis"]
    out = {"workload": f"learned preconditioner: -div(exp(g) grad u) = f on {N}^2, {mb} RHS, U-Net widths "
                       f"{list(widths)}, {cfg['train_fields']} training fields, {cfg['test_fields']} unseen fields, "
                       f"block FGMRES restart {p} blocks, SRHT k={k}, basis {basis}",
           "config": {kk: (list(v) if isinstance(v, tuple) else v) for kk, v in cfg.items()}}
    stride = (N + 1) * (N + 2) + (N + 2) * (N + 1)

    def field(seed):
        a = torch.exp(synth.gaussian_random_field_torch(N, seed, device=dev)).t().contiguous()
        return rb.diffusion_faces(a)

    # ---- training inputs
    t0 = time.perf_counter()
    F, ppf = cfg["train_fields"], cfg["pairs_per_field"]
    coef = torch.empty((F, stride), dtype=torch.float64, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(17)
    xab, fab, xc, fc = [], [], [], []
    nblk = (ppf + mb - 1) // mb + 1
    kw = dict(sketch="srht", seed=1, prec=basis, ls_iters=1, reorth=1, fine=FINE_MIXED)
    bdt = torch.float64 if basis == "fp64" else torch.float32  # the Arnoldi basis's storage type
    stops = (0, 1, 2, 4, 8, 14, 20, 30)  # plain-solver cycles whose residuals are kept
    corrs = (0.02, 0.05, 0.1, 0.2, 0.4, 0.8)
    for f in range(F):
        coef[f] = field(5000 + f)
        op = rb.diffusion_op(N, N, coef[f])
        # (A) the Arnoldi basis of a plain run from an N(0,1) block
        B = torch.randn((mb, n), generator=g, device=dev, dtype=bdt).t()
        Q, _ = rb.block_arnoldi(op, B, p=nblk, k=2 * nblk * mb, **kw)
        xab.append(rb.unet_scale_inputs(Q[:, :ppf]))
        fab += [f] * ppf
        # (S) residuals along plain solves: x* smooth, b = A x*, r_k = b - A x_k
        kept = 0
        rep = 0
        while kept < ppf:
            cols = []
            for jj in range(mb):
                e = synth.gaussian_random_field_torch(N, 31000 + 100 * f + 10 * rep + jj,
                                                      corr=corrs[(rep * mb + jj + f) % len(corrs)], device=dev)
                cols.append(e[1:-1, 1:-1].t().contiguous().reshape(n))
            b = rb.colmajor(rb.op_apply(op, rb.colmajor(torch.stack(cols, 1).double())))
            X = torch.zeros((mb, n), dtype=torch.float64, device=dev).t()
            done = 0
            for stop in stops:
                if stop > done:
                    X, _, _, _ = rb.block_fgmres(op, None, None, b, X, p=20, rtol=0.0, max_cycles=stop - done, k=160,
                                                 **kw)
                    done = stop
                take = min(mb, ppf - kept)
                if take <= 0:
                    break
                R = rb.colmajor(b - rb.op_apply(op, X))
                xc.append(rb.unet_scale_inputs(R[:, :take]))
                fc += [f] * take
                kept += take
            rep += 1
    XA = torch.cat([x.t() for x in xab], 0).t()
    FA = torch.tensor(fab, dtype=torch.int32, device=dev)
    XC = torch.cat([x.t() for x in xc], 0).t()
    FC = torch.tensor(fc, dtype=torch.int32, device=dev)
    del xab, xc
    torch.cuda.synchronize()
    out["pairs"] = {"arnoldi": XA.shape[1], "solver_residuals": XC.shape[1], "s": time.perf_counter() - t0}
    # ---- training
    params = torch.from_numpy(synth.unet_flat_params(synth.unet_params_levels(widths, 21), widths)).to(dev)
    m1, v1 = torch.zeros_like(params), torch.zeros_like(params)
    grads = torch.empty_like(params)
    bs = cfg["batch"]
    nc = bs // 2
    lbuf = torch.zeros(1, dtype=torch.float64, device=dev)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(1, cfg["steps"] + 1):
        ia = torch.randint(0, XA.shape[1], (bs - nc,), device=dev, generator=g)
        ic = torch.randint(0, XC.shape[1], (nc,), device=dev, generator=g)
        xb = torch.cat([XA[:, ia].t(), XC[:, ic].t()], 0).contiguous().t()
        fb = torch.cat([FA[ia], FC[ic]]).contiguous()
        y = rb.unet_forward(widths, params, N, xb, save=True, sync=False)
        _, gy = rb.unet_residual_loss(N, coef, fb, xb, y, loss=lbuf, sync=False)
        rb.unet_backward(widths, params, N, xb, gy, grads=grads, sync=False)
        rb.adam_step(params, grads, m1, v1, step, lr=cfg["lr"], sync=False)
        if step % 500 == 0 or step == 1:
            losses.append([step, float(lbuf.item())])
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    img_per_s = cfg["steps"] * bs / train_s
    gflop_img = 3.0 * unet_forward_gflop(N, widths)
    out["training"] = {"steps": cfg["steps"], "batch": bs, "s": train_s, "images_per_s": img_per_s,
                       "tflops_fwd_bwd": img_per_s * gflop_img / 1e3, "loss_history": losses}
    del XA, XC
    torch.cuda.empty_cache()
    # ---- evaluation on unseen fields
    rows = []
    for t in range(cfg["test_fields"]):
        fcoef = field(90000 + t)
        op = rb.diffusion_op(N, N, fcoef)
        B = torch.randn((mb, n), generator=g, device=dev, dtype=torch.float64).t()
        res = {}
        for label, net in (("learned", widths), ("plain", None)):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, cyc, rel, fbk = rb.block_fgmres(op, net, params if net else None, B, None, p=p, rtol=1e-8,
                                               max_cycles=cfg["max_cycles"], accept=0.9, k=k, **kw)
            torch.cuda.synchronize()
            res[label] = {"s": time.perf_counter() - t1, "cycles": cyc, "relres_max": max(rel), "fallbacks": fbk}
        rows.append(res)
    lt = [r["learned"] for r in rows]
    pt = [r["plain"] for r in rows]
    out["fields"] = rows
    for label, rr in (("learned", lt), ("plain", pt)):
        out[label] = {"reached_1e-8": sum(1 for r in rr if r["relres_max"] <= 1e-8), "s_total": sum(r["s"] for r in rr),
                      "cycles_mean": sum(r["cycles"] for r in rr) / len(rr),
                      "relres_max_worst": max(r["relres_max"] for r in rr),
                      "relres_geomean": math.exp(sum(math.log(max(r["relres_max"], 1e-300)) for r in rr) / len(rr)),
                      "fallbacks_mean": sum(r["fallbacks"] for r in rr) / len(rr)}
    return out


def unet_forward_gflop(N, widths):
    """Multiply-add flops (2 per MAC) of one forward pass of the L-level U-Net
    on one N x N image: 18 C_in C_out per pixel per 3 x 3 convolution."""
    L = len(widths)
    f = 0.0
    for l in range(L):
        px = (N >> l) ** 2
        cin = 1 if l == 0 else widths[l - 1]
        f += px * 18.0 * (cin * widths[l] + widths[l] * widths[l])
        if l < L - 1:
            f += px * 18.0 * (widths[l + 1] + widths[l]) * widths[l]
    f += N * N * 18.0 * widths[0]
    return f / 1e9


def copy_rates(W_h, Q_h, W, Q):
    """GB/s of one plain copy of W up and of Q down between the bench's pinned
    host buffers and device tensors, alone and both at once on two streams.
    W and Q hold the same values before and after."""
    import torch

    nbytes = W_h.element_size() * W_h.numel()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def both():
        cur = torch.cuda.current_stream()
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            W.copy_(W_h, non_blocking=True)
        with torch.cuda.stream(s2):
            Q_h.copy_(Q, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    up = timed(lambda: W.copy_(W_h, non_blocking=True))
    down = timed(lambda: Q_h.copy_(Q, non_blocking=True))
    bo = timed(both)
    return {"up": nbytes / up / 1e6, "down": nbytes / down / 1e6, "both_ways_total": 2 * nbytes / bo / 1e6}


def _refill(W, cfg, dev, dtype):
    """W was overwritten by the e2e copies of itself; it holds the same values."""
    return W


def fp64_compare(rb, cfg, args, dev):
    """The plain FP64 GPU path (DFMA tall product, FP64 sketches and sketch
    space) on the same input, one warm-up and one timed step."""
    import torch

    n, m, mb, k = cfg["n"], cfg["m"], cfg["mb"], cfg["k"]
    W64 = make_w(cfg, dev, torch.float64)
    Q64 = torch.empty((m, n), dtype=torch.float64, device=dev).t()
    R64 = torch.empty((m, m), dtype=torch.float64, device=dev).t()

    def step():
        return rb.rbgs_qr(W64, mb, cfg["sketch"], k, cfg["seed_theta"], prec="fp64", ls_iters=args.ls_iters,
                          reorth=args.reorth, reorth_tol=args.reorth_tol, Q=Q64, R=R64, sync=True)[2]

    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    st = step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    flops = algorithmic_flops(n, m, mb, k, cfg["sketch"])
    q = quality(rb, W64, Q64, R64, cfg) if not args.no_quality else None
    del W64, Q64, R64
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "quality": q}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2")
    ap.add_argument("--prec", choices=["f16x3", "tf32x3", "fp32", "fp64"], default=None)
    ap.add_argument("--ls-iters", type=int, default=1)
    ap.add_argument("--reorth", type=int, default=1, choices=[0, 1, 2])
    ap.add_argument("--reorth-tol", type=float, default=1e-6)
    ap.add_argument("--fine", type=int, default=2, choices=[0, 1, 2],
                    help="mixed precision: 1 = sketch-space steps (least squares, block QR, R) in FP64; 2 = the same "
                         "with their products in double-FP32 arithmetic; 0 = in FP32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip the measurement with the other sketch-space precision")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-krylov", action="store_true", help="skip the block GMRES measurement on the stencil")
    ap.add_argument("--no-batched", action="store_true", help="skip the many-small-problems measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner measurement")
    ap.add_argument("--c5-full", action="store_true",
                    help="learned preconditioner at the configured sizes (200 training fields x 100 pairs, "
                         "50 unseen fields; tens of minutes) instead of the reduced default")
    ap.add_argument("--c5-short", action="store_true",
                    help="learned preconditioner with one training field, 20 steps and a 2-cycle solve (the "
                         "kernels at the configured sizes, for profiler captures)")
    ap.add_argument("--rows", type=int, default=None,
                    help="override n (smaller cases for profiler captures; recorded in config.workload)")
    args = ap.parse_args(argv)
    cfg = WORKLOADS[args.workload]
    if args.rows:
        cfg = dict(cfg, n=args.rows, desc=cfg["desc"] + f" [n overridden: {args.rows} rows]")
    if args.prec is None:
        args.prec = "fp64" if args.workload == "c1" else "f16x3"
    global FINE_MIXED
    FINE_MIXED = args.fine if args.fine else 2
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_ours(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
