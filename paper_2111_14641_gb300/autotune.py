"""Autotuner for batches of independent factorizations (rbgs_qr_batched).

The problems of a batch are grouped by shape class (n rounded down to a power
of two, m, m_p).  For each class the tuner times the candidate launch
configurations on up to `sample` of the class's own problems and keeps the
fastest:

* the tall-product variant for FP32 storage: F16X3 (the pre-split tcgen05
  kernel), 3xTF32 (tcgen05 with split operands) or FP32 SIMT.  All three meet
  the FP32-level accuracy of the mixed path, so the choice is a speed choice;
  FP64 problems keep the FP64 path;
* the number of internal streams the batch runs on.

The tall kernels' own tiles are fixed by the tcgen05 layout (128 rows, 64-column
chunks), so the configuration space is the kernel variant and the
concurrency.  Choices are cached per (device name, class, options) in memory
and, when a cache file is given, in a JSON file.  Every candidate is a tested
path of the library: the tuner only decides which one runs.
"""
from __future__ import annotations

import json
import os
import time

FP32_VARIANTS = ("f16x3", "tf32x3", "fp32")
STREAM_COUNTS = (1, 4, 8, 16)


def _failed(out) -> bool:
    """True when a run's per-problem statuses (the third item of what the
    batched entry point returns) hold a nonzero code: RBGS_EBREAKDOWN or
    RBGS_ETIMEOUT are reported there rather than raised."""
    try:
        statuses = out[2]
    except (TypeError, IndexError):
        return False
    return any(int(s) != 0 for s in statuses)


def shape_class(n: int, m: int, mb: int) -> tuple:
    """(2^floor(log2 n), m, m_p): problems of one class share a configuration."""
    return (1 << (max(int(n), 1).bit_length() - 1), int(m), int(mb))


class BatchTuner:
    """Times candidate (variant, streams) configurations per shape class.

    run(problem_indices, prec, nstreams) must execute those problems once with
    that configuration; timer() returns seconds (wall time around a
    synchronised run).  Both are injectable so that the selection logic can
    be exercised without a device."""

    def __init__(self, variants=FP32_VARIANTS, streams=STREAM_COUNTS, sample: int = 8, reps: int = 2,
                 cache_file: str | None = None, timer=None, device_name: str = ""):
        self.variants = tuple(variants)
        self.streams = tuple(streams)
        self.sample = int(sample)
        self.reps = int(reps)
        self.cache_file = cache_file
        self.timer = timer or time.perf_counter
        self.device_name = device_name
        self.cache: dict = {}
        self.trials: dict = {}  # key -> {(prec, nstreams): best seconds}, for inspection
        self.rejected: dict = {}  # key -> [(prec, nstreams)] whose sampled problems reported a failure
        if cache_file and os.path.exists(cache_file):
            with open(cache_file) as f:
                self.cache = json.load(f)

    def key(self, cls: tuple, fp64: bool, opts: dict) -> str:
        o = ",".join(f"{k}={opts[k]}" for k in sorted(opts))
        return f"{self.device_name}|{cls[0]}x{cls[1]}/{cls[2]}|{'fp64' if fp64 else 'fp32'}|{o}"

    def choose(self, key: str, indices: list, fp64: bool, run) -> tuple:
        """The cached configuration for key, else the fastest candidate on up
        to `sample` of the given problems (each candidate runs once to warm
        up, then `reps` timed runs; the minimum counts)."""
        if key in self.cache:
            prec, ns = self.cache[key]
            return prec, int(ns)
        probe = list(indices)[: self.sample]
        variants = ("fp64",) if fp64 else self.variants
        results = {}
        for prec in variants:
            for ns in self.streams:
                try:
                    out = run(probe, prec, ns)  # warm-up: sketch plans, kernel attributes, workspaces
                except RuntimeError:
                    # a variant the problems cannot take (the tensor-core
                    # variants need leading dimensions that are multiples of 4)
                    continue
                if _failed(out):
                    # a breakdown or a timeout on a sampled problem: a variant
                    # that stops early would otherwise time fastest
                    self.rejected.setdefault(key, []).append((prec, ns))
                    continue
                best = float("inf")
                ok = True
                for _ in range(self.reps):
                    t0 = self.timer()
                    out = run(probe, prec, ns)
                    best = min(best, self.timer() - t0)
                    ok = ok and not _failed(out)
                if not ok:
                    self.rejected.setdefault(key, []).append((prec, ns))
                    continue
                results[(prec, ns)] = best
        if not results:
            raise RuntimeError("no candidate configuration runs on these problems without a breakdown")
        prec, ns = min(results, key=lambda c: (results[c], self.variants.index(c[0]) if c[0] in self.variants else 0,
                                               c[1]))
        self.trials[key] = results
        self.cache[key] = [prec, int(ns)]
        if self.cache_file:
            tmp = self.cache_file + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_file)
        return prec, int(ns)


def rbgs_qr_batched_auto(Ws: list, mbs, ks, seeds, sketch: str = "gauss", tuner: BatchTuner | None = None,
                         ls_iters: int = 2, reorth: int = 0, fine: bool = False, interblock: int = 5,
                         batched=None, sync=None):
    """rbgs_qr_batched with the launch configuration chosen per shape class by
    `tuner`.  Returns (Qs, Rs, statuses, passes2, configs) in the order of Ws;
    configs[i] is the (variant, streams) problem i ran with.  `batched` (the
    batched entry point) and `sync` (a device synchronisation) default to the
    library's and torch's."""
    if batched is None or sync is None:
        import torch

        from .rbgs import rbgs_qr_batched

        batched = batched or rbgs_qr_batched
        sync = sync or torch.cuda.synchronize
        if tuner is None:
            tuner = BatchTuner(device_name=torch.cuda.get_device_name())
    tuner = tuner or BatchTuner()
    cnt = len(Ws)
    pick = (lambda v, i: v[i] if isinstance(v, (list, tuple)) else v)
    opts = dict(sketch=sketch, ls_iters=ls_iters, reorth=reorth, fine=int(bool(fine)), interblock=interblock)
    groups: dict = {}
    for i, W in enumerate(Ws):
        n, m = W.shape
        fp64 = str(W.dtype).endswith("float64")
        groups.setdefault((shape_class(n, m, pick(mbs, i)), fp64), []).append(i)

    def run_on(idx, prec, ns):
        out = batched([Ws[i] for i in idx], [pick(mbs, i) for i in idx], [pick(ks, i) for i in idx],
                      [pick(seeds, i) for i in idx], sketch, prec=prec, ls_iters=ls_iters, reorth=reorth,
                      fine=fine, interblock=interblock, nstreams=ns)
        sync()
        return out

    Qs, Rs, st, p2, cfg = [None] * cnt, [None] * cnt, [0] * cnt, [0] * cnt, [None] * cnt
    for (cls, fp64), idx in groups.items():
        prec, ns = tuner.choose(tuner.key(cls, fp64, opts), idx, fp64, run_on)
        q, r, s, pp = run_on(idx, prec, ns)
        for j, i in enumerate(idx):
            Qs[i], Rs[i], st[i], p2[i], cfg[i] = q[j], r[j], s[j], pp[j], (prec, ns)
    return Qs, Rs, st, p2, cfg
