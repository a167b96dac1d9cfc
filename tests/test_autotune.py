"""The batch autotuner's selection logic (no device: the batched entry point,
the timer and the synchronisation are fakes)."""
import json

import numpy as np
import pytest

from paper_2111_14641_gb300 import autotune as at


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def make_fake(clock, cost, calls, fail=()):
    """A batched entry point whose run advances the clock by cost(prec, ns, n_problems)."""

    def batched(Ws, mbs, ks, seeds, sketch, prec, ls_iters, reorth, fine, interblock, nstreams):
        if prec in fail:
            raise RuntimeError("variant refused")
        calls.append((len(Ws), prec, nstreams))
        clock.t += cost(prec, nstreams, len(Ws))
        return ([("Q", W.shape, prec) for W in Ws], [("R", W.shape[1]) for W in Ws], [0] * len(Ws),
                [W.shape[1] // mb - 1 for W, mb in zip(Ws, mbs)])

    return batched


def test_shape_class_rounds_n_down_to_a_power_of_two():
    assert at.shape_class(20000, 128, 16) == (16384, 128, 16)
    assert at.shape_class(32768, 64, 32) == (32768, 64, 32)
    assert at.shape_class(1, 1, 1) == (1, 1, 1)


def test_tuner_picks_the_fastest_candidate_and_caches_it(tmp_path):
    clock = FakeClock()
    calls = []
    cost = {("f16x3", 8): 1.0, ("tf32x3", 4): 0.5}
    fake = make_fake(clock, lambda p, ns, c: cost.get((p, ns), 2.0), calls)
    cache = str(tmp_path / "tune.json")
    tuner = at.BatchTuner(streams=(1, 4, 8), sample=3, reps=2, cache_file=cache, timer=clock, device_name="dev")
    Ws = [np.zeros((3000, 64), dtype=np.float32) for _ in range(5)]
    Qs, Rs, st, p2, cfg = at.rbgs_qr_batched_auto(Ws, 16, 128, 1, tuner=tuner, batched=fake, sync=lambda: None)
    assert cfg == [("tf32x3", 4)] * 5 and st == [0] * 5 and p2 == [3] * 5
    assert all(q[2] == "tf32x3" for q in Qs)
    # 3 variants x 3 stream counts x (1 warm-up + 2 timed) on the 3-problem sample, then the batch
    assert len(calls) == 27 + 1 and calls[-1] == (5, "tf32x3", 4)
    assert all(c[0] == 3 for c in calls[:-1])
    saved = json.load(open(cache))
    assert list(saved.values()) == [["tf32x3", 4]]
    # a second tuner reads the cache and times nothing
    calls.clear()
    tuner2 = at.BatchTuner(streams=(1, 4, 8), cache_file=cache, timer=clock, device_name="dev")
    _, _, _, _, cfg2 = at.rbgs_qr_batched_auto(Ws, 16, 128, 1, tuner=tuner2, batched=fake, sync=lambda: None)
    assert cfg2 == cfg and calls == [(5, "tf32x3", 4)]


def test_classes_are_tuned_separately_and_results_keep_the_input_order():
    clock = FakeClock()
    calls = []
    # small problems prefer SIMT FP32 on one stream, large ones F16X3 on 16 streams
    def cost(prec, ns, cnt):
        return {"fp32": 1.0, "tf32x3": 2.0, "f16x3": 3.0}[prec] / ns if small[0] else \
            {"fp32": 3.0, "tf32x3": 2.0, "f16x3": 1.0}[prec] / ns

    small = [True]
    fake_inner = make_fake(clock, cost, calls)

    def fake(Ws, *a, **kw):
        small[0] = Ws[0].shape[0] < 10000
        return fake_inner(Ws, *a, **kw)

    tuner = at.BatchTuner(streams=(1, 16), sample=2, reps=1, timer=clock)
    Ws = [np.zeros((n, 64), dtype=np.float32) for n in (3000, 50000, 3100, 60000, 2900)]
    Qs, Rs, st, p2, cfg = at.rbgs_qr_batched_auto(Ws, 16, 128, [1, 2, 3, 4, 5], tuner=tuner, batched=fake,
                                                  sync=lambda: None)
    assert cfg[0] == cfg[2] == cfg[4] == ("fp32", 16)
    assert cfg[1] == ("f16x3", 16) and cfg[3] == ("f16x3", 16)
    assert [q[1][0] for q in Qs] == [3000, 50000, 3100, 60000, 2900]
    assert len(tuner.cache) == 2  # the 2048 class (2900, 3000, 3100) and the 32768 class (50000, 60000)


def test_fp64_problems_only_tune_the_stream_count():
    clock = FakeClock()
    calls = []
    fake = make_fake(clock, lambda p, ns, c: 1.0 / ns, calls)
    tuner = at.BatchTuner(streams=(1, 2), sample=4, reps=1, timer=clock)
    Ws = [np.zeros((4096, 32), dtype=np.float64) for _ in range(3)]
    _, _, _, _, cfg = at.rbgs_qr_batched_auto(Ws, 8, 64, 0, tuner=tuner, batched=fake, sync=lambda: None)
    assert cfg == [("fp64", 2)] * 3
    assert {c[1] for c in calls} == {"fp64"}


def test_refused_variants_are_skipped():
    clock = FakeClock()
    calls = []
    fake = make_fake(clock, lambda p, ns, c: 1.0, calls, fail=("f16x3", "tf32x3"))
    tuner = at.BatchTuner(streams=(4,), sample=1, reps=1, timer=clock)
    Ws = [np.zeros((1001, 16), dtype=np.float32)]
    _, _, _, _, cfg = at.rbgs_qr_batched_auto(Ws, 4, 32, 0, tuner=tuner, batched=fake, sync=lambda: None)
    assert cfg == [("fp32", 4)]
    fake_all = make_fake(clock, lambda p, ns, c: 1.0, [], fail=("f16x3", "tf32x3", "fp32"))
    with pytest.raises(RuntimeError):
        at.rbgs_qr_batched_auto(Ws, 4, 32, 0, tuner=at.BatchTuner(streams=(4,), timer=clock), batched=fake_all,
                                sync=lambda: None)


def test_variant_with_failing_statuses_is_rejected_even_when_fastest():
    """rbgs_qr_batched reports breakdowns (4) and timeouts (6) as per-problem
    statuses instead of raising.  A variant that breaks down stops early and
    would time fastest; the tuner must not cache it."""
    clock = FakeClock()
    calls = []
    cost = {"f16x3": 0.1, "tf32x3": 1.0, "fp32": 2.0}

    def fake(Ws, mbs, ks, seeds, sketch, prec, ls_iters, reorth, fine, interblock, nstreams):
        calls.append((len(Ws), prec, nstreams))
        clock.t += cost[prec]
        st = [4 if prec == "f16x3" and i == 1 else 0 for i in range(len(Ws))]
        return ([None] * len(Ws), [None] * len(Ws), st, [0] * len(Ws))

    tuner = at.BatchTuner(streams=(1,), sample=3, reps=2, timer=clock)
    Ws = [np.zeros((5000, 64), dtype=np.float32) for _ in range(4)]
    _, _, st, _, cfg = at.rbgs_qr_batched_auto(Ws, 16, 128, 0, tuner=tuner, batched=fake, sync=lambda: None)
    assert cfg == [("tf32x3", 1)] * 4 and st == [0] * 4
    key = next(iter(tuner.cache))
    assert ("f16x3", 1) in tuner.rejected[key] and ("f16x3", 1) not in tuner.trials[key]
    # a timeout on every candidate leaves nothing to choose from
    fake_to = make_fake(clock, lambda p, ns, c: 1.0, [])

    def timing_out(*a, **kw):
        q, r, s, p2 = fake_to(*a, **kw)
        return q, r, [6] * len(s), p2

    with pytest.raises(RuntimeError):
        at.rbgs_qr_batched_auto(Ws, 16, 128, 0, tuner=at.BatchTuner(streams=(1,), timer=clock), batched=timing_out,
                                sync=lambda: None)
