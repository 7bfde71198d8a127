"""Host logic of the autotuner without a GPU: the library calls are replaced by
fakes whose evaluation time depends on the applied setting, and the tuner must
try every combination once, leave the fastest applied and report it."""
import itertools

from paper_1307_8052_gb300 import autotune as at
from paper_1307_8052_gb300 import binding as b


def test_autotune_tries_every_combination_and_applies_the_fastest(monkeypatch):
    applied = {}
    calls = []
    # fake cost: fastest at chunk 512 with flush 256
    cost = {(c, f): 1.0 + abs(c - 512) / 1000 + (0.0 if f == 256 else 0.3)
            for c, f in itertools.product([0, 128, 512, 2048], [64, 256])}
    clock = [0.0]

    def fake_set_tuning(ctx, param, value):
        assert ctx == "ctx"
        applied[param] = value

    def fake_energy(ctx, iqs, wq, omega, W):
        key = (applied.get(b.RPA_TUNE_PAIR_CHUNK, 0), applied.get(b.RPA_TUNE_TC_FLUSH, 256))
        calls.append(key)
        clock[0] += cost[key]
        return 0.0, None

    monkeypatch.setattr(b, "rpa_set_tuning", fake_set_tuning)
    monkeypatch.setattr(b, "rpa_energy", fake_energy)
    monkeypatch.setattr(at.time, "perf_counter", lambda: clock[0])
    res = at.autotune("ctx", [0], [1.0], [1.0], [1.0], sync=lambda: None)
    assert res["best"] == {b.RPA_TUNE_PAIR_CHUNK: 512, b.RPA_TUNE_TC_FLUSH: 256}
    assert abs(res["best_s"] - 1.0) < 1e-12
    # one warm-up, then each of the 8 combinations once
    assert len(calls) == 1 + 8
    assert sorted(set(calls[1:])) == sorted(cost)
    assert applied == res["best"]
    assert len(res["tried"]) == 8


def test_apply_and_shape_bucket(monkeypatch):
    seen = []
    monkeypatch.setattr(b, "rpa_set_tuning", lambda ctx, k, v: seen.append((ctx, k, v)))
    at.apply("c", {str(b.RPA_TUNE_PAIR_CHUNK): "128"})
    assert seen == [("c", b.RPA_TUNE_PAIR_CHUNK, 128)]
    assert at.shape_bucket(1200, 153600) == at.shape_bucket(1100, 140000)
    assert at.shape_bucket(1200, 153600) != at.shape_bucket(3000, 153600)
    assert at.shape_bucket(0, 0) == (1, 1)


def _fake_lib(monkeypatch, cost_of):
    applied = {}
    calls = []
    clock = [0.0]

    def fake_set_tuning(ctx, param, value):
        applied.setdefault(ctx, {})[param] = value

    def fake_energy(ctx, iqs, wq, omega, W):
        calls.append((ctx, dict(applied.get(ctx, {}))))
        clock[0] += cost_of(applied.get(ctx, {}))
        return 0.0, None

    monkeypatch.setattr(b, "rpa_set_tuning", fake_set_tuning)
    monkeypatch.setattr(b, "rpa_energy", fake_energy)
    monkeypatch.setattr(at.time, "perf_counter", lambda: clock[0])
    return applied, calls


def test_greedy_tunes_one_knob_at_a_time(monkeypatch):
    # separable cost: each knob's best value is independent of the others
    best = {b.RPA_TUNE_PAIR_CHUNK: 512, b.RPA_TUNE_PD_FUSE: 0, b.RPA_TUNE_TC_FLUSH: 256,
            b.RPA_TUNE_TC_PIPE: 1, b.RPA_TUNE_TC_FUSE: 0}

    def cost(s):
        return 1.0 + sum(0.1 for k, v in best.items() if s.get(k) != v)

    applied, calls = _fake_lib(monkeypatch, cost)
    space = at.space_for("bf16x2")
    res = at.autotune("ctx", [0], [1.0], [1.0], [1.0], space=space, sync=lambda: None, greedy=True)
    assert res["best"] == best
    # warm-up + first point + (values - 1) per knob, not the product
    assert len(calls) == 1 + 1 + sum(len(v) - 1 for v in space.values())
    assert applied["ctx"] == best


def test_space_depends_on_precision():
    assert b.RPA_TUNE_TC_PIPE not in at.space_for("fp64")
    assert b.RPA_TUNE_TC_FLUSH not in at.space_for("fp32")
    assert b.RPA_TUNE_TC_FUSE in at.space_for("bf16x2")
    assert b.RPA_TUNE_TC_FUSE not in at.space_for("bf16x3")


def test_bucket_tuner_tunes_each_bucket_once(monkeypatch):
    def cost(s):
        return 1.0 + (0.5 if s.get(b.RPA_TUNE_PAIR_CHUNK) != 2048 else 0.0)

    applied, calls = _fake_lib(monkeypatch, cost)
    bt = at.BucketTuner("fp64", sync=lambda: None)
    r1 = bt.tune("c1", 1200, 150000, [0], [1.0], [1.0], [1.0])
    n1 = len(calls)
    r2 = bt.tune("c2", 1100, 140000, [0], [1.0], [1.0], [1.0])   # same bucket: no new timing
    assert len(calls) == n1 and r1 == r2
    assert applied["c2"][b.RPA_TUNE_PAIR_CHUNK] == 2048
    bt.tune("c3", 3000, 140000, [0], [1.0], [1.0], [1.0])        # new bucket: tuned
    assert len(calls) > n1 and len(bt.table) == 2
