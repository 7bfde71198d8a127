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
