"""Autotuner for the launch shapes of the chi0 / E_c path.

Tunable shapes (all change speed, none changes the result beyond rounding):

* RPA_TUNE_PAIR_CHUNK: pairs per pair-density launch (the pair tile of the
  three transform kernels);
* RPA_TUNE_PD_FUSE: middle- and fastest-axis transforms as one kernel through
  shared memory, or two through global memory (bit-identical);
* RPA_TUNE_TC_PIPE: the tensor-core pipeline shape (64-element K stages x 2
  or 32-element stages x 4), split-bfloat16 modes only;
* RPA_TUNE_TC_FUSE: frequency weights applied inside the tensor-core kernel
  or stored per frequency before it (bit-identical), two-term mode only;
* RPA_TUNE_TC_FLUSH: folds between the register running sums' additions to
  the FP64 chi0, tensor-core modes only.

The tensor-core fold length is not tuned: it controls the truncation bias of
the FP32 accumulation (see include/rpa.h), not just speed.

``autotune(ctx, iqs, wq, omega, W)`` times one E_c evaluation per candidate
with the caller's synchronisation and leaves the fastest setting applied.
With ``greedy=True`` it tunes one knob at a time (the others at their best so
far), which needs the sum of the value counts instead of their product.
``BucketTuner`` keeps one result per (shape bucket, precision), so a batch of
instances tunes each distinct size class once and applies its result to every
instance of that class.
"""
from __future__ import annotations

import itertools
import time

from . import binding as b

DEFAULT_SPACE = {
    b.RPA_TUNE_PAIR_CHUNK: [0, 128, 512, 2048],
    b.RPA_TUNE_TC_FLUSH: [64, 256],
}


def space_for(precision: str) -> dict:
    """Search space of one precision mode: the tensor-core knobs only where
    they act."""
    sp = {b.RPA_TUNE_PAIR_CHUNK: [0, 512, 2048], b.RPA_TUNE_PD_FUSE: [0, 1]}
    if precision in ("bf16x2", "bf16x3"):
        sp[b.RPA_TUNE_TC_FLUSH] = [256, 64]
    if precision == "bf16x2":
        sp[b.RPA_TUNE_TC_PIPE] = [0, 1]
        sp[b.RPA_TUNE_TC_FUSE] = [0, 1]
    return sp


def shape_bucket(ng: int, pairs: int) -> tuple:
    """Coarse (NG, pairs) bucket: powers of two."""
    return (max(ng, 1).bit_length(), max(pairs, 1).bit_length())


def _time_once(ctx, iqs, wq, omega, W, sync) -> float:
    sync()
    t0 = time.perf_counter()
    b.rpa_energy(ctx, iqs, wq, omega, W)
    sync()
    return time.perf_counter() - t0


def autotune(ctx, iqs, wq, omega, W, space=None, reps=1, sync=None, log=None, greedy=False) -> dict:
    """Try the combinations of ``space`` ({param: [values]}, exhaustive, or one
    knob at a time with ``greedy``); apply and return the best."""
    space = DEFAULT_SPACE if space is None else space
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    keys = list(space)
    results = []

    def trial(setting):
        for k, v in setting.items():
            b.rpa_set_tuning(ctx, k, v)
        t = min(_time_once(ctx, iqs, wq, omega, W, sync) for _ in range(reps))
        results.append((t, dict(setting)))
        if log:
            log(f"autotune {setting}: {t * 1e3:.2f} ms")
        return t

    _time_once(ctx, iqs, wq, omega, W, sync)  # warm-up: buffers, grids
    if greedy:
        cur = {k: space[k][0] for k in keys}
        best_t = trial(cur)
        for k in keys:
            for v in space[k][1:]:
                cand = dict(cur)
                cand[k] = v
                t = trial(cand)
                if t < best_t:
                    best_t, cur = t, cand
        best = (best_t, cur)
    else:
        best = None
        for combo in itertools.product(*[space[k] for k in keys]):
            setting = dict(zip(keys, combo))
            t = trial(setting)
            if best is None or t < best[0]:
                best = (t, setting)
    for k, v in best[1].items():
        b.rpa_set_tuning(ctx, k, v)
    return {"best": best[1], "best_s": best[0], "tried": [(s, t) for t, s in results]}


def apply(ctx, setting: dict) -> None:
    for k, v in setting.items():
        b.rpa_set_tuning(ctx, int(k), int(v))


class BucketTuner:
    """One tuning result per (shape bucket, precision), applied per instance."""

    def __init__(self, precision: str, space=None, greedy=True, sync=None, log=None):
        self.precision = precision
        self.space = space_for(precision) if space is None else space
        self.greedy = greedy
        self.sync = sync
        self.log = log
        self.table: dict = {}

    def key(self, ng: int, pairs: int) -> tuple:
        return shape_bucket(ng, pairs) + (self.precision,)

    def tune(self, ctx, ng: int, pairs: int, iqs, wq, omega, W) -> dict:
        """Tune ``ctx`` if its bucket has no result yet; apply the bucket's result."""
        k = self.key(ng, pairs)
        if k not in self.table:
            self.table[k] = autotune(ctx, iqs, wq, omega, W, space=self.space, sync=self.sync, log=self.log,
                                     greedy=self.greedy)["best"]
        apply(ctx, self.table[k])
        return self.table[k]
