"""Autotuner for the launch shapes of the chi0 / E_c path.

The tunable shapes are the number of pairs per pair-density launch
(RPA_TUNE_PAIR_CHUNK: the pair tile of the three transform kernels), the
register flush interval of the tensor-core epilogue (RPA_TUNE_TC_FLUSH) and the
operand budget that sets how many occupied rows share one rank-k block
(RPA_TUNE_OPERAND_MB).  The tensor-core fold length is not tuned: it controls
the truncation bias of the FP32 accumulation (see include/rpa.h), not just speed.

``autotune(ctx, iqs, wq, omega, W)`` times one E_c evaluation per candidate
with CUDA events on the context's stream and leaves the fastest setting
applied.  Results are keyed by a coarse shape bucket so a batch of instances of
similar size can share one tuning run.
"""
from __future__ import annotations

import itertools
import time

from . import binding as b

DEFAULT_SPACE = {
    b.RPA_TUNE_PAIR_CHUNK: [0, 128, 512, 2048],
    b.RPA_TUNE_TC_FLUSH: [64, 256],
}


def shape_bucket(ng: int, pairs: int) -> tuple:
    """Coarse (NG, pairs) bucket: powers of two."""
    return (max(ng, 1).bit_length(), max(pairs, 1).bit_length())


def _time_once(ctx, iqs, wq, omega, W, sync) -> float:
    sync()
    t0 = time.perf_counter()
    b.rpa_energy(ctx, iqs, wq, omega, W)
    sync()
    return time.perf_counter() - t0


def autotune(ctx, iqs, wq, omega, W, space=None, reps=1, sync=None, log=None) -> dict:
    """Try every combination in ``space`` ({param: [values]}); apply and return the best."""
    space = DEFAULT_SPACE if space is None else space
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    keys = list(space)
    best = None
    results = []
    _time_once(ctx, iqs, wq, omega, W, sync)  # warm-up: buffers, grids
    for combo in itertools.product(*[space[k] for k in keys]):
        for k, v in zip(keys, combo):
            b.rpa_set_tuning(ctx, k, v)
        t = min(_time_once(ctx, iqs, wq, omega, W, sync) for _ in range(reps))
        setting = dict(zip(keys, combo))
        results.append((t, setting))
        if log:
            log(f"autotune {setting}: {t * 1e3:.2f} ms")
        if best is None or t < best[0]:
            best = (t, setting)
    for k, v in best[1].items():
        b.rpa_set_tuning(ctx, k, v)
    return {"best": best[1], "best_s": best[0], "tried": [(s, t) for t, s in results]}


def apply(ctx, setting: dict) -> None:
    for k, v in setting.items():
        b.rpa_set_tuning(ctx, int(k), int(v))
