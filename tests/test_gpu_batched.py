"""Batched evaluation: (q, cell) instances of different sizes queued without
host synchronisation and captured into one CUDA graph must reproduce the plain
per-instance rpa_energy results and match the oracle.  In the split-bfloat16
mode the graph is built around persistent rank-k launches that pull (block,
tile, frequency) items of every instance from a device queue; those give
bit-identical energies to the per-instance form, with one group for all
blocks and with a budget small enough that every block forms its own group
(q-points whose blocks span several launches)."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu

SHAPES = [(2, 14, 1.2), (3, 20, 1.5), (4, 9, 1.0), (2, 30, 1.8), (5, 12, 1.3), (3, 25, 1.6), (2, 7, 0.9), (4, 18, 1.4)]


def _instances():
    out = []
    for i, (nocc, nunocc, ecut) in enumerate(SHAPES):
        out.append(syn.small_problem(config_tag=110 + i, a=5.5 + 0.25 * i, grid=(14, 14, 14), ecut_wf=2.5,
                                     ecut_chi=ecut, nocc=nocc, nunocc=nunocc, mesh=(2, 1, 1), nproj=(2, 3), nw=6))
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()


def _contexts(probs, precision, stream):
    ctxs = []
    for p in probs:
        ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision, stream=stream.cuda_stream)
        b.load_problem(ctx, p, paw_Q=lambda iq, gm, p=p: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
        ctxs.append(ctx)
    return ctxs


def _graph_energies(ctxs, probs, W):
    g = b.rpa_graph_create(ctxs, [list(range(len(p.qpoints))) for p in probs])
    try:
        out = []
        for replay in range(2):
            b.rpa_graph_launch(g)
            out.append([b.rpa_energy_collect(ctx, [qp.weight for qp in p.qpoints], W, len(p.qpoints))[0]
                        for ctx, p in zip(ctxs, probs)])
        return out
    finally:
        b.rpa_graph_destroy(g)


@pytest.mark.parametrize("precision", ["fp64", "bf16x2"])
def test_graph_matches_sequential_and_oracle(precision):
    import torch
    probs = _instances()
    stream = torch.cuda.Stream()
    ctxs = _contexts(probs, precision, stream)
    try:
        om, W = o.frequency_grid(6)
        seq = []
        for ctx, p in zip(ctxs, probs):
            b.rpa_set_frequencies(ctx, om)
            iqs = list(range(len(p.qpoints)))
            seq.append(b.rpa_energy(ctx, iqs, [qp.weight for qp in p.qpoints], om, W)[0])
        for replay in _graph_energies(ctxs, probs, W):
            for k in range(len(probs)):
                assert abs(replay[k] - seq[k]) <= 1e-12 * abs(seq[k]), k
        tol = 1e-10 if precision == "fp64" else 1e-6
        for k, p in enumerate(probs):
            Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
            Er, _ = o.energy(p, om, W, Qs)
            assert abs(seq[k] - Er) < tol * abs(Er), k
    finally:
        for ctx in ctxs:
            b.rpa_destroy(ctx)


@pytest.mark.parametrize("budget_mb", [16384, 1])
def test_persistent_graph_is_bit_identical_to_per_context_graph(budget_mb):
    import torch
    probs = _instances()
    stream = torch.cuda.Stream()
    ctxs = _contexts(probs, "bf16x2", stream)
    try:
        om, W = o.frequency_grid(6)
        for ctx in ctxs:
            b.rpa_set_frequencies(ctx, om)
        b.rpa_set_tuning(ctxs[0], b.RPA_TUNE_BATCH_PERSIST, 0)
        plain = _graph_energies(ctxs, probs, W)[0]
        b.rpa_set_tuning(ctxs[0], b.RPA_TUNE_BATCH_PERSIST, 1)
        b.rpa_set_tuning(ctxs[0], b.RPA_TUNE_BATCH_MB, budget_mb)
        persistent = _graph_energies(ctxs, probs, W)
        for replay in persistent:
            assert replay == plain
        # the per-context sequence after the graphs still agrees
        for k, (ctx, p) in enumerate(zip(ctxs, probs)):
            E = b.rpa_energy(ctx, list(range(len(p.qpoints))), [qp.weight for qp in p.qpoints], om, W)[0]
            assert E == plain[k]
    finally:
        for ctx in ctxs:
            b.rpa_destroy(ctx)


def test_graph_requires_shared_stream():
    p = _instances()[0]
    a = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, "fp64")
    c = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, "fp64")
    try:
        for ctx in (a, c):
            b.load_problem(ctx, p, paw_Q=lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
            b.rpa_set_frequencies(ctx, [0.5, 1.0])
        with pytest.raises(b.RpaError) as e:
            b.rpa_graph_create([a, c], [[0], [0]])
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(a)
        b.rpa_destroy(c)
