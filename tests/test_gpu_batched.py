"""Batched evaluation: several (q, cell) instances of different sizes queued
without host synchronisation and captured into one CUDA graph must reproduce
the plain per-instance rpa_energy results (same kernels, same order), and
match the oracle."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu


def _instances():
    out = []
    for i, (nocc, nunocc, ecut) in enumerate([(2, 14, 1.2), (3, 20, 1.5), (4, 9, 1.0)]):
        out.append(syn.small_problem(config_tag=110 + i, a=5.5 + 0.5 * i, grid=(14, 14, 14), ecut_wf=2.5,
                                     ecut_chi=ecut, nocc=nocc, nunocc=nunocc, mesh=(2, 1, 1), nproj=(2, 3), nw=6))
    return out


@pytest.mark.parametrize("precision", ["fp64", "bf16x2"])
def test_graph_matches_sequential_and_oracle(precision):
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()
    probs = _instances()
    stream = torch.cuda.Stream()
    ctxs = []
    try:
        for p in probs:
            ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision,
                               stream=stream.cuda_stream)
            b.load_problem(ctx, p, paw_Q=lambda iq, gm, p=p: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
            ctxs.append(ctx)
        om, W = o.frequency_grid(6)
        seq = []
        for ctx, p in zip(ctxs, probs):
            b.rpa_set_frequencies(ctx, om)
            iqs = list(range(len(p.qpoints)))
            seq.append(b.rpa_energy(ctx, iqs, [qp.weight for qp in p.qpoints], om, W)[0])
        g = b.rpa_graph_create(ctxs, [list(range(len(p.qpoints))) for p in probs])
        try:
            for replay in range(2):
                b.rpa_graph_launch(g)
                for k, (ctx, p) in enumerate(zip(ctxs, probs)):
                    E, terms = b.rpa_energy_collect(ctx, [qp.weight for qp in p.qpoints], W, len(p.qpoints))
                    assert abs(E - seq[k]) <= 1e-12 * abs(seq[k]), (replay, k)
        finally:
            b.rpa_graph_destroy(g)
        p = probs[1]
        Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
        Er, _ = o.energy(p, om, W, Qs)
        assert abs(seq[1] - Er) < (1e-10 if precision == "fp64" else 1e-6) * abs(Er)
    finally:
        for ctx in ctxs:
            b.rpa_destroy(ctx)


def test_graph_requires_shared_stream():
    import torch
    build()
    b.load()
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
