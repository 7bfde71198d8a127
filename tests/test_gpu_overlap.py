"""The log-det of each q-point (Eqs. 1-2) on its own stream beside chi0 of the
next q-point: the same kernels on the same data, so E_c and every term must be
bit-identical to the one-stream order, in the FP64 and the mixed modes, for a
q-set whose response spheres differ in size, through rpa_energy and through a
captured per-context graph."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()


@pytest.mark.parametrize("precision", ["fp64", "bf16x2"])
def test_logdet_overlap_bit_identical(precision):
    import torch
    p = syn.small_problem(config_tag=96, mesh=(2, 2, 1), nw=6)
    iqs = list(range(len(p.qpoints)))
    wq = [qp.weight for qp in p.qpoints]
    om, W = o.frequency_grid(p.nw)
    stream = torch.cuda.Stream()
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision, stream=stream.cuda_stream)
    try:
        ngs = b.load_problem(ctx, p, paw_Q=lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
        assert len(set(ngs)) > 1
        E1, t1 = b.rpa_energy(ctx, iqs, wq, om, W)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_LD_OVERLAP, 0)
        E0, t0 = b.rpa_energy(ctx, iqs, wq, om, W)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_LD_OVERLAP, 1)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_BATCH_PERSIST, 0)  # the per-context graph form
        b.rpa_set_frequencies(ctx, om)
        g = b.rpa_graph_create([ctx], [iqs])
        try:
            b.rpa_graph_launch(g)
            Eg, tg = b.rpa_energy_collect(ctx, wq, W, len(iqs))
        finally:
            b.rpa_graph_destroy(g)
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_LD_OVERLAP, 2)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)
    assert E1 == E0 and np.array_equal(t1, t0)
    assert Eg == E0 and np.array_equal(np.asarray(tg), np.asarray(t0))
    Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
    E_ref, _ = o.energy(p, om, W, Qs)
    assert abs(E1 - E_ref) <= (1e-10 if precision == "fp64" else 1e-6) * abs(E_ref)
