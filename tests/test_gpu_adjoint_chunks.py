"""The pair-density adjoint (Eq. 10 transposed) under its chunk shapes, through
the C ABI: the fused stage-A^T kernel on chunks of two occupied bands and a
one-band tail, ragged chunks of unoccupied bands, and the two-kernel form
that keeps x-bar in memory (taken when the slowest axis of the G sphere is
wider than 16), each against the oracle's analytic gradient."""
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


def _grad(p, precision, chunk=0):
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, paw_Q=lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PAIR_CHUNK, chunk)
        om, W = o.frequency_grid(p.nw)
        iqs = list(range(len(p.qpoints)))
        dC = [np.zeros_like(s.C) for s in p.sets]
        dP = [np.zeros_like(s.P) for s in p.sets]
        E = b.rpa_energy_backward(ctx, iqs, [q.weight for q in p.qpoints], om, W, 1.0, list(range(len(p.sets))),
                                  dC, dP)
    finally:
        b.rpa_destroy(ctx)
    return E, dC, dP


def _rel(a, r):
    return np.abs(a - r).max() / max(np.abs(r).max(), 1e-300)


def _oracle(p):
    om, W = o.frequency_grid(p.nw)
    Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
    E, gC, gP, _ = o.energy_grad(p, om, W, Qs)
    return E, gC, gP


@pytest.fixture(scope="module")
def three_band():
    # three occupied bands: one two-band chunk and a one-band tail
    p = syn.small_problem(config_tag=98, a=5.0, grid=(12, 12, 12), ecut_wf=2.5, ecut_chi=1.2, nocc=3, nunocc=7,
                          mesh=(2, 1, 1), nproj=(2, 3), nw=4)
    return p, _oracle(p)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("bf16x2", 1e-4)])
@pytest.mark.parametrize("chunk", [0, 5])
def test_adjoint_chunks_match_oracle(three_band, precision, tol, chunk):
    # chunk 5: two occupied x two unoccupied bands per launch, the last
    # unoccupied chunk one band wide
    p, (Er, gC, gP) = three_band
    E, dC, dP = _grad(p, precision, chunk)
    assert abs(E - Er) < max(tol, 1e-10) * abs(Er)
    for s in range(len(p.sets)):
        assert _rel(dC[s], gC[s]) < tol, ("dC", s)
        assert _rel(dP[s], gP[s]) < tol, ("dP", s)


def test_adjoint_chunk_shapes_agree_fp64(three_band):
    p, _ = three_band
    E0, dC0, dP0 = _grad(p, "fp64", 0)
    E5, dC5, dP5 = _grad(p, "fp64", 5)
    assert abs(E5 - E0) <= 1e-13 * abs(E0)
    for s in range(len(p.sets)):
        assert _rel(dC5[s], dC0[s]) < 1e-12
        assert _rel(dP5[s], dP0[s]) < 1e-12


def test_adjoint_wide_slowest_axis_two_kernel_form():
    # a cell long along its first axis: the chi0 sphere spans 17 planes there
    cell = np.diag([36.0, 5.5, 4.5])
    kmesh = [np.zeros(3), np.array([0.5, 0.0, 0.0])]
    sets = [syn.make_orbitals(99, i, cell, k, 2.5, 2, 5) for i, k in enumerate(kmesh)]
    paw = syn.make_paw_setup(99, [2, 3])
    for i, s in enumerate(sets):
        s.P = syn.make_projections(99, i, s.C.shape[0], int(paw.nproj.sum()))
    p = syn.Problem("wide-99", 99, cell, (48, 12, 12), 2.5, 1.2, 2.0, 2, sets, syn.mesh_qpoints(kmesh, kmesh), 3, paw)
    g = o.g_sphere(cell, p.qpoints[0].q_red, p.ecut_chi)
    assert np.ptp(g[:, 0]) + 1 > 16
    Er, gC, gP = _oracle(p)
    E, dC, dP = _grad(p, "fp64")
    assert abs(E - Er) < 1e-10 * abs(Er)
    for s in range(len(p.sets)):
        assert _rel(dC[s], gC[s]) < 1e-9, ("dC", s)
        assert _rel(dP[s], gP[s]) < 1e-9, ("dP", s)
