"""Edge cases through the C ABI against the oracle, in every mode: a
transition without pairs, degenerate band energies across the Fermi level,
a one-vector response sphere (far below one tensor-core tile), a single
frequency, and response spheres around the Cholesky panel width."""
import dataclasses

import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu

MODES = ["fp64", "fp32", "bf16x2", "bf16x3"]
TOL = {"fp64": 1e-11, "fp32": 4e-6, "bf16x2": 2e-5, "bf16x3": 4e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()


def _run(p, precision, iq, om, W):
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        qf = (lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm)) if p.paw else None
        b.load_problem(ctx, p, paw_Q=qf)
        chi = b.rpa_chi0(ctx, iq, om)
        E, t = b.rpa_energy(ctx, [iq], [1.0], om, W)
        return chi, E, t
    finally:
        b.rpa_destroy(ctx)


def _ref(p, iq, om, W):
    qp = p.qpoints[iq]
    gm = o.g_sphere(p.cell, qp.q_red, p.ecut_chi)
    Q = syn.paw_Q(p.paw, p.cell, qp.q_red, gm) if p.paw else None
    chi = o.chi0(p, iq, om, Q)
    return chi, o.ec_terms(chi, o.coulomb(p.cell, qp.q_red, gm))


@pytest.mark.parametrize("precision", MODES)
def test_transition_without_pairs(precision):
    """All bands of set 0 empty: its transitions add nothing; the other
    transition of the same q-point still counts."""
    p = syn.small_problem(config_tag=86)
    s0 = p.sets[0]
    p = dataclasses.replace(p, sets=[dataclasses.replace(s0, f=np.zeros_like(s0.f))] + p.sets[1:])
    om, W = o.frequency_grid(4)
    chi, E, t = _run(p, precision, 1, om, W)
    ref, tr = _ref(p, 1, om, W)
    assert np.abs(ref).max() > 0
    assert np.abs(chi - ref).max() <= TOL[precision] * np.abs(ref).max()
    assert np.abs(t[0] - tr).max() <= max(TOL[precision], 1e-10) * np.abs(tr).max()


@pytest.mark.parametrize("precision", MODES)
def test_degenerate_energies_across_the_fermi_level(precision):
    """Occupied and empty bands with equal energies (weight 2 d/(w^2+d^2) = 0)."""
    p = syn.small_problem(config_tag=85)
    sets = []
    for s_ in p.sets:
        eps = s_.eps.copy()
        no = int(np.sum(s_.f > 0))
        eps[no] = eps[no - 1]  # lowest empty band degenerate with the highest occupied one
        sets.append(dataclasses.replace(s_, eps=eps))
    p = dataclasses.replace(p, sets=sets)
    om, W = o.frequency_grid(4)
    chi, E, t = _run(p, precision, 0, om, W)
    ref, tr = _ref(p, 0, om, W)
    assert np.abs(chi - ref).max() <= TOL[precision] * np.abs(ref).max()
    assert np.abs(t[0] - tr).max() <= max(TOL[precision], 1e-10) * np.abs(tr).max()


@pytest.mark.parametrize("precision", MODES)
def test_tiny_sphere_and_one_frequency(precision):
    """A response cutoff that keeps only the two shortest q+G (NG = 2, q at the
    zone boundary) and a single frequency."""
    p = syn.small_problem(config_tag=84, ecut_chi=0.15)
    iq = 1
    assert len(o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi)) == 2
    om, W = o.frequency_grid(1)
    chi, E, t = _run(p, precision, iq, om, W)
    ref, tr = _ref(p, iq, om, W)
    assert chi.shape == (1, 2, 2)
    assert np.abs(chi - ref).max() <= TOL[precision] * np.abs(ref).max()
    assert np.abs(t[0] - tr).max() <= max(TOL[precision], 1e-10) * np.abs(tr).max()


@pytest.mark.parametrize("ecut_chi", [2.0, 2.4, 3.3, 5.5])
def test_logdet_lookahead_at_panel_boundaries(ecut_chi):
    """Response spheres around the 32-wide Cholesky panels (NG 29/32: one
    panel; 35/40: a panel and a ragged strip; 65/64: a strip with and without
    a rest update; 141/130: several rest updates, ragged last tile): the
    float-float factorisation with the look-ahead equals the one-stream
    factorisation bit for bit, and both match FP64 eigenvalues of the GPU's own
    chi0."""
    p = syn.small_problem(config_tag=84, ecut_chi=ecut_chi)
    om, W = o.frequency_grid(p.nw)
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, "bf16x2")
    try:
        b.load_problem(ctx, p, paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))
        for iq, qp in enumerate(p.qpoints):
            chi = b.rpa_chi0(ctx, iq, om)
            want = o.ec_terms(chi, o.coulomb(p.cell, qp.q_red, b.rpa_gvectors(ctx, iq)))
            b.rpa_set_tuning(ctx, b.RPA_TUNE_LOGDET, 2)
            _, t2 = b.rpa_energy(ctx, [iq], [1.0], om, W)
            b.rpa_set_tuning(ctx, b.RPA_TUNE_LOGDET, 1)
            _, t1 = b.rpa_energy(ctx, [iq], [1.0], om, W)
            assert np.array_equal(t1, t2)
            assert np.abs(t2[0] - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        b.rpa_destroy(ctx)
