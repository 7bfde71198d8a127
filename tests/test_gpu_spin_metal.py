"""GPU parity for a spin-polarised metal (NEXT-2): one orbital set per
(k, spin), Fermi-Dirac occupations with partially occupied bands in both
channels, spin factor 1, same-spin transitions with umklapp, PAW."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-11, 1e-10), "fp32": (4e-6, 1e-6), "bf16x2": (2e-5, 5e-6), "bf16x3": (4e-6, 1e-6)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()


@pytest.fixture(scope="module")
def case():
    p = syn.spin_metal_problem()
    om, W = o.frequency_grid(p.nw)
    Qs = {iq: syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi))
          for iq, qp in enumerate(p.qpoints)}
    chis = {iq: o.chi0(p, iq, om, Qs[iq]) for iq in Qs}
    E, terms = o.energy(p, om, W, Qs=Qs)
    return p, om, W, chis, E, terms


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x2", "bf16x3"])
def test_spin_polarised_metal(case, precision):
    p, om, W, chis, E_ref, t_ref = case
    assert p.spin_factor == 1.0
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))
        tc, te = TOL[precision]
        for iq, ref in chis.items():
            chi = b.rpa_chi0(ctx, iq, om)
            assert np.abs(chi - ref).max() <= tc * np.abs(ref).max(), iq
        iqs = list(range(len(p.qpoints)))
        E, t = b.rpa_energy(ctx, iqs, [qp.weight for qp in p.qpoints], om, W)
        assert abs(E - E_ref) <= max(te, 1e-10) * abs(E_ref)
        assert np.abs(t - t_ref).max() <= te * np.abs(t_ref).max()
    finally:
        b.rpa_destroy(ctx)
