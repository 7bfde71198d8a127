"""GPU parity of the optical limit q -> 0 (Eqs. 12-14) through the C ABI:
chi0 and the energy terms of a q = 0 point with the head and wings, against
the oracle, in every precision mode."""
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
    p = syn.small_problem(config_tag=93)
    iq = 0
    assert np.all(p.qpoints[iq].q_red == 0)
    qdir = np.array([0.3, -0.4, 1.0])
    Qn = syn.paw_Qnabla(p.paw, 93)
    om, W = o.frequency_grid(p.nw)
    gm = o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi)
    Qf = syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm)
    chi = o.chi0(p, iq, om, Qf, optical=(qdir, Qn))
    v = o.coulomb(p.cell, p.qpoints[iq].q_red, gm, optical=True)
    return p, iq, qdir, Qn, om, W, chi, o.ec_terms(chi, v)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x2", "bf16x3"])
def test_optical_limit_chi0_and_terms(case, precision):
    p, iq, qdir, Qn, om, W, chi_ref, e_ref = case
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, qs=[iq], paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))
        plain = b.rpa_chi0(ctx, iq, om)
        b.rpa_set_optical(ctx, iq, qdir, p.paw.nproj, Qn)
        chi = b.rpa_chi0(ctx, iq, om)
        _, t = b.rpa_energy(ctx, [iq], [1.0], om, W)
        tc, te = TOL[precision]
        assert np.abs(chi - chi_ref).max() <= tc * np.abs(chi_ref).max()
        assert np.abs(t[0] - e_ref).max() <= te * np.abs(e_ref).max()
        # the head and wings differ from the plain q = 0 result, the body does not
        ig0 = int(np.flatnonzero(np.all(b.rpa_gvectors(ctx, iq) == 0, axis=1))[0])
        assert np.abs(chi[:, ig0, :] - plain[:, ig0, :]).max() > 1e-3 * np.abs(chi_ref).max()
        body = np.delete(np.delete(chi, ig0, axis=1), ig0, axis=2)
        body0 = np.delete(np.delete(plain, ig0, axis=1), ig0, axis=2)
        assert np.abs(body - body0).max() <= 1e-12 * np.abs(chi_ref).max() + (0 if precision == "fp64" else 1e-7)
        # switching the limit off restores the plain q = 0 point
        b.rpa_set_optical(ctx, iq, None)
        assert np.abs(b.rpa_chi0(ctx, iq, om) - plain).max() <= 1e-12 * np.abs(plain).max() + (
            0 if precision == "fp64" else 1e-7)
    finally:
        b.rpa_destroy(ctx)


def test_optical_limit_argument_checks(case):
    p, iq, qdir, Qn, om, W, _, _ = case
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, "fp64")
    try:
        b.load_problem(ctx, p, paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))
        nonzero = [i for i, qp in enumerate(p.qpoints) if np.any(qp.q_red != 0)][0]
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_optical(ctx, nonzero, qdir)
        assert e.value.status == b.RPA_ERR_ARG
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_optical(ctx, iq, [0.0, 0.0, 0.0])
        assert e.value.status == b.RPA_ERR_ARG
        b.rpa_set_optical(ctx, iq, qdir, p.paw.nproj, Qn)
        # the gradient runs through the head (tests/test_gpu_backward_optical.py
        # checks its values); its energy is the forward energy
        E_bwd = b.rpa_energy_backward(ctx, [iq], [1.0], om, W, 1.0, [0], [np.zeros_like(p.sets[0].C)])
        E_fwd, _ = b.rpa_energy(ctx, [iq], [1.0], om, W)
        assert abs(E_bwd - E_fwd) <= 1e-12 * abs(E_fwd)
    finally:
        b.rpa_destroy(ctx)
