"""GPU parity of rpa_energy_backward through the optical-limit head (q = 0 with
rpa_set_optical, Eqs. 12-14): dE_c/dC, dE_c/dP and dE_c/dchi0 against the
oracle's analytic gradient in every mode, and central finite differences of the
GPU energy in FP64."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu

QDIR = [0.3, 1.0, -0.4]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()


def _problem():
    # a q = 0 point (k -> k transitions) and a finite q with umklapp, PAW on both
    return syn.small_problem(config_tag=98, a=5.0, grid=(12, 12, 12), ecut_wf=2.5, ecut_chi=1.2, nocc=2, nunocc=7,
                             mesh=(2, 1, 1), nproj=(2, 3), nw=4)


def _ctx(p, precision):
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    b.load_problem(ctx, p, paw_Q=lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
    b.rpa_set_optical(ctx, 0, QDIR, p.paw.nproj, syn.paw_Qnabla(p.paw, p.config))
    return ctx


def _grad(ctx, p, om, W, iqs):
    sets = list(range(len(p.sets)))
    dC = [np.zeros_like(s.C) for s in p.sets]
    dP = [np.zeros_like(s.P) for s in p.sets]
    dchi = [np.zeros((len(om), len(b.rpa_gvectors(ctx, iq)), len(b.rpa_gvectors(ctx, iq))), dtype=np.complex128)
            for iq in iqs]
    E = b.rpa_energy_backward(ctx, iqs, [p.qpoints[i].weight for i in iqs], om, W, 1.0, sets, dC, dP, dchi)
    return E, dC, dP, dchi


def _rel(a, r):
    return np.abs(a - r).max() / max(np.abs(r).max(), 1e-300)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-5), ("bf16x2", 1e-4), ("bf16x3", 2e-5)])
def test_optical_backward_matches_oracle_gradient(precision, tol):
    p = _problem()
    assert np.all(p.qpoints[0].q_red == 0) and np.abs(p.qpoints[1].G0).sum() > 0
    om, W = o.frequency_grid(p.nw)
    Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
    opt = {0: (QDIR, syn.paw_Qnabla(p.paw, p.config))}
    iqs = [0, 1]
    Er, gC, gP, gchi = o.energy_grad(p, om, W, Qs, iqs=iqs, optical=opt)
    ctx = _ctx(p, precision)
    try:
        E, dC, dP, dchi = _grad(ctx, p, om, W, iqs)
    finally:
        b.rpa_destroy(ctx)
    assert abs(E - Er) < max(tol, 1e-10) * abs(Er)
    for s in range(len(p.sets)):
        assert _rel(dC[s], gC[s]) < tol, ("dC", s)
        assert _rel(dP[s], gP[s]) < tol, ("dP", s)
    for i, iq in enumerate(iqs):
        assert _rel(dchi[i], gchi[iq]) < max(tol, 1e-10), ("dchi", iq)


def test_optical_backward_central_differences_fp64():
    p = _problem()
    om, W = o.frequency_grid(p.nw)
    iqs = [0]
    ctx = _ctx(p, "fp64")
    try:
        E0, dC, dP, _ = _grad(ctx, p, om, W, iqs)
        rng = np.random.default_rng(23)
        h = 1e-6
        for trial in range(4):
            s = trial % len(p.sets)
            which = "C" if trial < 2 else "P"
            base = getattr(p.sets[s], which).copy()
            d = rng.standard_normal(base.shape) + 1j * rng.standard_normal(base.shape)
            vals = []
            for sign in (1, -1):
                new = base + sign * h * d
                if which == "C":
                    b.rpa_set_orbitals(ctx, s, p.sets[s].k_red, p.sets[s].miller, new, p.sets[s].eps, p.sets[s].f)
                    b.rpa_set_paw(ctx, s, p.paw.nproj, p.sets[s].P)
                else:
                    b.rpa_set_paw(ctx, s, p.paw.nproj, new)
                vals.append(b.rpa_energy(ctx, iqs, [p.qpoints[0].weight], om, W)[0])
            b.rpa_set_orbitals(ctx, s, p.sets[s].k_red, p.sets[s].miller, p.sets[s].C, p.sets[s].eps, p.sets[s].f)
            b.rpa_set_paw(ctx, s, p.paw.nproj, p.sets[s].P)
            fd = (vals[0] - vals[1]) / (2 * h)
            g = dC[s] if which == "C" else dP[s]
            an = float(np.sum(np.conj(g) * d).real)
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (which, fd, an)
    finally:
        b.rpa_destroy(ctx)
