"""GPU parity of rpa_energy_backward: dE_c/dchi0, dE_c/dC and dE_c/dP against
the oracle's analytic gradient and against central finite differences of the
GPU energy."""
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


def _problem(tag=97):
    return syn.small_problem(config_tag=tag, a=5.0, grid=(12, 12, 12), ecut_wf=2.5, ecut_chi=1.2, nocc=2, nunocc=7,
                             mesh=(2, 1, 1), nproj=(2, 3), nw=4)


def _ctx(p, precision):
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    b.load_problem(ctx, p, paw_Q=lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm))
    return ctx


def _grad(ctx, p, om, W, iqs):
    sets = list(range(len(p.sets)))
    dC = [np.zeros_like(s.C) for s in p.sets]
    dP = [np.zeros_like(s.P) for s in p.sets]
    dchi = []
    for iq in iqs:
        ng = len(b.rpa_gvectors(ctx, iq))
        dchi.append(np.zeros((len(om), ng, ng), dtype=np.complex128))
    wq = [p.qpoints[i].weight for i in iqs]
    E = b.rpa_energy_backward(ctx, iqs, wq, om, W, 1.0, sets, dC, dP, dchi)
    return E, dC, dP, dchi


def _rel(a, r):
    return np.abs(a - r).max() / max(np.abs(r).max(), 1e-300)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("bf16x2", 1e-4)])
def test_general_paw_q_forward_and_backward(precision, tol):
    """Q^a_ij(G) without i <-> j symmetry (the synthetic c_ij are symmetric, as
    for real partial waves; the header's Q is general): chi0 and the gradient
    must tell i, the conjugated projection's index, from j.  Element by element
    against the oracle."""
    p = _problem(tag=86)
    om, W = o.frequency_grid(p.nw)
    rng = np.random.default_rng(19)
    Qs = []
    for qp in p.qpoints:
        Q = syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi))
        Qs.append(Q + 0.05 * (rng.standard_normal(Q.shape) + 1j * rng.standard_normal(Q.shape)))

    def paw_Q(iq, gm):
        assert np.array_equal(gm, o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi))
        return Qs[iq]

    iqs = list(range(len(p.qpoints)))
    Er, gC, gP, gchi = o.energy_grad(p, om, W, Qs)
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, paw_Q=paw_Q)
        chi = b.rpa_chi0(ctx, 1, om)
        E, dC, dP, dchi = _grad(ctx, p, om, W, iqs)
    finally:
        b.rpa_destroy(ctx)
    # an i <-> j transposition changes chi0 by 5e-3, E_c by 1.6e-3 and the
    # gradient by 7e-3 (dC) and 0.1 (dP) relative on this case (oracle)
    assert _rel(chi, o.chi0(p, 1, om, Qs[1])) < (1e-11 if precision == "fp64" else 1e-4)
    assert abs(E - Er) < tol * abs(Er)
    for s in range(len(p.sets)):
        assert _rel(dC[s], gC[s]) < tol, ("dC", s)
        assert _rel(dP[s], gP[s]) < tol, ("dP", s)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-5), ("bf16x2", 1e-4), ("bf16x3", 2e-5)])
def test_backward_matches_oracle_gradient(precision, tol):
    p = _problem()
    om, W = o.frequency_grid(p.nw)
    Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
    iqs = list(range(len(p.qpoints)))
    Er, gC, gP, gchi = o.energy_grad(p, om, W, Qs)
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


def test_autograd_function_matches_direct_backward():
    import torch
    from paper_1307_8052_gb300.autograd import RpaEngine, RpaEnergy
    p = _problem(tag=99)
    qf = lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm)
    eng = RpaEngine(p, "fp64", paw_Q=qf)
    try:
        Cs = [torch.from_numpy(s.C.copy()).cuda().requires_grad_(True) for s in p.sets]
        Ps = [torch.from_numpy(s.P.copy()).cuda().requires_grad_(True) for s in p.sets]
        E = RpaEnergy.apply(eng, *Cs, *Ps)
        (2.5 * E).backward()
        E_ref, dC, dP, _ = _grad(eng.ctx, p, eng.omega, eng.W, eng.iqs)
        assert abs(E.item() - E_ref) < 1e-12 * abs(E_ref)
        for s in range(len(p.sets)):
            assert _rel(Cs[s].grad.cpu().numpy(), 2.5 * dC[s]) < 1e-12
            assert _rel(Ps[s].grad.cpu().numpy(), 2.5 * dP[s]) < 1e-12
    finally:
        eng.close()


def test_backward_central_differences_fp64():
    """Central differences (h = 1e-6) of the GPU energy along random directions of C and P."""
    p = _problem(tag=98)
    om, W = o.frequency_grid(p.nw)
    iqs = list(range(len(p.qpoints)))
    wq = [qp.weight for qp in p.qpoints]
    ctx = _ctx(p, "fp64")
    try:
        E0, dC, dP, _ = _grad(ctx, p, om, W, iqs)
        rng = np.random.default_rng(17)
        h = 1e-6
        for trial in range(4):
            s = trial % len(p.sets)
            which = "C" if trial < 3 else "P"
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
                vals.append(b.rpa_energy(ctx, iqs, wq, om, W)[0])
            b.rpa_set_orbitals(ctx, s, p.sets[s].k_red, p.sets[s].miller, p.sets[s].C, p.sets[s].eps, p.sets[s].f)
            b.rpa_set_paw(ctx, s, p.paw.nproj, p.sets[s].P)
            fd = (vals[0] - vals[1]) / (2 * h)
            g = dC[s] if which == "C" else dP[s]
            an = float(np.sum(np.conj(g) * d).real)
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (which, fd, an)
    finally:
        b.rpa_destroy(ctx)


def test_config4_geometry_central_differences_fp64():
    """Gradient workload geometry (bulk box, 40^3 grid, all 8 k-points, q = (1/2, 0, 0),
    3 x 13 projectors, NG ~ 1200, 16 frequencies) on a band subset (16 occupied +
    100 empty per set): directional derivatives of the FP64 energy along 32 random
    directions (C and P of every orbital set) against the sixth-order central
    difference [45(E(h) - E(-h)) - 9(E(2h) - E(-2h)) + (E(3h) - E(-3h))] / 60h
    with h = 1e-5.  The unnormalised directions move all 116 x 3119
    coefficients of a set (h |d| ~ 1e-2), where the fourth-order quotient's
    truncation (~1e-8) already exceeds 1e-6 of some derivatives; the
    sixth-order one leaves only its roundoff, bounded in the assertion (at
    this size it, not the gradient, limits the agreement: the oracle's
    analytic gradient agrees with this one to ~1e-13 in these directions).  With all 1216 bands one FP64 energy takes
    ~13 s, so 32 directions (128 energies) are run on the band subset; the
    full-band gradient is checked in the next test."""
    full = syn.config1(nocc=16, nunocc=100)
    iq = [i for i, qp in enumerate(full.qpoints) if np.allclose(qp.q_red, [0.5, 0.0, 0.0])][0]
    p = syn.Problem(full.name, 4, full.cell, full.grid, full.ecut_wf, full.ecut_chi, full.spin_factor,
                    full.nk_bz, full.sets, [full.qpoints[iq]], 16, full.paw)
    om, W = o.frequency_grid(p.nw)
    ctx = _ctx(p, "fp64")
    try:
        E0, dC, dP, dchi = _grad(ctx, p, om, W, [0])
        assert dchi[0].shape[1] > 1000
        rng = np.random.default_rng(4)
        h = 1e-5
        dirs = [(t % len(p.sets), "C" if t % 4 != 3 else "P") for t in range(32)]
        worst = 0.0
        for trial, (s, which) in enumerate(dirs):
            base = getattr(p.sets[s], which).copy()
            d = rng.standard_normal(base.shape) + 1j * rng.standard_normal(base.shape)
            vals = []
            for sign in (1, -1, 2, -2, 3, -3):
                new = base + sign * h * d
                if which == "C":
                    b.rpa_set_orbitals(ctx, s, p.sets[s].k_red, p.sets[s].miller, new, p.sets[s].eps, p.sets[s].f)
                    b.rpa_set_paw(ctx, s, p.paw.nproj, p.sets[s].P)
                else:
                    b.rpa_set_paw(ctx, s, p.paw.nproj, new)
                vals.append(b.rpa_energy(ctx, [0], [p.qpoints[0].weight], om, W)[0])
            b.rpa_set_orbitals(ctx, s, p.sets[s].k_red, p.sets[s].miller, p.sets[s].C, p.sets[s].eps, p.sets[s].f)
            b.rpa_set_paw(ctx, s, p.paw.nproj, p.sets[s].P)
            fd = (45.0 * (vals[0] - vals[1]) - 9.0 * (vals[2] - vals[3]) + (vals[4] - vals[5])) / (60.0 * h)
            g = dC[s] if which == "C" else dP[s]
            an = float(np.sum(np.conj(g) * d).real)
            worst = max(worst, abs(fd - an) / abs(an))
            # 1e-6 relative, above the roundoff of the quotient itself:
            # (45 + 45 + 9 + 9 + 1 + 1) / 60 = 1.83 energy errors over h, an
            # energy error being the FP64 mode's accuracy (1e-13 of E_c at
            # NG ~ 1200: rounding of the log-dets, not a few ulps)
            assert abs(fd - an) <= 1e-6 * abs(an) + 1.83 * 1e-13 * abs(E0) / h, (which, s, fd, an)
        print(f"config-4 geometry, 32 directions: worst relative FD error {worst:.2e}, E {E0:.6f}")
    finally:
        b.rpa_destroy(ctx)


def test_config4_full_bands_central_differences_fp64():
    """The gradient workload at full size (16 + 1200 bands per set, all 8 k,
    q = (1/2, 0, 0), NG ~ 1200, 16 frequencies, 3 x 13 projectors): the FP64
    directional derivative along one random C direction and one random P
    direction (all coefficients of a set) against the sixth-order central
    difference with h = 1e-5.  Each FP64 energy at this size takes ~13 s, so
    two directions (12 energies) are checked here; the 32-direction sweep runs
    on the band subset above, and the mixed modes against this FP64 gradient
    in the next test."""
    full = syn.config1()
    iq = [i for i, qp in enumerate(full.qpoints) if np.allclose(qp.q_red, [0.5, 0.0, 0.0])][0]
    p = syn.Problem(full.name, 4, full.cell, full.grid, full.ecut_wf, full.ecut_chi, full.spin_factor,
                    full.nk_bz, full.sets, [full.qpoints[iq]], 16, full.paw)
    om, W = o.frequency_grid(p.nw)
    ctx = _ctx(p, "fp64")
    try:
        E0, dC, dP, _ = _grad(ctx, p, om, W, [0])
        rng = np.random.default_rng(5)
        h = 1e-5
        for s, which in ((1, "C"), (6, "P")):
            base = getattr(p.sets[s], which).copy()
            d = rng.standard_normal(base.shape) + 1j * rng.standard_normal(base.shape)
            vals = []
            for sign in (1, -1, 2, -2, 3, -3):
                new = base + sign * h * d
                if which == "C":
                    b.rpa_set_orbitals(ctx, s, p.sets[s].k_red, p.sets[s].miller, new, p.sets[s].eps, p.sets[s].f)
                    b.rpa_set_paw(ctx, s, p.paw.nproj, p.sets[s].P)
                else:
                    b.rpa_set_paw(ctx, s, p.paw.nproj, new)
                vals.append(b.rpa_energy(ctx, [0], [p.qpoints[0].weight], om, W)[0])
            b.rpa_set_orbitals(ctx, s, p.sets[s].k_red, p.sets[s].miller, p.sets[s].C, p.sets[s].eps, p.sets[s].f)
            b.rpa_set_paw(ctx, s, p.paw.nproj, p.sets[s].P)
            fd = (45.0 * (vals[0] - vals[1]) - 9.0 * (vals[2] - vals[3]) + (vals[4] - vals[5])) / (60.0 * h)
            g = dC[s] if which == "C" else dP[s]
            an = float(np.sum(np.conj(g) * d).real)
            print(f"config-4 full bands, {which} of set {s}: analytic {an:.10e}, FD {fd:.10e}, "
                  f"rel {abs(fd - an) / abs(an):.2e}")
            # the bound of the band-subset test: 1e-6 plus the quotient's roundoff
            assert abs(fd - an) <= 1e-6 * abs(an) + 1.83 * 1e-13 * abs(E0) / h, (which, s, fd, an)
    finally:
        b.rpa_destroy(ctx)


def test_config4_full_bands_mixed_against_fp64_gradient():
    """The gradient workload at full size (16 + 1200 bands per set, all 8 k, q =
    (1/2, 0, 0), NG ~ 1200, 16 frequencies, 3 x 13 projectors): dE/dC, dE/dP and
    dE/dchi0 of the FP32 and split-bfloat16 (bf16x2) modes against the FP64
    mode's gradient (itself checked against central differences and the
    oracle), errors relative to the largest entry, with dE/dchi0 formed in FP64
    (RPA_TUNE_GAMMA = 0), on the FP32 pipe (1) and in float-float (2, the
    default).  Measured on a GB300: FP32 mode 4.3e-7 / 3.2e-7 / 5.8e-8 (dC / dP
    / dchi), bf16x2 2.9e-6 / 5.5e-7 / 2.2e-7 with the FP64 and the float-float
    form alike; with the FP32 form 3e-4 / 4e-4 / 1.2e-5.  The float-float
    gradient must also agree with the FP64-form gradient of the same mode far
    below those errors."""
    full = syn.config1()
    iq = [i for i, qp in enumerate(full.qpoints) if np.allclose(qp.q_red, [0.5, 0.0, 0.0])][0]
    p = syn.Problem(full.name, 4, full.cell, full.grid, full.ecut_wf, full.ecut_chi, full.spin_factor,
                    full.nk_bz, full.sets, [full.qpoints[iq]], 16, full.paw)
    om, W = o.frequency_grid(p.nw)
    res = {}
    for precision, g32 in (("fp64", 0), ("fp32", 0), ("bf16x2", 0), ("bf16x2", 1), ("bf16x2", 2)):
        ctx = _ctx(p, precision)
        try:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_GAMMA, g32)
            res[(precision, g32)] = _grad(ctx, p, om, W, [0])
        finally:
            b.rpa_destroy(ctx)
    E64, dC64, dP64, dchi64 = res[("fp64", 0)]
    bounds = {("fp32", 0): (1e-6, 2e-6, 2e-6, 1e-6), ("bf16x2", 0): (1e-6, 1e-5, 2e-6, 1e-6),
              ("bf16x2", 1): (1e-6, 1e-3, 1e-3, 5e-5), ("bf16x2", 2): (1e-6, 1e-5, 2e-6, 1e-6)}
    for key, (E, dC, dP, dchi) in res.items():
        if key[0] == "fp64":
            continue
        eE = abs(E - E64) / abs(E64)
        eC = max(_rel(dC[s], dC64[s]) for s in range(len(p.sets)))
        eP = max(_rel(dP[s], dP64[s]) for s in range(len(p.sets)))
        ech = _rel(dchi[0], dchi64[0])
        print(f"config-4 full bands {key[0]} (dE/dchi0 {['FP64', 'FP32', 'float-float'][key[1]]}) vs fp64: "
              f"E {eE:.2e}, dC {eC:.2e}, dP {eP:.2e}, dchi {ech:.2e}")
        bE, bC, bP, bch = bounds[key]
        assert eE <= bE and eC <= bC and eP <= bP and ech <= bch, (key, eE, eC, eP, ech)
    # float-float against FP64 products, same mode: only the Gamma products
    # differ; dE/dchi0 itself to ~2^-44, dE/dC and dE/dP through the FP32
    # rounding of Gamma that feeds the N-bar product (a last-bit flip here and
    # there)
    _, dCf, dPf, dchif = res[("bf16x2", 2)]
    _, dCd, dPd, dchid = res[("bf16x2", 0)]
    ech = _rel(dchif[0], dchid[0])
    eCP = max(max(_rel(dCf[s], dCd[s]) for s in range(len(p.sets))),
              max(_rel(dPf[s], dPd[s]) for s in range(len(p.sets))))
    print(f"config-4 full bands bf16x2, float-float vs FP64 products: dchi {ech:.2e}, dC/dP {eCP:.2e}")
    # measured 6e-8 and 1.2e-7 on two transform grids of the same workload
    assert ech <= 1e-10 and eCP <= 5e-7, (ech, eCP)
