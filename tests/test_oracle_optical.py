"""Pins of the oracle's optical limit (Eqs. 12-14) against things that do not
use its formula: the finite-q pair density of eigenstates of a model crystal
Hamiltonian (the limit the formula is the first order of), anti-Hermiticity
of the gradient, plane-wave orbitals, and the PAW term's limits."""
import numpy as np

import oracle as o
from paper_1307_8052_gb300 import synthetic as syn


def _model(k_red, cell, miller, V):
    """Eigenpairs of H = -grad^2/2 + V in the plane-wave basis at k:
    H[Q, Q'] = |k+Q|^2 / 2 delta + V(Q - Q')."""
    B = o.reciprocal(cell)
    kq = (np.asarray(k_red)[None, :] + miller) @ B
    H = np.diag(0.5 * np.einsum("ij,ij->i", kq, kq)).astype(np.complex128)
    for i in range(len(miller)):
        for j in range(len(miller)):
            H[i, j] += V(tuple(miller[i] - miller[j]))
    e, U = np.linalg.eigh(H)
    return e, U.T.copy()  # C[n][Q]


def test_optical_head_is_the_small_q_limit_of_the_pair_density():
    a = 5.0
    cell = np.eye(3) * a
    k = np.array([0.11, 0.23, 0.07])
    miller = syn.wf_sphere(cell, k, 2.5)
    rng = np.random.default_rng(1307)
    pot = {}

    def V(G):
        if G == (0, 0, 0):
            return 0.0
        if G not in pot:
            g2 = float(np.dot(G, G))
            val = 0.35 * np.exp(-0.2 * g2) * (rng.standard_normal() + 1j * rng.standard_normal())
            pot[G] = val
            pot[tuple(-x for x in G)] = np.conj(val)
        return pot[G]

    e, C = _model(k, cell, miller, V)
    assert np.min(np.diff(e[:12])) > 1e-3  # non-degenerate bands in the window
    qhat = np.array([0.3, -0.5, 0.8])
    qhat /= np.linalg.norm(qhat)
    eta = 1e-5
    B = o.reciprocal(cell)
    q_red = (eta * qhat) @ np.linalg.inv(B)
    e2, C2 = _model(k + q_red, cell, miller, V)
    # parallel-transport gauge: <u_m(k)|u_m(k+q)> real and positive
    for m in range(12):
        ov = np.vdot(C[m], C2[m])
        C2[m] *= np.conj(ov) / abs(ov)
    nsel, msel = np.arange(3), np.arange(3, 12)
    n_fd = o.pair_density(C, miller, C2, miller, np.zeros((1, 3), np.int64), np.zeros(3), nsel, msel)[0]
    oset = syn.OrbitalSet(k, miller, C, e, np.r_[np.ones(3), np.zeros(len(e) - 3)], None)
    D = o.nabla_matrix(oset, cell, qhat, nsel, msel)
    head = eta * o.optical_head(D, e[nsel], e[msel])
    assert np.max(np.abs(head)) > 1e-7
    assert np.max(np.abs(n_fd - head)) <= 1e-3 * np.max(np.abs(head))
    # a sign error, a missing i or a dropped 1/(e_m - e_n) would be O(1) wrong
    assert np.max(np.abs(n_fd + head)) > 0.5 * np.max(np.abs(head))


def test_gradient_matrix_is_anti_hermitian_and_plane_waves_are_diagonal():
    cell = np.diag([6.0, 6.6, 5.4])
    s = syn.make_orbitals(5, 0, cell, [0.1, 0.0, 0.3], 3.0, 4, 10)
    nproj = [3, 2]
    rng = np.random.default_rng(7)
    s.P = rng.standard_normal((14, 5)) + 1j * rng.standard_normal((14, 5))
    Qn = []
    for ni in nproj:
        A = rng.standard_normal((3, ni, ni)) + 1j * rng.standard_normal((3, ni, ni))
        Qn.append(A - np.conj(np.transpose(A, (0, 2, 1))))  # anti-Hermitian like <phi|grad|phi>
    allb = np.arange(14)
    D = o.nabla_matrix(s, cell, [1.0, 2.0, -0.5], allb, allb, nproj, Qn)
    assert np.allclose(D, -D.conj().T, atol=1e-13)
    # P = 0 removes the PAW part; scaling qdir does not change the result
    s0 = syn.OrbitalSet(s.k_red, s.miller, s.C, s.eps, s.f, np.zeros_like(s.P))
    D0 = o.nabla_matrix(s0, cell, [2.0, 4.0, -1.0], allb, allb, nproj, Qn)
    Dpw = o.nabla_matrix(s, cell, [1.0, 2.0, -0.5], allb, allb)
    assert np.allclose(D0, Dpw, atol=1e-14)
    # plane-wave orbitals: <psi_n|grad|psi_m> = i (k+Q_n) delta_nm
    miller = s.miller[:5]
    pw = syn.OrbitalSet(s.k_red, miller, np.eye(5, dtype=np.complex128), np.arange(5.0), np.ones(5), None)
    qhat = np.array([0.0, 0.0, 1.0])
    Dp = o.nabla_matrix(pw, cell, qhat, np.arange(5), np.arange(5))
    kq = (np.asarray(s.k_red)[None, :] + miller) @ o.reciprocal(cell)
    assert np.allclose(Dp, np.diag(1j * kq[:, 2]), atol=1e-14)


def test_optical_coulomb_head():
    cell = np.eye(3) * 7.0
    gm = o.g_sphere(cell, [0, 0, 0], 1.0)
    v0 = o.coulomb(cell, [0, 0, 0], gm)
    v1 = o.coulomb(cell, [0, 0, 0], gm, optical=True)
    i0 = int(np.flatnonzero(np.all(gm == 0, axis=1))[0])
    assert v0[i0] == 0.0 and v1[i0] == 4 * np.pi
    assert np.array_equal(np.delete(v0, i0), np.delete(v1, i0))


def test_optical_gradient_matches_central_differences():
    """The gradient through the optical head (adjoint of Eqs. 12-13, plane-wave
    and PAW parts) against central differences of the optical-limit energy,
    in random C and P directions of both orbital sets of a q = 0 point."""
    p = syn.small_problem(config_tag=98, a=5.0, grid=(10, 10, 10), ecut_wf=2.0, ecut_chi=1.2,
                          nocc=2, nunocc=6, mesh=(2, 1, 1), nproj=(2, 3), nw=4)
    iq = 0
    assert np.all(p.qpoints[iq].q_red == 0)
    Qs = {i: syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi))
          for i, qp in enumerate(p.qpoints)}
    opt = {iq: ([0.3, 1.0, -0.4], syn.paw_Qnabla(p.paw, p.config))}
    om, W = o.frequency_grid(4)
    E0, gC, gP, _ = o.energy_grad(p, om, W, Qs, iqs=[iq], optical=opt)
    Eref, _ = o.energy(p, om, W, Qs, iqs=[iq], optical=opt)
    assert abs(E0 - Eref) <= 1e-14 * abs(Eref)
    # the head matters: without the optical limit the energy and gradient differ
    _, gC_plain, _, _ = o.energy_grad(p, om, W, Qs, iqs=[iq])
    assert np.abs(gC[0] - gC_plain[0]).max() > 1e-3 * np.abs(gC[0]).max()
    rng = np.random.default_rng(29)
    h = 1e-6
    for trial in range(8):
        s = trial % len(p.sets)
        which = "C" if trial < 4 else "P"
        base = getattr(p.sets[s], which)
        d = rng.standard_normal(base.shape) + 1j * rng.standard_normal(base.shape)
        setattr(p.sets[s], which, base + h * d)
        Ep, _ = o.energy(p, om, W, Qs, iqs=[iq], optical=opt)
        setattr(p.sets[s], which, base - h * d)
        Em, _ = o.energy(p, om, W, Qs, iqs=[iq], optical=opt)
        setattr(p.sets[s], which, base)
        fd = (Ep - Em) / (2 * h)
        g = gC[s] if which == "C" else gP[s]
        an = float(np.sum(np.conj(g) * d).real)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (which, s, fd, an)
