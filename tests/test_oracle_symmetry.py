"""Pins of the oracle's IBZ -> BZ rotation (Eq. 9; steps 4 and 7) against
things that do not use it: orbitals diagonalised directly at the rotated
k-point of a symmetric model crystal, and group properties of the projector
rotation."""
import dataclasses

import numpy as np

import oracle as o
from paper_1307_8052_gb300 import synthetic as syn


def _model_sets(cell, kpts, V, ecut=2.0, nocc=3, nb=10):
    """Eigenstates of H = -grad^2/2 + V on a shared plane-wave list."""
    B = o.reciprocal(cell)
    miller = syn.wf_sphere(cell, [0, 0, 0], ecut + 0.8)
    out = []
    for k in kpts:
        kq = (np.asarray(k)[None, :] + miller) @ B
        H = np.diag(0.5 * np.einsum("ij,ij->i", kq, kq)).astype(np.complex128)
        for i in range(len(miller)):
            for j in range(len(miller)):
                H[i, j] += V(tuple(miller[i] - miller[j]))
        e, U = np.linalg.eigh(H)
        f = np.r_[np.ones(nocc), np.zeros(nb - nocc)]
        out.append(syn.OrbitalSet(np.asarray(k, float), miller, U.T[:nb].copy(), e[:nb], f, None))
    return out


def _cubic_potential():
    # V(G) invariant under the 90-degree rotation about z and under G -> -G with a real potential
    def V(G):
        if G == (0, 0, 0):
            return 0.0
        g = np.array(G, float)
        return 0.3 * np.exp(-0.3 * g @ g) * (1.0 + 0.2 * np.cos(g[0] * g[1]) + 0.1 * g[2] ** 2)
    return V


def test_rotated_orbitals_give_the_chi0_of_the_rotated_k_point():
    cell = np.eye(3) * 5.0
    V = _cubic_potential()
    k = np.array([0.5, 0.0, 0.0])
    M = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]])  # 90 degrees about z (reduced = Cartesian here)
    kr = M @ k
    direct = _model_sets(cell, [k, kr], V)
    rot = o.rotate_set(direct[0], M)
    assert np.allclose(rot.k_red, kr)
    om, _ = o.frequency_grid(3)
    q = np.zeros(3)

    def chi(sets):
        qp = syn.QPoint(q, np.array([0]), np.array([0]), np.zeros((1, 3), np.int32), 1.0)
        prob = syn.Problem("sym", 0, cell, (20, 20, 20), 2.8, 1.2, 2.0, 1, sets, [qp], 3)
        return o.chi0(prob, 0, om)

    a = chi([rot])
    b = chi([direct[1]])
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    assert np.abs(b).max() > 1e-4
    # time reversal: the set at -k is the conjugate (real potential)
    tr = o.rotate_set(direct[0], np.eye(3, dtype=int), time_reversal=True)
    neg = _model_sets(cell, [-k], V)[0]
    assert np.abs(chi([tr]) - chi([neg])).max() <= 1e-10 * np.abs(b).max()
    # a wrong rotation (transpose) breaks it
    wrong = o.rotate_set(direct[0], M.T)
    assert np.abs(chi([wrong]) - b).max() > 1e-3 * np.abs(b).max()


def _psi(s, x):
    """Orbitals of set s at reduced positions x (npts, 3) by the plane-wave sum
    of Eq. 8 without the Omega^-1/2 factor: (nbands, npts)."""
    kq = np.asarray(s.k_red, float)[None, :] + np.asarray(s.miller, float)
    return np.asarray(s.C) @ np.exp(2j * np.pi * (kq @ x.T))


def test_rotated_set_is_the_transformed_function_in_real_space():
    """Eq. 9 point by point.  With k' = M k on reduced reciprocal coordinates the
    operation {T|tau} maps reduced positions by x -> M^-T x + tau, so the set
    it produces must satisfy psi'(x) = psi(M^T (x - tau)); time reversal
    conjugates that.  Checked on the plane-wave sums of both sets at random
    points, for a unimodular M that is not a rotation of this cell (the
    identity holds for any), a fractional translation and time reversal."""
    s = syn.make_orbitals(6, 0, np.diag([5.0, 5.5, 6.0]), [0.1, 0.25, -0.2], 2.0, 2, 3)
    M = np.array([[1, 1, 0], [0, 1, 0], [0, 1, 1]])
    assert round(np.linalg.det(M)) == 1
    tau = np.array([0.1, -0.35, 0.2])
    x = np.random.default_rng(8).uniform(-1.0, 1.0, (9, 3))
    for tr in (False, True):
        r = o.rotate_set(s, M, time_reversal=tr, tau=tau)
        want = _psi(s, (x - tau) @ M)
        if tr:
            want = np.conj(want)
        assert np.abs(_psi(r, x) - want).max() < 1e-12 * np.abs(want).max()
    # the inversion image psi(-x) is a different function: conjugation matters
    assert np.abs(_psi(s, -x) - np.conj(_psi(s, x))).max() > 1e-2 * np.abs(_psi(s, x)).max()


def test_time_reversal_conjugates_the_pair_densities_with_paw():
    """psi -> conj(psi) maps (k, k+q) to (-k, -k-q), and the full pair density
    of Eqs. 4 and 6 to n'(G; -q) = conj(n(-G; q)): the plane-wave part by the
    relabelling Q -> -Q with conjugated coefficients, the PAW part through
    P -> conj(P) (real projector functions) and Q_ij(-k) = conj(Q_ij(k))
    (real partial waves, as the synthetic Q has)."""
    cell = np.diag([5.0, 5.5, 4.5])
    k, q = np.array([0.1, 0.2, 0.0]), np.array([0.25, 0.0, -0.1])
    nproj = [2, 3]
    paw = syn.make_paw_setup(5, nproj)
    sets = []
    for i, kk in enumerate((k, k + q)):
        s_ = syn.make_orbitals(5, i, cell, kk, 2.0, 2, 4)
        sets.append(dataclasses.replace(s_, P=syn.make_projections(5, i, 6, sum(nproj))))
    eye = [np.eye(n) for n in nproj]
    trs = [o.rotate_set(s_, np.eye(3, dtype=int), True, nproj, [0, 1], eye) for s_ in sets]
    assert np.allclose(trs[0].k_red, -k) and np.allclose(trs[1].k_red, -k - q)
    gm = o.g_sphere(cell, q, 1.5)
    n, _, _ = o.pair_block(sets, paw.nproj, syn.paw_Q(paw, cell, q, gm), gm, 0, 1, [0, 0, 0])
    nt, _, _ = o.pair_block(trs, paw.nproj, syn.paw_Q(paw, cell, -q, -gm), -gm, 0, 1, [0, 0, 0])
    assert np.abs(nt - np.conj(n)).max() <= 1e-13 * np.abs(n).max()
    # the PAW part alone is not invariant: P -> conj(P) is what matches
    assert np.abs(syn.paw_Q(paw, cell, -q, -gm) - np.conj(syn.paw_Q(paw, cell, q, gm))).max() < 1e-14
    assert np.abs(np.imag(sets[0].P)).max() > 1e-3


def test_projector_rotation_composes_and_identity_is_a_no_op():
    s = syn.make_orbitals(4, 0, np.eye(3) * 6.0, [0.1, 0.2, 0.0], 3.0, 3, 5)
    nproj = [3, 3, 2]
    rng = np.random.default_rng(2)
    s = dataclasses.replace(s, P=rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8)))
    eye = [np.eye(n) for n in nproj]
    same = o.rotate_set(s, np.eye(3, dtype=int), False, nproj, [0, 1, 2], eye)
    assert np.array_equal(same.P, s.P) and np.array_equal(same.miller, s.miller)

    def unit(n):
        q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        return q

    D1 = [unit(n) for n in nproj]
    D2 = [unit(n) for n in nproj]
    amap1, amap2 = [1, 0, 2], [1, 0, 2]
    twice = o.rotate_set(o.rotate_set(s, np.eye(3, dtype=int), False, nproj, amap1, D1),
                         np.eye(3, dtype=int), False, nproj, amap2, D2)
    # composition: target a takes source amap1[amap2[a]] with D2[a] D1[amap2[a]]
    comp = [D2[a] @ D1[amap2[a]] for a in range(3)]
    once = o.rotate_set(s, np.eye(3, dtype=int), False, nproj, [amap1[amap2[a]] for a in range(3)], comp)
    assert np.allclose(twice.P, once.P, atol=1e-13)


def test_fractional_translation_multiplies_chi0_by_the_phase():
    """Translating every orbital by tau (operation {I|tau}) gives
    n'(G) = exp(-i (q+G).tau) n(G), hence chi0'_GG' = exp(-i (G-G').tau) chi0_GG'."""
    p = syn.small_problem(config_tag=88, nproj=None)
    tau = np.array([0.25, 0.1, -0.3])
    I3 = np.eye(3, dtype=int)
    moved = dataclasses.replace(p, sets=[o.rotate_set(s_, I3, tau=tau) for s_ in p.sets])
    om, _ = o.frequency_grid(3)
    iq = 1
    gm = o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi)
    a = o.chi0(p, iq, om)
    b = o.chi0(moved, iq, om)
    ph = np.exp(-2j * np.pi * (gm @ tau))
    assert np.abs(b - a * ph[None, :, None] * np.conj(ph)[None, None, :]).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(b - a).max() > 1e-3 * np.abs(a).max()
