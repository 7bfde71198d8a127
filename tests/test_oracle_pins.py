"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, textbook quadrature values, lattice-point counts, brute-force
real-space sums, the literal (complex-weight) form of Eq. 3, the two-level
correlation-energy integral and central finite differences.
"""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- quadrature

def test_gauss_legendre_textbook_values():
    x, w = o.gauss_legendre(2)
    assert np.allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15)
    x, w = o.gauss_legendre(3)
    assert np.allclose(x, [-np.sqrt(0.6), 0.0, np.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)
    # exact for polynomials up to degree 2n-1
    x, w = o.gauss_legendre(16)
    for d in range(0, 32):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    # independent library cross-check
    xr, wr = np.polynomial.legendre.leggauss(16)
    assert np.allclose(x, xr, atol=1e-15) and np.allclose(w, wr, atol=1e-14)


@pytest.mark.parametrize("delta", [0.1, 0.5, 1.0, 3.0])
def test_frequency_map_lorentzian_integral(delta):
    # int_0^inf dw / (w^2 + D^2) = pi / (2 D); the mapped rule converges to it
    errs = []
    for n in (8, 16, 64):
        om, W = o.frequency_grid(n)
        errs.append(abs(np.sum(W / (om ** 2 + delta ** 2)) - np.pi / (2 * delta)) / (np.pi / (2 * delta)))
    assert errs[2] < 1e-9
    assert errs[1] < 2e-3
    om, W = o.frequency_grid(16)
    assert np.all(om > 0) and np.all(W > 0) and np.all(np.diff(om) > 0)
    # the scale omega0 of the map is free: the rule integrates the same
    # Lorentzian for any omega0
    for omega0 in (0.4, 2.5):
        om, W = o.frequency_grid(64, omega0)
        assert abs(np.sum(W / (om ** 2 + delta ** 2)) - np.pi / (2 * delta)) < 1e-8 * np.pi / (2 * delta)


# ---------------------------------------------------------------- G sphere

def test_gsphere_lattice_point_counts():
    # a = 2 pi makes B = identity: |G|^2 is the integer m1^2+m2^2+m3^2;
    # counts of integer points with m.m <= n are 1,7,19,27,33,57,81,81,93
    cell = np.eye(3) * 2 * np.pi
    counts = [len(o.g_sphere(cell, [0, 0, 0], 0.5 * n + 1e-9)) for n in range(9)]
    assert counts == [1, 7, 19, 27, 33, 57, 81, 81, 93]
    g = o.g_sphere(cell, [0, 0, 0], 2.5)
    key = [tuple(r) for r in g]
    assert key == sorted(key)


def test_gsphere_off_gamma():
    """At q = (1/2, 0, 0) of a cell with B = identity, |q+G| = 1/2 for G = 0 and
    G = (-1, 0, 0) only, so a cutoff just above 1/8 holds exactly those two;
    just above 5/8 adds the eight G with |q+G|^2 = 5/4.  Moving q by a lattice
    vector G0 moves the sphere by -G0."""
    cell = np.eye(3) * 2 * np.pi
    q = np.array([0.5, 0.0, 0.0])
    g = o.g_sphere(cell, q, 0.125 * 1.001)
    assert sorted(map(tuple, g)) == [(-1, 0, 0), (0, 0, 0)]
    assert len(o.g_sphere(cell, q, 0.625 * 1.001)) == 10
    tri = np.array([[7.0, 0.0, 0.0], [2.1, 6.4, 0.0], [-1.3, 1.7, 8.2]])
    qt = np.array([0.25, -0.125, 1.0 / 3.0])
    G0 = np.array([1, -2, 1])
    a = o.g_sphere(tri, qt, 3.0)
    b = o.g_sphere(tri, qt + G0, 3.0)
    assert np.array_equal(b, a - G0)


def test_reciprocal_lattice_is_dual_to_the_cell():
    """Plane waves e^{iG.r} of reciprocal lattice vectors are periodic on the
    crystal lattice (G.R a multiple of 2 pi for every lattice vector R), for a
    hexagonal and a triclinic cell whose lattice matrices are not symmetric;
    the hexagonal one has six equal shortest G in its basal plane."""
    hexa = np.array([[4.0, 0.0, 0.0], [-2.0, 2.0 * np.sqrt(3.0), 0.0], [0.0, 0.0, 2.5]])
    tri = np.array([[7.0, 0.0, 0.0], [2.1, 6.4, 0.0], [-1.3, 1.7, 8.2]])
    rng = np.random.default_rng(5)
    for cell in (hexa, tri):
        B = o.reciprocal(cell)
        G = rng.integers(-4, 5, size=(40, 3)) @ B
        R = rng.integers(-4, 5, size=(40, 3)) @ cell
        assert np.abs(np.exp(1j * (G @ R.T)) - 1.0).max() < 1e-11
        # half a lattice vector is not a period of every plane wave
        assert np.abs(np.exp(1j * (G @ (0.5 * R.T))) - 1.0).max() > 1.0
    b1 = 2.0 * np.pi / (4.0 * np.sqrt(3.0) / 2.0)   # |b1| of the hexagonal lattice
    gm = o.g_sphere(hexa, [0, 0, 0], 0.5 * b1 ** 2 * 1.001)
    assert len(gm) == 7
    g2 = np.sum((gm @ o.reciprocal(hexa)) ** 2, 1)
    assert np.allclose(np.sort(g2)[1:], b1 ** 2, rtol=1e-12)


def test_coulomb_on_a_hexagonal_lattice():
    """v_G = 4 pi / |G|^2 depends on |G| only: the six shortest basal G of a
    hexagonal lattice (a = 4, c = 2.5 bohr; |b1| = 4 pi / (a sqrt 3), the
    textbook length) share v = 4 pi / |b1|^2, and v_0 = 0 at q = 0."""
    a = 4.0
    hexa = np.array([[a, 0.0, 0.0], [-a / 2, a * np.sqrt(3.0) / 2, 0.0], [0.0, 0.0, 2.5]])
    b1 = 4.0 * np.pi / (a * np.sqrt(3.0))
    gm = o.g_sphere(hexa, [0, 0, 0], 0.5 * b1 ** 2 * 1.001)
    v = o.coulomb(hexa, [0, 0, 0], gm)
    zero = ~gm.any(axis=1)
    assert zero.sum() == 1 and v[zero][0] == 0.0
    assert np.allclose(v[~zero], 4.0 * np.pi / b1 ** 2, rtol=1e-13) and (~zero).sum() == 6


def test_coulomb_zero_only_at_q_plus_g_zero():
    cell = np.eye(3) * 10.0
    gm = o.g_sphere(cell, [0, 0, 0], 1.0)
    v = o.coulomb(cell, [0, 0, 0], gm)
    i0 = [i for i, g in enumerate(gm) if not g.any()][0]
    assert v[i0] == 0.0 and np.all(np.delete(v, i0) > 0)
    # |G| = 2 pi / 10 for the six nearest vectors: v = 4 pi / (2 pi / 10)^2 = 100 / pi
    six = [i for i, g in enumerate(gm) if np.abs(g).sum() == 1]
    assert np.allclose(v[six], 100.0 / np.pi, rtol=1e-14)


# ---------------------------------------------------------------- pair density

def _tiny_sets(config=91, nb=6, ecut=2.0, a=5.0, k2=(0.5, 0.0, 0.0)):
    cell = np.diag([a, a * 1.2, a * 0.9])
    s0 = syn.make_orbitals(config, 0, cell, [0, 0, 0], ecut, 2, nb - 2)
    s1 = syn.make_orbitals(config, 1, cell, k2, ecut, 2, nb - 2)
    return cell, s0, s1


def test_pair_density_orthonormality_q0():
    cell, s0, _ = _tiny_sets()
    nb = s0.C.shape[0]
    n = o.pair_density(s0.C, s0.miller, s0.C, s0.miller, np.zeros((1, 3), np.int64), [0, 0, 0],
                       np.arange(nb), np.arange(nb))
    assert np.abs(n[0] - np.eye(nb)).max() < 1e-14


def _u_on_grid(C, miller, grid):
    # explicit sum u(j) = sum_Q C(Q) exp(2 pi i Q.j/N), no FFT
    j = np.stack(np.meshgrid(*[np.arange(n) for n in grid], indexing="ij"), -1).reshape(-1, 3)
    ph = np.exp(2j * np.pi * (j / np.array(grid)) @ miller.T.astype(float))  # (Nr, npw)
    return C @ ph.T, j


def test_pair_density_matches_realspace_bruteforce_and_fft():
    cell, s0, s1 = _tiny_sets()
    grid = (12, 14, 11)
    G0 = np.array([1, 0, 0])
    gm = o.g_sphere(cell, [0.5, 0, 0], 1.2)
    nsel, msel = np.array([0, 1]), np.array([2, 3, 5])
    n = o.pair_density(s0.C, s0.miller, s1.C, s1.miller, gm, G0, nsel, msel)
    u0, j = _u_on_grid(s0.C[nsel], s0.miller, grid)
    u1, _ = _u_on_grid(s1.C[msel], s1.miller, grid)
    Nr = np.prod(grid)
    ph = np.exp(-2j * np.pi * (j / np.array(grid)) @ (gm + G0).T.astype(float))  # (Nr, NG)
    for a in range(len(nsel)):
        for b in range(len(msel)):
            prod = np.conj(u0[a]) * u1[b]
            ref = prod @ ph / Nr
            assert np.abs(ref - n[:, a, b]).max() < 1e-14
            f = np.fft.fftn(prod.reshape(grid)) / Nr
            idx = tuple(((gm + G0) % np.array(grid)).T)
            assert np.abs(f[idx] - n[:, a, b]).max() < 1e-14


def test_pair_density_plane_wave_orbitals():
    cell = np.eye(3) * 6.0
    mk = syn.wf_sphere(cell, [0, 0, 0], 1.5).astype(np.int64)
    mkp = syn.wf_sphere(cell, [0.5, 0, 0], 1.5).astype(np.int64)
    Ck = np.eye(len(mk), dtype=complex)[:5]
    Ckp = np.eye(len(mkp), dtype=complex)[3:11]
    gm = o.g_sphere(cell, [0.5, 0, 0], 1.0)
    G0 = np.array([0, 0, 0])
    n = o.pair_density(Ck, mk, Ckp, mkp, gm, G0, np.arange(5), np.arange(8))
    for a in range(5):
        for b in range(8):
            for ig, G in enumerate(gm):
                expect = 1.0 if np.array_equal(mk[a] + G + G0, mkp[3 + b]) else 0.0
                assert n[ig, a, b] == expect


# ---------------------------------------------------------------- PAW term

def test_paw_term_zero_and_constant_q():
    rng = np.random.default_rng(5)
    nproj = np.array([3, 4])
    ng = 7
    Pn = rng.standard_normal((2, 7)) + 1j * rng.standard_normal((2, 7))
    Pm = rng.standard_normal((3, 7)) + 1j * rng.standard_normal((3, 7))
    c = [rng.standard_normal((3, 3)), rng.standard_normal((4, 4))]
    Q = np.concatenate([np.repeat(ca.reshape(-1, 1), ng, 1).reshape(-1) for ca in c]).astype(complex)
    t = o.paw_term(Pn, Pm, Q, nproj, ng)
    # constant Q_ij(G) = c_ij: every G carries sum_a conj(P_n^a) c^a (P_m^a)^T
    expect = (np.conj(Pn[:, :3]) @ c[0] @ Pm[:, :3].T + np.conj(Pn[:, 3:]) @ c[1] @ Pm[:, 3:].T)
    for g in range(ng):
        assert np.abs(t[g] - expect).max() < 1e-13
    assert np.abs(o.paw_term(0 * Pn, Pm, Q, nproj, ng)).max() == 0.0


# ---------------------------------------------------------------- chi0

def test_chi0_lindhard_plane_waves():
    """Plane-wave orbitals with free-electron energies: chi0 is diagonal and equals
    the discrete Lindhard sum over Q occupied at k with Q+G empty at k+q."""
    cell = np.eye(3) * 7.0
    B = o.reciprocal(cell)
    q = np.array([0.25, 0.0, 0.0])
    sets = []
    for i, k in enumerate([np.zeros(3), q]):
        m = syn.wf_sphere(cell, k, 3.0).astype(np.int32)
        e = 0.5 * np.sum(((m + k) @ B) ** 2, 1)
        order = np.argsort(e, kind="stable")
        m, e = m[order], e[order]
        f = (e < 0.45).astype(float)
        sets.append(syn.OrbitalSet(k, m, np.eye(len(m), dtype=complex), e, f))
    qp = syn.QPoint(q, np.array([0]), np.array([1]), np.zeros((1, 3), np.int32), 1.0)
    prob = syn.Problem("lindhard", 0, cell, (24, 24, 24), 3.0, 0.6, 2.0, 1, sets, [qp], 4)
    om, _ = o.frequency_grid(4)
    chi = o.chi0(prob, 0, om)
    gm = o.g_sphere(cell, q, 0.6)
    vol = 343.0
    expect = np.zeros((len(om), len(gm)))
    occ = [(m, e) for m, e, f in zip(sets[0].miller, sets[0].eps, sets[0].f) if f == 1.0]
    emp = {tuple(m): e for m, e, f in zip(sets[1].miller, sets[1].eps, sets[1].f) if f == 0.0}
    for ig, G in enumerate(gm):
        for m, e in occ:
            t = tuple(m + G)
            if t in emp:
                d = e - emp[t]
                # literal Eq. 3 summed over the pair and its time-reversed partner
                lit = (2.0 / vol) * (1.0 / (1j * om + d) + 1.0 / (-1j * om + d))
                expect[:, ig] += lit.real
    assert np.abs(chi - np.einsum("wg,gh->wgh", expect, np.eye(len(gm)))).max() < 1e-15 * max(1, np.abs(expect).max())
    assert np.abs(expect).max() > 1e-4


def test_chi0_hermitian_negative_semidefinite_and_additive():
    p = syn.small_problem()
    om, _ = o.frequency_grid(4)
    Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
    iq = 1
    chi = o.chi0(p, iq, om, Qs[iq])
    for j in range(len(om)):
        c = chi[j]
        assert np.abs(c - c.conj().T).max() <= 1e-15 * np.abs(c).max()
        lam = np.linalg.eigvalsh(c)
        assert lam.max() <= 1e-14 * np.abs(lam).max()
    a = o.chi0(p, iq, om, Qs[iq], pair_filter=lambda t, n, m: (np.arange(len(n)), np.arange(len(m)) % 2 == 0))
    b = o.chi0(p, iq, om, Qs[iq], pair_filter=lambda t, n, m: (np.arange(len(n)), np.arange(len(m)) % 2 == 1))
    assert np.abs(a + b - chi).max() <= 1e-14 * np.abs(chi).max()


def test_chi0_is_a_bz_average():
    """Eq. 3 averages over the BZ mesh, s/(Omega N_k) sum_k: listing every
    transition of a q-point r times on a mesh of r N_k points averages r equal
    terms, so chi0 and E_c do not change."""
    import dataclasses
    p = syn.small_problem(config_tag=87)
    om, W = o.frequency_grid(3)
    iq = 1
    Q = syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi))
    qp = p.qpoints[iq]
    ref = o.chi0(p, iq, om, Q)
    E, _ = o.energy(p, om, W, {iq: Q}, iqs=[iq])
    for r in (2, 3):
        rep = syn.QPoint(qp.q_red, np.tile(qp.k_of, r), np.tile(qp.kq_of, r), np.tile(qp.G0, (r, 1)), qp.weight)
        pr = dataclasses.replace(p, nk_bz=r * p.nk_bz, qpoints=[p.qpoints[0], rep])
        assert np.abs(o.chi0(pr, iq, om, Q) - ref).max() <= 1e-14 * np.abs(ref).max()
        Er, _ = o.energy(pr, om, W, {iq: Q}, iqs=[iq])
        assert abs(Er - E) <= 1e-13 * abs(E)
    assert np.abs(ref).max() > 1e-4


def test_chi0_time_reversal_equals_literal_eq3():
    """Gamma point, q = 0, real orbitals (C(-Q) = conj C(Q)): the oracle's real
    pair weight over f_n > f_m equals Eq. 3 with the complex factor
    (f - f')/(i w + e - e') summed over all ordered band pairs."""
    cell = np.diag([5.0, 5.5, 4.5])
    m = syn.wf_sphere(cell, [0, 0, 0], 2.5).astype(np.int64)
    rng = np.random.default_rng(3)
    idx = {tuple(r): i for i, r in enumerate(m)}
    nb = 8
    A = rng.standard_normal((len(m), nb)) + 1j * rng.standard_normal((len(m), nb))
    for i, r in enumerate(m):   # impose A(-Q) = conj A(Q): real orbitals in real space
        j = idx[tuple(-r)]
        if j < i:
            A[i] = np.conj(A[j])
        elif j == i:
            A[i] = A[i].real
    Qm, _ = np.linalg.qr(A)
    # QR mixes columns with complex coefficients; recombine to real orbitals
    Ur = np.real(Qm) + 0j
    Ui = np.imag(Qm) + 0j
    cand = np.concatenate([Ur, Ui], 1)
    # orthonormalise real-space-real combinations in the real vector space of coefficient pairs
    C = []
    for col in cand.T:
        v = col.copy()
        for c in C:
            v = v - np.vdot(c, v).real * c
        nrm = np.sqrt(np.vdot(v, v).real)
        if nrm > 1e-8:
            C.append(v / nrm)
        if len(C) == nb:
            break
    C = np.array(C)
    assert np.abs(C @ C.conj().T - np.eye(nb)).max() < 1e-12
    eps = np.sort(rng.uniform(-1, 2, nb))
    # two partly occupied bands: the pair (0.4, 0.7) enters once, with f_n > f_m
    f = np.array([1, 1, 0.7, 0.4, 0, 0, 0, 0.0])
    s = syn.OrbitalSet(np.zeros(3), m.astype(np.int32), C, eps, f)
    qp = syn.QPoint(np.zeros(3), np.array([0]), np.array([0]), np.zeros((1, 3), np.int32), 1.0)
    prob = syn.Problem("tr", 0, cell, (16, 16, 16), 2.5, 1.0, 2.0, 1, [s], [qp], 4)
    om, _ = o.frequency_grid(4)
    chi = o.chi0(prob, 0, om)
    gm = o.g_sphere(cell, [0, 0, 0], 1.0)
    n = o.pair_density(C, m, C, m, gm, [0, 0, 0], np.arange(nb), np.arange(nb))
    vol = float(np.prod([5.0, 5.5, 4.5]))
    lit = np.zeros_like(chi)
    for a in range(nb):
        for b in range(nb):
            if a == b:
                continue
            for j, w in enumerate(om):
                A_w = (2.0 / vol) * (f[a] - f[b]) / (1j * w + eps[a] - eps[b])
                lit[j] += A_w * np.outer(n[:, a, b], np.conj(n[:, a, b]))
    assert np.abs(lit - chi).max() < 1e-13 * np.abs(chi).max()


# ---------------------------------------------------------------- correlation energy

def _two_level_problem(q=(0.15, 0.0, 0.0)):
    cell = np.diag([6.0, 6.5, 7.0])
    s0 = syn.make_orbitals(92, 0, cell, [0, 0, 0], 2.0, 1, 1)
    s1 = syn.make_orbitals(92, 1, cell, q, 2.0, 1, 1)
    s0.eps = np.array([-0.3, 0.7])
    s1.eps = np.array([-0.2, 0.45])
    qp = syn.QPoint(np.array(q), np.array([0]), np.array([1]), np.zeros((1, 3), np.int32), 1.0)
    B = o.reciprocal(cell)
    qc = np.array(q) @ B
    ecut = 0.5 * float(qc @ qc) * 1.01
    return syn.Problem("two-level", 0, cell, (12, 12, 12), 2.0, ecut, 2.0, 1, [s0, s1], [qp], 8)


def test_ec_two_level_closed_form():
    """One G-vector and one pair: M(w) = -c/(w^2 + D^2) and
    E = 1/(2pi) int_0^inf [ln(1 + c/(w^2+D^2)) - c/(w^2+D^2)] dw = (sqrt(D^2+c) - D - c/(2D))/2."""
    p = _two_level_problem()
    qp = p.qpoints[0]
    gm = o.g_sphere(p.cell, qp.q_red, p.ecut_chi)
    assert len(gm) == 1 and not gm[0].any()
    n = o.pair_density(p.sets[0].C, p.sets[0].miller, p.sets[1].C, p.sets[1].miller, gm, [0, 0, 0], [0], [1])
    D = p.sets[1].eps[1] - p.sets[0].eps[0]
    qc = qp.q_red @ o.reciprocal(p.cell)
    v = 4 * np.pi / float(qc @ qc)
    c = v * (2.0 / p.volume) * 2.0 * D * abs(n[0, 0, 0]) ** 2
    exact = 0.5 * (np.sqrt(D * D + c) - D - c / (2 * D))
    om, W = o.frequency_grid(96)
    E, terms = o.energy(p, om, W)
    assert exact < 0
    assert abs(E - exact) < 1e-10 * abs(exact)
    assert np.all(terms <= 0)
    # derivative of the closed form with respect to c (analytic gradient path)
    dEdc = 0.5 * (0.5 / np.sqrt(D * D + c) - 0.5 / D)
    gchi = o.dE_dchi(o.chi0(p, 0, om), o.coulomb(p.cell, qp.q_red, gm), W, 1.0)
    # dE/dc = sum_j gchi_j * dchi_j/dc with chi_j = M_j / v = -(c/v)/(w^2 + D^2) / c * c
    dchi_dc = -1.0 / v / (om ** 2 + D * D)
    assert abs(np.sum(gchi[:, 0, 0].real * dchi_dc) - dEdc) < 1e-9 * abs(dEdc)


def test_ec_negative_and_logdet_crosscheck():
    p = syn.small_problem()
    om, W = o.frequency_grid(6)
    Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
    E, terms = o.energy(p, om, W, Qs)
    assert E < 0 and np.all(terms <= 0)
    qp = p.qpoints[0]
    gm = o.g_sphere(p.cell, qp.q_red, p.ecut_chi)
    v = o.coulomb(p.cell, qp.q_red, gm)
    chi = o.chi0(p, 0, om, Qs[0])
    for j in range(len(om)):
        M = np.sqrt(v)[:, None] * chi[j] * np.sqrt(v)[None, :]
        sign, ld = np.linalg.slogdet(np.eye(len(v)) - M)
        assert sign.real > 0
        assert abs(ld + np.trace(M).real - terms[0, j]) < 1e-12 * max(1.0, abs(ld))


# ---------------------------------------------------------------- gradient

def _fd_problem():
    p = syn.small_problem(config_tag=93, a=5.0, grid=(10, 10, 10), ecut_wf=2.5, ecut_chi=1.2,
                          nocc=2, nunocc=6, mesh=(2, 1, 1), nproj=(2, 3), nw=4)
    Qs = [syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) for qp in p.qpoints]
    # the synthetic c_ij are symmetric (real partial waves); a general Q_ij(G)
    # is not, and the adjoint must tell i from j
    rng = np.random.default_rng(17)
    Qs = [Q + 0.05 * (rng.standard_normal(Q.shape) + 1j * rng.standard_normal(Q.shape)) for Q in Qs]
    return p, Qs


def test_gradient_matches_central_differences():
    p, Qs = _fd_problem()
    om, W = o.frequency_grid(4)
    E0, gC, gP, _ = o.energy_grad(p, om, W, Qs)
    rng = np.random.default_rng(11)
    h = 1e-6
    for trial in range(6):
        s = trial % len(p.sets)
        which = "C" if trial < 4 else "P"
        base = getattr(p.sets[s], which)
        d = rng.standard_normal(base.shape) + 1j * rng.standard_normal(base.shape)
        setattr(p.sets[s], which, base + h * d)
        Ep, _ = o.energy(p, om, W, Qs)
        setattr(p.sets[s], which, base - h * d)
        Em, _ = o.energy(p, om, W, Qs)
        setattr(p.sets[s], which, base)
        fd = (Ep - Em) / (2 * h)
        g = gC[s] if which == "C" else gP[s]
        an = float(np.sum(np.conj(g) * d).real)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (which, fd, an)


def test_spin_channels_add_up():
    """Spin polarisation (NEXT-2): chi0 is the sum over spin channels with
    spin factor 1, so two identical channels at s = 1 equal one channel at s = 2,
    and the channels of a polarised metal add up."""
    p = syn.spin_metal_problem(nw=4)
    om, _ = o.frequency_grid(4)
    iq = 1
    qp = p.qpoints[iq]
    Q = syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi))
    nt = len(qp.k_of) // 2
    # partially occupied bands in both channels
    assert any(0.05 < f < 0.95 for s_ in p.sets[0::2] for f in s_.f)
    assert any(0.05 < f < 0.95 for s_ in p.sets[1::2] for f in s_.f)
    full = o.chi0(p, iq, om, Q)
    up = o.chi0(p, iq, om, Q, pair_filter=lambda t, n, m: (np.arange(len(n)) if t < nt else np.arange(0),
                                                            np.arange(len(m))))
    dn = o.chi0(p, iq, om, Q, pair_filter=lambda t, n, m: (np.arange(len(n)) if t >= nt else np.arange(0),
                                                            np.arange(len(m))))
    assert np.abs(up + dn - full).max() <= 1e-14 * np.abs(full).max()
    # identical channels at s = 1 == one channel at s = 2
    import dataclasses
    same = dataclasses.replace(p, sets=[p.sets[2 * (i // 2)] for i in range(len(p.sets))])
    paired = dataclasses.replace(p, spin_factor=2.0, sets=p.sets[0::2], qpoints=[
        syn.QPoint(q.q_red, q.k_of[:len(q.k_of) // 2] // 2, q.kq_of[:len(q.kq_of) // 2] // 2,
                   q.G0[:len(q.G0) // 2], q.weight) for q in p.qpoints])
    a = o.chi0(same, iq, om, Q)
    b = o.chi0(paired, iq, om, Q)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def test_epsilon_inverse_adiabatic_connection():
    """The RPA correlation term from the coupling-constant integral
    e = int_0^1 dlambda tr[((1 - lambda M)^-1 - 1) M] (adiabatic connection, exact
    for the RPA) against the eigenvalue form ln det(1 - M) + tr M of the oracle."""
    p = syn.small_problem(config_tag=89)
    om, _ = o.frequency_grid(3)
    iq = 1
    qp = p.qpoints[iq]
    gm = o.g_sphere(p.cell, qp.q_red, p.ecut_chi)
    Q = syn.paw_Q(p.paw, p.cell, qp.q_red, gm)
    chi = o.chi0(p, iq, om, Q)
    v = o.coulomb(p.cell, qp.q_red, gm)
    e_ref = o.ec_terms(chi, v)
    x, wl = o.gauss_legendre(40)
    lam, wl = 0.5 * (x + 1.0), 0.5 * wl
    sv = np.sqrt(v)
    e = np.zeros(len(om))
    for lm, wgt in zip(lam, wl):
        einv = o.epsilon_inv(lm * chi, v)
        for j in range(len(om)):
            M = sv[:, None] * chi[j] * sv[None, :]
            e[j] -= wgt * np.trace((einv[j] - np.eye(len(v))) @ M).real
    # d/dlambda [ln det(1 - lambda M) + lambda tr M] = -tr[(1-lambda M)^-1 M] + tr M
    # so e = int_0^1 (tr M - tr[(1 - lambda M)^-1 M]) dlambda = -int tr[((1-lM)^-1 - 1) M]
    assert np.allclose(e, e_ref, rtol=1e-9, atol=1e-12 * np.abs(e_ref).max())
    assert np.abs(e_ref).max() > 1e-3
