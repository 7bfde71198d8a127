"""The seeded input generator follows the recipe stated for the workloads:
orthonormal damped plane-wave coefficients on the wavefunction sphere, band
energies in the stated windows, 0/1 occupations, projections of scale 0.1,
augmentation functions of the closed form c_ij exp(-0.3|q+G|^2)
exp(-i(q+G).R_a) with c symmetric, umklapp-consistent q-point meshes, and
bit-identical draws for equal seeds."""
import numpy as np

from paper_1307_8052_gb300 import synthetic as syn


def test_orbitals_follow_the_recipe():
    cell = np.eye(3) * 7.0
    k = [0.5, 0.0, 0.25]
    s = syn.make_orbitals(5, 2, cell, k, 4.0, 3, 20)
    B = syn.reciprocal_cell(cell)
    kq = (s.miller + np.asarray(k)) @ B
    assert np.all(0.5 * np.einsum("ij,ij->i", kq, kq) <= 4.0 + 1e-12)
    # the sphere is complete and has no duplicates (brute force over a box)
    r = np.arange(-8, 9)
    box = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    kb = (box + np.asarray(k)) @ B
    inside = {tuple(m) for m in box[0.5 * np.einsum("ij,ij->i", kb, kb) <= 4.0]}
    assert {tuple(m) for m in s.miller} == inside and len(inside) == len(s.miller)
    assert np.allclose(s.C @ s.C.conj().T, np.eye(23), atol=1e-12)
    assert np.all((s.eps[:3] >= -0.8) & (s.eps[:3] <= -0.05)) and np.all(np.diff(s.eps[:3]) >= 0)
    assert np.all((s.eps[3:] >= 0.05) & (s.eps[3:] <= 3.0)) and np.all(np.diff(s.eps[3:]) >= 0)
    assert np.array_equal(s.f, np.r_[np.ones(3), np.zeros(20)])
    # damping exp(-|k+Q|^2/8): the coefficient weight falls off with |k+Q|
    w = np.sum(np.abs(s.C) ** 2, axis=0)
    k2 = np.einsum("ij,ij->i", kq, kq)
    lo, hi = k2 < np.median(k2), k2 >= np.median(k2)
    assert w[lo].mean() > w[hi].mean()


def test_draws_are_deterministic_and_seeded_per_role():
    cell = np.eye(3) * 7.0
    a = syn.make_orbitals(5, 2, cell, [0, 0, 0], 4.0, 2, 10)
    b = syn.make_orbitals(5, 2, cell, [0, 0, 0], 4.0, 2, 10)
    c = syn.make_orbitals(5, 3, cell, [0, 0, 0], 4.0, 2, 10)
    assert np.array_equal(a.C, b.C) and np.array_equal(a.eps, b.eps)
    assert not np.allclose(a.C, c.C)
    assert syn.seed_of(1, 3, 2) == syn.SEED_BASE + 1000 + 30 + 2
    P = syn.make_projections(5, 2, 40, 9)
    assert P.shape == (40, 9) and 0.08 < np.sqrt(np.mean(np.abs(P) ** 2)) < 0.12
    assert np.array_equal(P, syn.make_projections(5, 2, 40, 9))


def test_augmentation_functions_have_the_closed_form():
    cell = np.diag([6.0, 6.6, 5.4])
    paw = syn.make_paw_setup(7, [3, 4])
    q = np.array([0.5, 0.0, 0.5])
    gm = syn.wf_sphere(cell, q, 1.5)
    Q = syn.paw_Q(paw, cell, q, gm)
    B = syn.reciprocal_cell(cell)
    qG = (gm + q) @ B
    off = 0
    for a, ni in enumerate(paw.nproj):
        blk = Q[off:off + ni * ni * len(gm)].reshape(ni, ni, len(gm))
        off += ni * ni * len(gm)
        c = paw.c[a]
        assert np.allclose(c, c.T)
        R = paw.R_frac[a] @ cell
        want = c[:, :, None] * (np.exp(-0.3 * np.einsum("ij,ij->i", qG, qG)) * np.exp(-1j * qG @ R))[None, None]
        assert np.allclose(blk, want, rtol=1e-14, atol=1e-15)
    assert off == len(Q)


def test_qpoint_meshes_are_umklapp_consistent():
    kmesh = [np.array(x, dtype=np.float64) * 0.5 for x in np.ndindex(2, 2, 2)]
    qps = syn.mesh_qpoints(kmesh, kmesh)
    assert len(qps) == 8 and abs(sum(qp.weight for qp in qps) - 1.0) < 1e-15
    for qp in qps:
        for t in range(len(qp.k_of)):
            k, kp = kmesh[qp.k_of[t]], kmesh[qp.kq_of[t]]
            assert np.allclose(k + qp.q_red, kp + qp.G0[t])
