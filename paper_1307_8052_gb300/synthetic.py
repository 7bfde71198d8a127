"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *draws* inputs: cells, k/q meshes, plane-wave coefficient
sets (random, damped, orthonormalised), band energies, occupations, PAW
projections P_ni and the augmentation functions Q^a_ij(q+G) of a synthetic
analytic form.  It contains none of the response-function arithmetic
(no pair densities, no chi0, no energies), so both the GPU library and the
CPU oracle can consume the same inputs without sharing method code.

The paper (Sec. 4, Table 5) runs on molecules, bulk oxides and adsorbate
slabs whose DFT ground states and PAW setups are not available here; these
generators stand in for them with the same array shapes:

* ``config0``: tiny cubic cell (a = 10 bohr, 16^3 grid), Gamma plus one
  shifted k-set, q = (0.1, 0, 0), 4 occupied + 60 empty bands, no PAW.
* ``config1``: Li2O-sized cubic box (9 bohr, 40^3 grid), Gamma-centred
  2x2x2 k-mesh, 8 q-points, 16 occupied + 1200 empty bands, 20 Ha
  wavefunction cutoff, 10.5 Ha response cutoff, 3 PAW atoms x 13
  projectors.

Seeds: ``13078052 + 1000*config + 10*kidx + role`` with role 0 = orbitals,
1 = projections P, 2 = augmentation constants c_ij, 3 = atom positions.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 13078052


def seed_of(config: int, kidx: int, role: int) -> int:
    return SEED_BASE + 1000 * config + 10 * kidx + role


def reciprocal_cell(cell: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(cell, dtype=np.float64)).T


def wf_sphere(cell: np.ndarray, k_red, ecut: float) -> np.ndarray:
    """Miller indices Q with |k+Q|^2/2 <= ecut, lexicographic order, int32 [npw,3]."""
    B = reciprocal_cell(cell)
    kc = np.asarray(k_red, dtype=np.float64)
    rmax = np.sqrt(2.0 * ecut)
    # |Q_i + k_i| <= |k+Q| * |column i of B^-1| bounds the box along each Miller axis
    inv = np.linalg.inv(B)
    ext = [int(np.ceil(rmax * np.linalg.norm(inv[:, i]))) + 2 for i in range(3)]
    r = [np.arange(-e, e + 1) for e in ext]
    Q = np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3)
    kq = (Q + kc) @ B
    keep = 0.5 * np.einsum("ij,ij->i", kq, kq) <= ecut
    return np.ascontiguousarray(Q[keep].astype(np.int32))


@dataclasses.dataclass
class OrbitalSet:
    k_red: np.ndarray        # (3,) reduced coordinates
    miller: np.ndarray       # (npw, 3) int32
    C: np.ndarray            # (nbands, npw) complex128, orthonormal rows
    eps: np.ndarray          # (nbands,) Ha
    f: np.ndarray            # (nbands,) occupation per spin channel, in [0, 1]
    P: np.ndarray | None = None   # (nbands, sum nproj) complex128


@dataclasses.dataclass
class QPoint:
    q_red: np.ndarray        # (3,)
    k_of: np.ndarray         # (nk,) index of the orbital set at k
    kq_of: np.ndarray        # (nk,) index of the orbital set k' with k+q = k' + G0
    G0: np.ndarray           # (nk, 3) int32 umklapp vectors
    weight: float            # w_q of the BZ sum


@dataclasses.dataclass
class PawSetup:
    nproj: np.ndarray        # (natoms,) int32
    c: list                  # per atom (ni, ni) real symmetric
    R_frac: np.ndarray       # (natoms, 3) fractional positions


@dataclasses.dataclass
class Problem:
    name: str
    config: int
    cell: np.ndarray
    grid: tuple
    ecut_wf: float
    ecut_chi: float
    spin_factor: float
    nk_bz: int               # N_k of the BZ average
    sets: list               # list[OrbitalSet]
    qpoints: list            # list[QPoint]
    nw: int
    paw: PawSetup | None = None

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.cell)))


def make_orbitals(config: int, kidx: int, cell, k_red, ecut_wf: float,
                  nocc: int, nunocc: int) -> OrbitalSet:
    """Random complex-Gaussian coefficients damped by exp(-|k+Q|^2/8), QR-orthonormalised."""
    rng = np.random.default_rng(seed_of(config, kidx, 0))
    miller = wf_sphere(cell, k_red, ecut_wf)
    npw = miller.shape[0]
    nb = nocc + nunocc
    if nb > npw:
        raise ValueError("more bands than plane waves")
    B = reciprocal_cell(cell)
    kq = (miller + np.asarray(k_red)) @ B
    damp = np.exp(-np.einsum("ij,ij->i", kq, kq) / 8.0)
    A = (rng.standard_normal((npw, nb)) + 1j * rng.standard_normal((npw, nb))) / np.sqrt(2.0)
    A *= damp[:, None]
    Qm, _ = np.linalg.qr(A, mode="reduced")
    C = np.ascontiguousarray(Qm.T)
    eps = np.concatenate([np.sort(rng.uniform(-0.8, -0.05, nocc)),
                          np.sort(rng.uniform(0.05, 3.0, nunocc))])
    f = np.concatenate([np.ones(nocc), np.zeros(nunocc)])
    return OrbitalSet(np.asarray(k_red, dtype=np.float64), miller, C, eps, f)


def make_projections(config: int, kidx: int, nbands: int, nproj_total: int) -> np.ndarray:
    rng = np.random.default_rng(seed_of(config, kidx, 1))
    return 0.1 * (rng.standard_normal((nbands, nproj_total))
                  + 1j * rng.standard_normal((nbands, nproj_total))) / np.sqrt(2.0)


def make_paw_setup(config: int, nproj) -> PawSetup:
    nproj = np.asarray(nproj, dtype=np.int32)
    rng = np.random.default_rng(seed_of(config, 0, 2))
    cs = []
    for ni in nproj:
        a = rng.standard_normal((ni, ni))
        cs.append(0.5 * (a + a.T))
    rngR = np.random.default_rng(seed_of(config, 0, 3))
    R = rngR.uniform(0.0, 1.0, (len(nproj), 3))
    return PawSetup(nproj, cs, R)


def paw_Qnabla(paw: PawSetup, config: int) -> list:
    """Synthetic q -> 0 PAW gradient matrices of Eq. 14, one complex (3, ni, ni)
    block per atom, anti-Hermitian in (i, j) like <phi_i|grad|phi_j> - <phi~_i|grad|phi~_j>."""
    rng = np.random.default_rng(seed_of(config, 0, 3))
    out = []
    for ni in paw.nproj:
        A = 0.2 * (rng.standard_normal((3, ni, ni)) + 1j * rng.standard_normal((3, ni, ni)))
        out.append(A - np.conj(np.transpose(A, (0, 2, 1))))
    return out


def paw_Q(paw: PawSetup, cell, q_red, gmiller) -> np.ndarray:
    """Synthetic augmentation Q^a_ij(q+G) = c_ij exp(-0.3|q+G|^2) exp(-i (q+G).R_a).

    Returned flattened atom after atom, each block (ni, ni, NG), complex128,
    for the G list ``gmiller`` (whatever order the caller uses).
    """
    B = reciprocal_cell(cell)
    qG = (np.asarray(gmiller, dtype=np.float64) + np.asarray(q_red)) @ B
    q2 = np.einsum("ij,ij->i", qG, qG)
    out = []
    for a, ni in enumerate(paw.nproj):
        Rc = paw.R_frac[a] @ np.asarray(cell)
        phase = np.exp(-1j * (qG @ Rc)) * np.exp(-0.3 * q2)
        out.append((paw.c[a][:, :, None] * phase[None, None, :]).reshape(-1))
    return np.ascontiguousarray(np.concatenate(out)) if out else np.zeros(0, np.complex128)


def mesh_qpoints(kmesh_red: list, q_list: list) -> list:
    """For every q, pair each mesh k with k' = (k+q) mod 1 and G0 = floor(k+q)."""
    karr = np.asarray(kmesh_red, dtype=np.float64)
    out = []
    for q in q_list:
        q = np.asarray(q, dtype=np.float64)
        k_of, kq_of, G0 = [], [], []
        for i, k in enumerate(karr):
            kq = k + q
            g0 = np.floor(kq + 1e-9)
            red = kq - g0
            j = int(np.argmin(np.abs(karr - red).sum(1)))
            if np.abs(karr[j] - red).sum() > 1e-9:
                raise ValueError("k+q not on the mesh")
            k_of.append(i)
            kq_of.append(j)
            G0.append(g0.astype(np.int32))
        out.append(QPoint(q, np.array(k_of, np.int32), np.array(kq_of, np.int32),
                          np.array(G0, np.int32).reshape(-1, 3), 1.0 / len(q_list)))
    return out


def config0() -> Problem:
    a = 10.0
    cell = np.eye(3) * a
    q = np.array([0.1, 0.0, 0.0])
    sets = [make_orbitals(0, 0, cell, [0.0, 0.0, 0.0], 5.0, 4, 60),
            make_orbitals(0, 1, cell, q, 5.0, 4, 60)]
    qp = QPoint(q, np.array([0], np.int32), np.array([1], np.int32),
                np.zeros((1, 3), np.int32), 1.0)
    return Problem("config0-tiny-cubic", 0, cell, (16, 16, 16), 5.0, 2.0, 2.0, 1,
                   sets, [qp], 8, None)


def config1(nocc: int = 16, nunocc: int = 1200, with_paw: bool = True) -> Problem:
    a = 9.0
    cell = np.eye(3) * a
    kmesh = [np.array(x, dtype=np.float64) * 0.5 for x in np.ndindex(2, 2, 2)]
    sets = [make_orbitals(1, i, cell, k, 20.0, nocc, nunocc) for i, k in enumerate(kmesh)]
    paw = None
    if with_paw:
        paw = make_paw_setup(1, [13, 13, 13])
        for i, s in enumerate(sets):
            s.P = make_projections(1, i, s.C.shape[0], int(paw.nproj.sum()))
    qps = mesh_qpoints(kmesh, kmesh)
    return Problem("config1-bulk-9bohr-40^3", 1, cell, (40, 40, 40), 20.0, 10.5, 2.0, 8,
                   sets, qps, 16, paw)


def config2(nocc: int = 120, nunocc: int = 3000, kidx=None, with_paw: bool = True) -> Problem:
    """Surface slab: 9.4 x 8.1 x 40 bohr cell, 48 x 40 x 200 grid, 20 Ha orbitals
    (13039 plane waves at Gamma), Gamma-centred 4 x 2 x 1 in-plane k-mesh whose
    8 points are also the 8 q-points (k+q stays on the mesh, with umklapp),
    7.55 Ha response cutoff (NG 2988-3058), 16 frequencies, 16 PAW atoms x 18
    projectors + 2 x 8.  ``kidx`` keeps a subset of the k-points (the q-points
    then pair only kept k with kept k+q)."""
    cell = np.diag([9.4, 8.1, 40.0])
    kmesh = [np.array([i / 4.0, j / 2.0, 0.0]) for i in range(4) for j in range(2)]
    keep = list(range(len(kmesh))) if kidx is None else list(kidx)
    sets = [make_orbitals(2, i, cell, kmesh[i], 20.0, nocc, nunocc) for i in keep]
    paw = None
    if with_paw:
        paw = make_paw_setup(2, [18] * 16 + [8] * 2)
        for s_, i in zip(sets, keep):
            s_.P = make_projections(2, i, s_.C.shape[0], int(paw.nproj.sum()))
    qps = []
    pos = {i: n for n, i in enumerate(keep)}
    for qp in mesh_qpoints(kmesh, kmesh):
        sel = [t for t in range(len(qp.k_of)) if int(qp.k_of[t]) in pos and int(qp.kq_of[t]) in pos]
        if not sel:
            continue
        qps.append(QPoint(qp.q_red, np.array([pos[int(qp.k_of[t])] for t in sel], np.int32),
                          np.array([pos[int(qp.kq_of[t])] for t in sel], np.int32),
                          qp.G0[sel].reshape(-1, 3), qp.weight))
    return Problem("config2-slab-48x40x200", 2, cell, (48, 40, 200), 20.0, 7.55, 2.0, 8,
                   sets, qps, 16, paw)


def spin_metal_problem(config_tag: int = 80, a: float = 6.0, grid=(12, 12, 12), ecut_wf: float = 4.0,
                       ecut_chi: float = 1.5, nb: int = 14, mesh=(2, 1, 1), nproj=(4, 5), nw: int = 8,
                       kT: float = 0.05) -> Problem:
    """Spin-polarised metal: one orbital set per (k, spin) (set 2k + spin),
    Fermi-Dirac occupations f = 1 / (1 + exp((e - mu_s) / kT)) with the chemical
    potential of spin s on band nb/2 - 1 + s of the first k-point, so both
    channels have partially occupied bands, spin factor 1, transitions
    k -> k+q within each spin channel."""
    cell = np.diag([a, a * 1.1, a * 0.9])
    kmesh = [np.array([i / mesh[0], j / mesh[1], l / mesh[2]]) for i in range(mesh[0])
             for j in range(mesh[1]) for l in range(mesh[2])]
    paw = make_paw_setup(config_tag, list(nproj)) if nproj else None
    sets = []
    mu = [None, None]
    for i, k in enumerate(kmesh):
        for sp in (0, 1):
            st = make_orbitals(config_tag, 2 * i + sp, cell, k, ecut_wf, nb // 2, nb - nb // 2)
            if mu[sp] is None:
                mu[sp] = float(st.eps[nb // 2 - 1 + sp])
            st.f = 1.0 / (1.0 + np.exp((st.eps - mu[sp]) / kT))
            if paw is not None:
                st.P = make_projections(config_tag, 2 * i + sp, st.C.shape[0], int(paw.nproj.sum()))
            sets.append(st)
    qps = []
    for qp in mesh_qpoints(kmesh, kmesh):
        k_of = np.concatenate([2 * qp.k_of, 2 * qp.k_of + 1]).astype(np.int32)
        kq_of = np.concatenate([2 * qp.kq_of, 2 * qp.kq_of + 1]).astype(np.int32)
        G0 = np.concatenate([qp.G0, qp.G0]).astype(np.int32)
        qps.append(QPoint(qp.q_red, k_of, kq_of, G0, qp.weight))
    return Problem(f"spin-metal-{config_tag}", config_tag, cell, tuple(grid), ecut_wf, ecut_chi, 1.0,
                   len(kmesh), sets, qps, nw, paw)


def config3_instance(i: int, nw: int = 16, ng_range=(400, 3000), nocc_range=(8, 120)) -> Problem:
    """One (q, cell) instance of the batched workload: the bulk box of config 1
    (9 bohr, 40^3 grid, 20 Ha orbitals), Gamma k-point, q drawn from the
    {0, 1/2}^3 mesh without 0, response basis size NG ~ U[400, 3000] (the
    cutoff is set from the target count), n_occ ~ U[8, 120], n_unocc ~ NG,
    3 PAW atoms x 13 projectors; seeds depend on the instance index.  The
    ranges of NG and n_occ are parameters (inclusive)."""
    tag = 300 + i
    rng = np.random.default_rng(seed_of(tag, 0, 9))
    a = 9.0
    cell = np.eye(3) * a
    mesh = [np.array(x, dtype=np.float64) * 0.5 for x in np.ndindex(2, 2, 2)][1:]
    q = mesh[int(rng.integers(len(mesh)))]
    ng_target = int(rng.integers(ng_range[0], ng_range[1] + 1))
    vol = a ** 3
    ecut_chi = 0.5 * (6.0 * np.pi ** 2 * ng_target / vol) ** (2.0 / 3.0)
    nocc = int(rng.integers(nocc_range[0], nocc_range[1] + 1))
    npw_min = min(len(wf_sphere(cell, [0, 0, 0], 20.0)), len(wf_sphere(cell, q, 20.0)))
    nunocc = int(min(ng_target, npw_min - nocc))
    sets = [make_orbitals(tag, 0, cell, [0.0, 0.0, 0.0], 20.0, nocc, nunocc),
            make_orbitals(tag, 1, cell, q, 20.0, nocc, nunocc)]
    paw = make_paw_setup(tag, [13, 13, 13])
    for k, s in enumerate(sets):
        s.P = make_projections(tag, k, s.C.shape[0], int(paw.nproj.sum()))
    qp = QPoint(q, np.array([0], np.int32), np.array([1], np.int32), np.zeros((1, 3), np.int32), 1.0)
    return Problem(f"batched-{i}", 3, cell, (40, 40, 40), 20.0, float(ecut_chi), 2.0, 1, sets, [qp], nw, paw)


def small_problem(config_tag: int = 90, a: float = 6.0, grid=(12, 12, 12), ecut_wf: float = 4.0,
                  ecut_chi: float = 1.5, nocc: int = 3, nunocc: int = 20, mesh=(2, 1, 1),
                  nproj=(4, 5), nw: int = 8) -> Problem:
    """A small but non-trivial mesh problem (umklapp, several k, PAW) for fast parity tests."""
    cell = np.diag([a, a * 1.1, a * 0.9])
    kmesh = [np.array([i / mesh[0], j / mesh[1], l / mesh[2]]) for i in range(mesh[0])
             for j in range(mesh[1]) for l in range(mesh[2])]
    sets = [make_orbitals(config_tag, i, cell, k, ecut_wf, nocc, nunocc) for i, k in enumerate(kmesh)]
    paw = None
    if nproj:
        paw = make_paw_setup(config_tag, list(nproj))
        for i, s in enumerate(sets):
            s.P = make_projections(config_tag, i, s.C.shape[0], int(paw.nproj.sum()))
    qps = mesh_qpoints(kmesh, kmesh)
    return Problem(f"small-{config_tag}", config_tag, cell, tuple(grid), ecut_wf, ecut_chi, 2.0,
                   len(kmesh), sets, qps, nw, paw)
