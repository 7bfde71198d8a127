"""Plain CPU FP64 oracle for the RPA response function and correlation energy.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module; the GPU
library never calls it and shares no code with it.

Every function follows the paper (Yan, Li, O'Grady, "GPU acceleration of the
random phase approximation in the PAW method") in the most literal form that
still finishes in seconds on small cases:

* pair densities by the direct plane-wave sum that Eq. 4 defines (no FFT),
* the PAW augmentation term of Eq. 6 evaluated as the outer product of step 8
  and the contraction of step 9 of Table 1 (not factorised),
* chi0 of Eq. 3 by an explicit sum over k-points and band pairs with the
  time-reversal-combined real weight (reading of Eq. 3 / Eq. 16, below),
* the correlation energy of Eqs. 1-2 from the FP64 eigenvalues of
  v^1/2 chi0 v^1/2 (``numpy.linalg.eigvalsh`` serves as the eigen step),
* the analytic gradient of E_c with respect to chi0, the pair densities, the
  projections P and the plane-wave coefficients C.

Readings of the paper that the oracle fixes (all listed in the design notes):

* Eq. 3 carries 2/Omega and a plain sum over BZ k-points; the oracle uses the
  BZ average s/(Omega N_k) with the spin factor s = 2 for spin-paired runs.
* Eq. 3 with the literal complex factor (f-f')/(i w + e - e') is Hermitian only
  after adding the time-reversed partner; pairs (n at k, m at k+q) with
  f_n > f_m are summed once with the real weight
  (f_n - f_m) * 2 (e_n - e_m) / (w^2 + (e_n - e_m)^2).
* The Gauss-Legendre nodes of Sec. 2.1 are mapped to [0, inf) by
  w = w0 (1+x)/(1-x); the nodes are an input of the energy.
* At q = 0 the G = 0 element of the Coulomb kernel is set to zero, unless the
  optical limit is requested: then the G = 0 pair density is the q -> 0 limit
  of Eq. 12 per unit |q| along a direction q^, -i q^.<psi_n|grad|psi_m> /
  (e_m - e_n), with the gradient of Eq. 13 (plane-wave part evaluated exactly
  in the plane-wave basis, PAW part from the input matrices q^.Q_grad of
  Eq. 14), and v_0 = 4 pi (the |q|^2 of v and of |n(0)|^2 cancel).
* The plane-wave normalisation is sum_Q |C(Q)|^2 = 1, so the pair density is
  n(G) = sum_Q conj(C_nk(Q)) C_m,k+q(Q+G) and n_nn(0) = 1 at q = 0.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


# ---------------------------------------------------------------------------
# lattice helpers (Sec. 2.1: plane-wave basis and cutoffs)
# ---------------------------------------------------------------------------

def reciprocal(cell) -> np.ndarray:
    """Reciprocal lattice rows b_i, a_i . b_j = 2 pi delta_ij."""
    return TWO_PI * np.linalg.inv(np.asarray(cell, dtype=np.float64)).T


def g_sphere(cell, q_red, ecut: float) -> np.ndarray:
    """Response basis {G : |q+G|^2 / 2 <= E_cut} (Sec. 2.1), Miller indices in
    lexicographic order (first index slowest), int64 array (NG, 3)."""
    B = reciprocal(cell)
    q = np.asarray(q_red, dtype=np.float64)
    rmax = np.sqrt(2.0 * ecut)
    inv = np.linalg.inv(B)
    ext = [int(np.ceil(rmax * np.linalg.norm(inv[:, i]))) + 2 for i in range(3)]
    out = []
    for g1 in range(-ext[0], ext[0] + 1):
        for g2 in range(-ext[1], ext[1] + 1):
            for g3 in range(-ext[2], ext[2] + 1):
                v = (np.array([g1, g2, g3], dtype=np.float64) + q) @ B
                if 0.5 * float(v @ v) <= ecut:
                    out.append((g1, g2, g3))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def coulomb(cell, q_red, gmiller, optical: bool = False) -> np.ndarray:
    """v_G(q) = 4 pi / |q+G|^2 (Sec. 2.2, text after Eq. 11); zero where q+G = 0,
    or 4 pi there in the optical limit (v_0 |n_0|^2 with both |q|^2 factored out)."""
    B = reciprocal(cell)
    qg = np.asarray(gmiller, dtype=np.float64) + np.asarray(q_red, dtype=np.float64)
    c = qg @ B
    q2 = np.einsum("ij,ij->i", c, c)
    v = np.zeros(len(q2))
    nz = np.any(qg != 0.0, axis=1)
    v[nz] = 4.0 * np.pi / q2[nz]
    if optical:
        v[~nz] = 4.0 * np.pi
    return v


# ---------------------------------------------------------------------------
# frequency quadrature (Sec. 2.1: 16 Gauss-Legendre points)
# ---------------------------------------------------------------------------

def gauss_legendre(n: int):
    """Nodes and weights of n-point Gauss-Legendre quadrature on [-1, 1].

    Newton iteration on P_n(x) with the three-term Legendre recurrence; the
    weight is 2 / ((1 - x^2) P_n'(x)^2) (textbook form)."""
    x = np.cos(np.pi * (np.arange(1, n + 1) - 0.25) / (n + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def frequency_grid(n: int, omega0: float = 1.0):
    """Map GL nodes to [0, inf): w = w0 (1+x)/(1-x), dw = 2 w0 / (1-x)^2 dx."""
    x, wx = gauss_legendre(n)
    omega = omega0 * (1.0 + x) / (1.0 - x)
    W = wx * 2.0 * omega0 / (1.0 - x) ** 2
    return omega, W


# ---------------------------------------------------------------------------
# pair densities (Eq. 4 and Eq. 6; Table 1 steps 5-9)
# ---------------------------------------------------------------------------

def _index_box(miller: np.ndarray):
    lo = miller.min(0)
    hi = miller.max(0)
    box = -np.ones(tuple(hi - lo + 1), dtype=np.int64)
    box[tuple((miller - lo).T)] = np.arange(len(miller))
    return box, lo, hi


def pair_density(Ck, millk, Ckp, millkp, gmiller, G0, nsel, msel) -> np.ndarray:
    """Pseudo pair density of Eq. 4 by the direct plane-wave sum.

    n~_nm(G) = <psi_nk| e^{-i(q+G).r} |psi_m,k+q> = sum_Q conj(C_nk(Q)) C_m,k+q(Q+G),
    with k+q = k' + G0 so that C_m,k+q(Q) = C_m,k'(Q+G0).  Returns an array
    (NG, len(nsel), len(msel)) complex128."""
    Ck = np.asarray(Ck)[nsel]
    Ckp = np.asarray(Ckp)[msel]
    millk = np.asarray(millk, dtype=np.int64)
    millkp = np.asarray(millkp, dtype=np.int64)
    box, lo, hi = _index_box(millkp)
    out = np.zeros((len(gmiller), Ck.shape[0], Ckp.shape[0]), dtype=np.complex128)
    for ig, G in enumerate(np.asarray(gmiller, dtype=np.int64)):
        tgt = millk + G + np.asarray(G0, dtype=np.int64)
        inside = np.all((tgt >= lo) & (tgt <= hi), axis=1)
        pos = -np.ones(len(tgt), dtype=np.int64)
        pos[inside] = box[tuple((tgt[inside] - lo).T)]
        ok = pos >= 0
        out[ig] = np.conj(Ck[:, ok]) @ Ckp[:, pos[ok]].T
    return out


def paw_term(Pn, Pm, Qflat, nproj, ng: int) -> np.ndarray:
    """Augmentation of Eq. 6: sum_a sum_ij conj(P_ni) P_mj Q^a_ij(q+G).

    Evaluated as Table 1 step 8 (outer product P(a,p) = conj(P(a,i)) x P(a,j))
    followed by step 9 (sum over a and p against Q(a,p,G)).  Returns
    (ng, len(Pn), len(Pm))."""
    out = np.zeros((ng, Pn.shape[0], Pm.shape[0]), dtype=np.complex128)
    off = 0
    qoff = 0
    for ni in np.asarray(nproj, dtype=np.int64):
        ni = int(ni)
        Pa_n = Pn[:, off:off + ni]
        Pa_m = Pm[:, off:off + ni]
        Qa = Qflat[qoff:qoff + ni * ni * ng].reshape(ni * ni, ng)
        outer = np.einsum("ni,mj->nmij", np.conj(Pa_n), Pa_m).reshape(Pn.shape[0], Pm.shape[0], ni * ni)
        out += np.einsum("nmp,pg->gnm", outer, Qa)
        off += ni
        qoff += ni * ni * ng
    return out


def pair_weights(eps_n, f_n, eps_m, f_m, omega, spin_factor, volume, nk) -> np.ndarray:
    """Real time-reversal-combined weight of Eq. 3 / Eq. 16 for pairs with f_n > f_m:

    w_nm(w) = s/(Omega N_k) (f_n - f_m) 2 (e_n - e_m) / (w^2 + (e_n - e_m)^2);
    zero for f_n <= f_m.  Shape (len(eps_n), len(eps_m), len(omega))."""
    d = np.asarray(eps_n)[:, None] - np.asarray(eps_m)[None, :]
    df = np.asarray(f_n)[:, None] - np.asarray(f_m)[None, :]
    df = np.where(df > 0.0, df, 0.0)
    om = np.asarray(omega, dtype=np.float64)
    pref = spin_factor / (volume * nk)
    return pref * df[:, :, None] * 2.0 * d[:, :, None] / (om[None, None, :] ** 2 + d[:, :, None] ** 2)


def _selection(f_k, f_kp):
    nsel = np.nonzero(np.asarray(f_k) > 0.0)[0]
    msel = np.nonzero(np.asarray(f_kp) < 1.0)[0]
    return nsel, msel


# ---------------------------------------------------------------------------
# IBZ -> BZ symmetry (Eq. 9; Table 1 steps 4 and 7)
# ---------------------------------------------------------------------------
def rotate_set(oset, M, time_reversal=False, paw_nproj=None, atom_map=None, D=None, tau=None):
    """Orbital set at k' = M k from the set at k (Eq. 9: psi'(r) = psi(T^-1 (r - tau))).

    In the plane-wave basis the rotated orbital has the coefficients
    C'(M Q) = C(Q) exp(-2 pi i (M (k+Q)).tau) on the rotated reciprocal vectors,
    with M the integer matrix of the operation on reduced reciprocal
    coordinates and tau the fractional translation in reduced real-space
    coordinates (zero by default).  Time reversal adds psi -> conj(psi):
    k', Q' -> -k', -Q' and C' -> conj(C').  Projections (step 7):
    P'[n, a, i] = sum_j D[a][i, j] P[n, atom_map[a], j] (conjugated under time
    reversal); D and atom_map describe the projectors and are inputs."""
    import dataclasses
    M = np.asarray(M, dtype=np.int64).reshape(3, 3)
    sg = -1 if time_reversal else 1
    kr = M @ np.asarray(oset.k_red, dtype=np.float64)
    Qr = np.asarray(oset.miller, dtype=np.int64) @ M.T
    k = sg * kr
    mil = (sg * Qr).astype(np.int32)
    C = np.array(oset.C, copy=True)
    if tau is not None:
        C = C * np.exp(-2j * np.pi * ((kr[None, :] + Qr) @ np.asarray(tau, dtype=np.float64)))[None, :]
    if time_reversal:
        C = np.conj(C)
    P = None
    if oset.P is not None and paw_nproj is not None:
        off = np.concatenate([[0], np.cumsum(paw_nproj)])
        P = np.zeros_like(oset.P)
        for a, ni in enumerate(paw_nproj):
            src = atom_map[a]
            P[:, off[a]:off[a] + ni] = oset.P[:, off[src]:off[src] + paw_nproj[src]] @ np.asarray(D[a]).T
        if time_reversal:
            P = np.conj(P)
    return dataclasses.replace(oset, k_red=k, miller=mil, C=C, P=P)


# ---------------------------------------------------------------------------
# optical limit q -> 0 (Eqs. 12-14)
# ---------------------------------------------------------------------------
def nabla_matrix(oset, cell, qdir, nsel, msel, paw_nproj=None, Qnabla=None) -> np.ndarray:
    """q^.<psi_n|grad|psi_m> of Eq. 13 for n in nsel, m in msel of one orbital set.

    Plane-wave part: <psi_n|grad|psi_m> = i sum_Q conj(C_n(Q)) (k+Q) C_m(Q) for
    psi = Omega^-1/2 sum_Q C(Q) e^{i(k+Q).r} (exact in the basis).  PAW part:
    sum_a sum_ij conj(P_ni) P_mj q^.Q_grad^a_ij, with ``Qnabla[a]`` shaped
    (3, ni, ni) (Eq. 14's matrices, an input).  ``qdir`` is normalised here."""
    qhat = np.asarray(qdir, dtype=np.float64)
    qhat = qhat / np.linalg.norm(qhat)
    B = reciprocal(cell)
    kQ = (np.asarray(oset.k_red, dtype=np.float64)[None, :] + np.asarray(oset.miller, dtype=np.float64)) @ B
    s = kQ @ qhat
    C = np.asarray(oset.C)
    D = 1j * (np.conj(C[nsel]) * s[None, :]) @ C[msel].T
    if paw_nproj is not None and Qnabla is not None and len(paw_nproj):
        P = np.asarray(oset.P)
        off = 0
        for a, ni in enumerate(paw_nproj):
            Qa = np.einsum("d,dij->ij", qhat, np.asarray(Qnabla[a]))
            D = D + np.conj(P[nsel][:, off:off + ni]) @ Qa @ P[msel][:, off:off + ni].T
            off += ni
    return D


def optical_head(D, eps_n, eps_m) -> np.ndarray:
    """n_{q->0}(G = 0) per unit |q| (Eq. 12): -i q^.<psi_n|grad|psi_m> / (e_m - e_n)."""
    return -1j * D / (np.asarray(eps_m)[None, :] - np.asarray(eps_n)[:, None])


def pair_block(sets, paw_nproj, Qflat, gmiller, ik, ikp, G0):
    """Full pair density n_nm(G) (pseudo part + PAW term) for one (k, k+q) block."""
    sk, skp = sets[ik], sets[ikp]
    nsel, msel = _selection(sk.f, skp.f)
    n = pair_density(sk.C, sk.miller, skp.C, skp.miller, gmiller, G0, nsel, msel)
    if paw_nproj is not None and Qflat is not None and len(paw_nproj):
        n = n + paw_term(sk.P[nsel], skp.P[msel], Qflat, paw_nproj, len(gmiller))
    return n, nsel, msel


# ---------------------------------------------------------------------------
# chi0 (Eq. 3 / Eqs. 15-17: explicit sum over k and band pairs)
# ---------------------------------------------------------------------------

def chi0(problem, iq: int, omega, Qflat=None, pair_filter=None, optical=None) -> np.ndarray:
    """chi0_GG'(q, i w_j) = sum_k sum_{f_n > f_m} w_nm(w_j) n_nm(G) conj(n_nm(G')).

    ``problem`` is any object with the attributes of ``synthetic.Problem``.
    ``pair_filter(ik, nsel, msel) -> (nsel', msel')`` restricts the band
    pairs (used for partial sums).  ``optical = (qdir, Qnabla)`` replaces the
    G = 0 pair densities of a q = 0 point by the optical limit of Eq. 12
    (``Qnabla`` per atom (3, ni, ni), or None without PAW).  Returns
    (nw, NG, NG) complex128."""
    qp = problem.qpoints[iq]
    gm = g_sphere(problem.cell, qp.q_red, problem.ecut_chi)
    ng = len(gm)
    omega = np.asarray(omega, dtype=np.float64)
    chi = np.zeros((len(omega), ng, ng), dtype=np.complex128)
    nproj = problem.paw.nproj if problem.paw is not None else None
    for t in range(len(qp.k_of)):
        ik, ikp, G0 = int(qp.k_of[t]), int(qp.kq_of[t]), qp.G0[t]
        n, nsel, msel = pair_block(problem.sets, nproj, Qflat, gm, ik, ikp, G0)
        if optical is not None:
            if np.any(np.asarray(qp.q_red) != 0) or ik != ikp or np.any(np.asarray(G0) != 0):
                raise ValueError("the optical limit needs q = 0 and k -> k transitions")
            ig0 = int(np.flatnonzero(np.all(np.asarray(gm) == 0, axis=1))[0])
            sk = problem.sets[ik]
            D = nabla_matrix(sk, problem.cell, optical[0], nsel, msel, nproj, optical[1])
            n[ig0] = optical_head(D, sk.eps[nsel], sk.eps[msel])
        if pair_filter is not None:
            a, b = pair_filter(t, nsel, msel)
            n = n[:, a][:, :, b]
            nsel, msel = nsel[a], msel[b]
        sk, skp = problem.sets[ik], problem.sets[ikp]
        w = pair_weights(sk.eps[nsel], sk.f[nsel], skp.eps[msel], skp.f[msel], omega,
                         problem.spin_factor, problem.volume, problem.nk_bz)
        N = n.reshape(ng, -1)
        W = w.reshape(-1, len(omega))
        for j in range(len(omega)):
            chi[j] += (N * W[:, j][None, :]) @ N.conj().T
    return chi


def chi0_sampled(problem, iq: int, omega, gidx, Qflat=None, transitions=None) -> np.ndarray:
    """Selected elements chi0_{G_a G_b}(q, i w_j) for G indices ``gidx`` of the
    sphere: Eq. 3 evaluated only at those G (the pair densities are computed at
    those G alone), so full-size problems can be sampled.  ``transitions``
    restricts the k-sum to a subset of the q-point's (k, k+q) transitions.
    Returns (nw, len(gidx), len(gidx))."""
    qp = problem.qpoints[iq]
    gm_all = g_sphere(problem.cell, qp.q_red, problem.ecut_chi)
    ng_all = len(gm_all)
    gidx = np.asarray(gidx, dtype=np.int64)
    gm = gm_all[gidx]
    omega = np.asarray(omega, dtype=np.float64)
    chi = np.zeros((len(omega), len(gidx), len(gidx)), dtype=np.complex128)
    nproj = problem.paw.nproj if problem.paw is not None else None
    Qsub = None
    if Qflat is not None and nproj is not None:
        parts, off = [], 0
        for ni in np.asarray(nproj, dtype=np.int64):
            blk = Qflat[off:off + ni * ni * ng_all].reshape(ni * ni, ng_all)
            parts.append(blk[:, gidx].reshape(-1))
            off += ni * ni * ng_all
        Qsub = np.concatenate(parts)
    ts = range(len(qp.k_of)) if transitions is None else transitions
    for t in ts:
        ik, ikp, G0 = int(qp.k_of[t]), int(qp.kq_of[t]), qp.G0[t]
        n, nsel, msel = pair_block(problem.sets, nproj, Qsub, gm, ik, ikp, G0)
        sk, skp = problem.sets[ik], problem.sets[ikp]
        w = pair_weights(sk.eps[nsel], sk.f[nsel], skp.eps[msel], skp.f[msel], omega,
                         problem.spin_factor, problem.volume, problem.nk_bz)
        N = n.reshape(len(gidx), -1)
        W = w.reshape(-1, len(omega))
        for j in range(len(omega)):
            chi[j] += (N * W[:, j][None, :]) @ N.conj().T
    return chi


# ---------------------------------------------------------------------------
# correlation energy (Eqs. 1-2, Table 1 step 13)
# ---------------------------------------------------------------------------

def ec_terms(chi, v) -> np.ndarray:
    """e(w_j) = Tr ln(1 - v^1/2 chi v^1/2) + Tr v^1/2 chi v^1/2, from FP64 eigenvalues."""
    sv = np.sqrt(np.asarray(v, dtype=np.float64))
    out = np.zeros(chi.shape[0])
    for j in range(chi.shape[0]):
        M = sv[:, None] * chi[j] * sv[None, :]
        M = 0.5 * (M + M.conj().T)
        lam = np.linalg.eigvalsh(M)
        out[j] = float(np.sum(np.log1p(-lam) + lam))
    return out


def epsilon_inv(chi, v) -> np.ndarray:
    """Symmetrised inverse dielectric matrix of the RPA, (1 - v^1/2 chi0 v^1/2)^-1,
    per frequency (the matrix whose log-determinant Eq. 1 integrates)."""
    sv = np.sqrt(np.asarray(v, dtype=np.float64))
    out = np.zeros_like(chi)
    for j in range(chi.shape[0]):
        M = sv[:, None] * chi[j] * sv[None, :]
        out[j] = np.linalg.inv(np.eye(len(sv)) - M)
    return out


def energy(problem, omega, W, Qs=None, iqs=None, optical=None):
    """E_c = sum_q w_q sum_j W_j / (2 pi) e_q(w_j) (Eq. 2 with the IBZ weights of Sec. 2.1).

    ``Qs[iq]`` holds the flattened augmentation functions for q-point iq;
    ``optical[iq] = (qdir, Qnabla)`` switches on the optical limit of a q = 0
    point.  Returns (E_c, terms[nq, nw])."""
    iqs = range(len(problem.qpoints)) if iqs is None else iqs
    terms = []
    E = 0.0
    for iq in iqs:
        qp = problem.qpoints[iq]
        opt = None if optical is None else optical.get(iq)
        chi = chi0(problem, iq, omega, None if Qs is None else Qs[iq], optical=opt)
        gm = g_sphere(problem.cell, qp.q_red, problem.ecut_chi)
        v = coulomb(problem.cell, qp.q_red, gm, optical=opt is not None)
        e = ec_terms(chi, v)
        terms.append(e)
        E += qp.weight * float(np.sum(np.asarray(W) * e)) / TWO_PI
    return E, np.array(terms)


# ---------------------------------------------------------------------------
# gradient (adjoint of Eqs. 1-6)
# ---------------------------------------------------------------------------

def dE_dchi(chi, v, omega_weights, wq) -> np.ndarray:
    """Gradient of E_c with respect to chi0(q, i w_j), PyTorch complex convention
    (dE = Re sum conj(g) dchi): g_j = (w_q W_j / 2 pi) v^1/2 [1 - (1 - M_j)^-1] v^1/2."""
    sv = np.sqrt(np.asarray(v, dtype=np.float64))
    ng = len(sv)
    out = np.zeros_like(chi)
    eye = np.eye(ng)
    for j in range(chi.shape[0]):
        M = sv[:, None] * chi[j] * sv[None, :]
        M = 0.5 * (M + M.conj().T)
        inv = np.linalg.inv(eye - M)
        G = sv[:, None] * (eye - inv) * sv[None, :]
        out[j] = (wq * omega_weights[j] / TWO_PI) * 0.5 * (G + G.conj().T)
    return out


def energy_grad(problem, omega, W, Qs=None, iqs=None, optical=None):
    """E_c and its gradient with respect to every orbital set's C and P.

    ``optical[iq] = (qdir, Qnabla)`` switches on the optical limit of a q = 0
    point as in ``energy``: the G = 0 pair densities are the head of Eq. 12,
    so their adjoint runs through Eq. 13 (the dipole matrix) instead of the
    plane-wave sum and the PAW term.  Returns (E, gC, gP, gchi) with gC[s]
    shaped like sets[s].C, gP[s] like sets[s].P (or None) and gchi[iq] the
    dE/dchi0 array of each q."""
    iqs = list(range(len(problem.qpoints))) if iqs is None else list(iqs)
    sets = problem.sets
    gC = [np.zeros_like(s.C) for s in sets]
    gP = [None if s.P is None else np.zeros_like(s.P) for s in sets]
    gchi = {}
    nproj = problem.paw.nproj if problem.paw is not None else None
    E = 0.0
    for iq in iqs:
        qp = problem.qpoints[iq]
        Qflat = None if Qs is None else Qs[iq]
        gm = g_sphere(problem.cell, qp.q_red, problem.ecut_chi)
        ng = len(gm)
        opt = None if optical is None else optical.get(iq)
        v = coulomb(problem.cell, qp.q_red, gm, optical=opt is not None)
        chi = chi0(problem, iq, omega, Qflat, optical=opt)
        ig0 = -1
        if opt is not None:
            ig0 = int(np.flatnonzero(np.all(np.asarray(gm) == 0, axis=1))[0])
        e = ec_terms(chi, v)
        E += qp.weight * float(np.sum(np.asarray(W) * e)) / TWO_PI
        Gam = dE_dchi(chi, v, np.asarray(W), qp.weight)
        gchi[iq] = Gam
        for t in range(len(qp.k_of)):
            ik, ikp, G0 = int(qp.k_of[t]), int(qp.kq_of[t]), qp.G0[t]
            sk, skp = sets[ik], sets[ikp]
            n, nsel, msel = pair_block(sets, nproj, Qflat, gm, ik, ikp, G0)
            if ig0 >= 0:
                D = nabla_matrix(sk, problem.cell, opt[0], nsel, msel, nproj, opt[1])
                n[ig0] = optical_head(D, sk.eps[nsel], sk.eps[msel])
            w = pair_weights(sk.eps[nsel], sk.f[nsel], skp.eps[msel], skp.f[msel], omega,
                             problem.spin_factor, problem.volume, problem.nk_bz)
            # dE/dn_p = 2 sum_j w_p(w_j) Gamma_j n_p
            nbar = np.zeros_like(n)
            for j in range(len(omega)):
                nbar += 2.0 * np.einsum("gh,hab->gab", Gam[j], n) * w[None, :, :, j]
            if ig0 >= 0:
                # the head replaced the G = 0 pair densities: their adjoint runs
                # through Eq. 12-13 only.  n0 = -i D / (e_m - e_n), so with
                # b = i nbar(0) / (e_m - e_n), dE = Re sum conj(b) dD and
                # D = i sum_Q conj(C_n) s C_m + sum_ij conj(P_ni) Qd_ij P_mj
                dlt = sk.eps[msel][None, :] - sk.eps[nsel][:, None]
                bmat = 1j * nbar[ig0] / dlt
                nbar[ig0] = 0.0
                qhat = np.asarray(opt[0], dtype=np.float64)
                qhat = qhat / np.linalg.norm(qhat)
                kQ = (np.asarray(sk.k_red, dtype=np.float64)[None, :] +
                      np.asarray(sk.miller, dtype=np.float64)) @ reciprocal(problem.cell)
                sv = kQ @ qhat
                # g_{C_m}(Q) += sum_n -i b_nm s(Q) C_n(Q);  g_{C_n}(Q) += sum_m i conj(b_nm) s(Q) C_m(Q)
                gC[ik][msel] += (-1j * bmat.T @ sk.C[nsel]) * sv[None, :]
                gC[ik][nsel] += (1j * np.conj(bmat) @ sk.C[msel]) * sv[None, :]
                if nproj is not None and opt[1] is not None and len(nproj):
                    off = 0
                    for a, ni in enumerate(np.asarray(nproj, dtype=np.int64)):
                        ni = int(ni)
                        Qd = np.einsum("d,dij->ij", qhat, np.asarray(opt[1][a]))
                        cols = np.arange(off, off + ni)
                        Pn = sk.P[nsel][:, off:off + ni]
                        Pm = sk.P[msel][:, off:off + ni]
                        # g_{P_mj} += sum_n b_nm sum_i P_ni conj(Qd_ij)
                        gP[ik][np.ix_(msel, cols)] += bmat.T @ Pn @ np.conj(Qd)
                        # g_{P_ni} += sum_m conj(b_nm) sum_j Qd_ij P_mj
                        gP[ik][np.ix_(nsel, cols)] += np.conj(bmat) @ Pm @ Qd.T
                        off += ni
            # through the pseudo pair density (Eq. 4): explicit adjoint of the plane-wave sum
            box, lo, hi = _index_box(np.asarray(skp.miller, dtype=np.int64))
            millk = np.asarray(sk.miller, dtype=np.int64)
            for ig, G in enumerate(gm):
                tgt = millk + G + np.asarray(G0, dtype=np.int64)
                inside = np.all((tgt >= lo) & (tgt <= hi), axis=1)
                pos = -np.ones(len(tgt), dtype=np.int64)
                pos[inside] = box[tuple((tgt[inside] - lo).T)]
                ok = np.nonzero(pos >= 0)[0]
                nb_g = nbar[ig]                       # (nocc_sel, nunocc_sel)
                # g_{C_n}(Q) += sum_m conj(nbar_nm(G)) C_m,k'(Q+G+G0)
                gC[ik][np.ix_(nsel, ok)] += np.conj(nb_g) @ skp.C[np.ix_(msel, pos[ok])]
                # g_{C_m}(Q') += sum_n nbar_nm(G) C_n,k(Q'-G-G0)
                gC[ikp][np.ix_(msel, pos[ok])] += nb_g.T @ sk.C[np.ix_(nsel, ok)]
            # through the PAW term (Eq. 6)
            if nproj is not None and Qflat is not None and len(nproj):
                off = 0
                qoff = 0
                for ni in np.asarray(nproj, dtype=np.int64):
                    ni = int(ni)
                    Qa = Qflat[qoff:qoff + ni * ni * ng].reshape(ni, ni, ng)
                    Pn = sk.P[nsel, off:off + ni]
                    Pm = skp.P[msel, off:off + ni]
                    # g_{P_ni} += sum_m sum_G conj(nbar_nm(G)) sum_j P_mj Q_ij(G)
                    gP[ik][np.ix_(nsel, np.arange(off, off + ni))] += np.einsum(
                        "gnm,mj,ijg->ni", np.conj(nbar), Pm, Qa)
                    # g_{P_mj} += sum_n sum_G nbar_nm(G) sum_i P_ni conj(Q_ij(G))
                    gP[ikp][np.ix_(msel, np.arange(off, off + ni))] += np.einsum(
                        "gnm,ni,ijg->mj", nbar, Pn, np.conj(Qa))
                    off += ni
                    qoff += ni * ni * ng
    return E, gC, gP, gchi
