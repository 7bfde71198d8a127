"""Every plausible mistake planted in the oracle fails at least one of its pins.

Each case edits one spot of the oracle's source (a dropped factor, a flipped
sign, a misplaced conjugate, a transposed operand, a wrong index, offset or
normalisation), loads the edited source as a separate module, and runs the
pin tests against it: those of test_oracle_pins.py, test_oracle_optical.py,
test_oracle_symmetry.py, test_oracle_sampled.py and the printed
Gauss-Legendre table.  At least one must fail.  The oracle module itself is
not touched.  Only pins that do not come from the oracle's own output take
part (the stored config-0 terms, which the oracle wrote, do not).
"""
import inspect
import os
import types

import pytest

import oracle.rpa_oracle as base
import test_golden
import test_oracle_optical
import test_oracle_pins
import test_oracle_sampled
import test_oracle_symmetry

PIN_MODULES = [test_oracle_pins, test_oracle_optical, test_oracle_symmetry, test_oracle_sampled, test_golden]
NOT_PINS = {"test_config0_oracle_reproduces_stored_terms"}
SLOW_LAST = ["test_sampled_bulk_geometry_band_subset"]

# (name, text in the oracle, replacement, occurrence of the text)
MUTATIONS = [
    # weights of Eq. 3 / Eq. 16
    ("weight: factor 2 dropped", "df[:, :, None] * 2.0 * d[:, :, None]", "df[:, :, None] * d[:, :, None]", 1),
    ("weight: energy difference reversed", "d = np.asarray(eps_n)[:, None] - np.asarray(eps_m)[None, :]",
     "d = np.asarray(eps_m)[None, :] - np.asarray(eps_n)[:, None]", 1),
    ("weight: frequency not squared", "om[None, None, :] ** 2", "om[None, None, :]", 1),
    ("weight: k-point average dropped", "pref = spin_factor / (volume * nk)", "pref = spin_factor / volume", 1),
    ("weight: spin factor dropped", "pref = spin_factor / (volume * nk)", "pref = 1.0 / (volume * nk)", 1),
    ("weight: occupation difference not clipped", "df = np.where(df > 0.0, df, 0.0)", "df = np.abs(df)", 1),
    # pair densities, Eq. 4
    ("pair density: conjugate on the k+q orbital", "out[ig] = np.conj(Ck[:, ok]) @ Ckp[:, pos[ok]].T",
     "out[ig] = Ck[:, ok] @ np.conj(Ckp[:, pos[ok]]).T", 1),
    ("pair density: G with the wrong sign", "tgt = millk + G + np.asarray(G0, dtype=np.int64)",
     "tgt = millk - G + np.asarray(G0, dtype=np.int64)", 1),
    ("pair density: umklapp shift dropped", "tgt = millk + G + np.asarray(G0, dtype=np.int64)",
     "tgt = millk + G", 1),
    # PAW term, Eq. 6
    ("PAW: Q_ij transposed", 'np.einsum("ni,mj->nmij", np.conj(Pa_n), Pa_m)',
     'np.einsum("ni,mj->nmji", np.conj(Pa_n), Pa_m)', 1),
    ("PAW: conjugate on the wrong projection", 'np.einsum("ni,mj->nmij", np.conj(Pa_n), Pa_m)',
     'np.einsum("ni,mj->nmij", Pa_n, np.conj(Pa_m))', 1),
    ("PAW: projector offset not advanced", '        out += np.einsum("nmp,pg->gnm", outer, Qa)\n        off += ni\n',
     '        out += np.einsum("nmp,pg->gnm", outer, Qa)\n', 1),
    # chi0, Eq. 3
    ("chi0: conjugate on the wrong factor", "chi[j] += (N * W[:, j][None, :]) @ N.conj().T",
     "chi[j] += (N.conj() * W[:, j][None, :]) @ N.T", 1),
    ("chi0 sampled: Q sliced by position", "parts.append(blk[:, gidx].reshape(-1))",
     "parts.append(blk[:, :len(gidx)].reshape(-1))", 1),
    # E_c, Eqs. 1-2, and the quadrature of Sec. 2.1
    ("E_c: trace term dropped", "out[j] = float(np.sum(np.log1p(-lam) + lam))",
     "out[j] = float(np.sum(np.log1p(-lam)))", 1),
    ("E_c: sign of M flipped", "out[j] = float(np.sum(np.log1p(-lam) + lam))",
     "out[j] = float(np.sum(np.log1p(lam) - lam))", 1),
    ("E_c: 1/(2 pi) dropped", "E += qp.weight * float(np.sum(np.asarray(W) * e)) / TWO_PI",
     "E += qp.weight * float(np.sum(np.asarray(W) * e))", 1),
    ("E_c: q-point weight dropped", "E += qp.weight * float(np.sum(np.asarray(W) * e)) / TWO_PI",
     "E += float(np.sum(np.asarray(W) * e)) / TWO_PI", 1),
    ("quadrature: Jacobian factor 2 dropped", "W = wx * 2.0 * omega0 / (1.0 - x) ** 2",
     "W = wx * omega0 / (1.0 - x) ** 2", 1),
    ("quadrature: Jacobian not squared", "W = wx * 2.0 * omega0 / (1.0 - x) ** 2",
     "W = wx * 2.0 * omega0 / (1.0 - x)", 1),
    ("quadrature: node map inverted", "omega = omega0 * (1.0 + x) / (1.0 - x)",
     "omega = omega0 * (1.0 - x) / (1.0 + x)", 1),
    ("Gauss-Legendre: weight factor 2 dropped", "w = 2.0 / ((1.0 - x * x) * dp * dp)",
     "w = 1.0 / ((1.0 - x * x) * dp * dp)", 1),
    # lattice, sphere and Coulomb kernel
    ("Coulomb: wrong power of |q+G|", "v[nz] = 4.0 * np.pi / q2[nz]", "v[nz] = 4.0 * np.pi / np.sqrt(q2[nz])", 1),
    ("Coulomb: 2 pi instead of 4 pi", "v[nz] = 4.0 * np.pi / q2[nz]", "v[nz] = 2.0 * np.pi / q2[nz]", 1),
    ("sphere: cutoff taken as |q+G|^2 <= E", "if 0.5 * float(v @ v) <= ecut:", "if float(v @ v) <= ecut:", 1),
    ("reciprocal lattice: transpose dropped", "return TWO_PI * np.linalg.inv(np.asarray(cell, dtype=np.float64)).T",
     "return TWO_PI * np.linalg.inv(np.asarray(cell, dtype=np.float64))", 1),
    # optical limit, Eqs. 12-14
    ("optical: energy denominator reversed",
     "return -1j * D / (np.asarray(eps_m)[None, :] - np.asarray(eps_n)[:, None])",
     "return -1j * D / (np.asarray(eps_n)[:, None] - np.asarray(eps_m)[None, :])", 1),
    ("optical: factor i of the plane-wave dipole dropped", "D = 1j * (np.conj(C[nsel]) * s[None, :]) @ C[msel].T",
     "D = (np.conj(C[nsel]) * s[None, :]) @ C[msel].T", 1),
    ("optical: PAW dipole matrix transposed", "D = D + np.conj(P[nsel][:, off:off + ni]) @ Qa @ P[msel][:, off:off + ni].T",
     "D = D + np.conj(P[nsel][:, off:off + ni]) @ Qa.T @ P[msel][:, off:off + ni].T", 1),
    ("optical: head of v left at zero", "v[~nz] = 4.0 * np.pi", "v[~nz] = 0.0", 1),
    # symmetry, Eq. 9
    ("symmetry: fractional-translation phase sign", "C = C * np.exp(-2j * np.pi *", "C = C * np.exp(2j * np.pi *", 1),
    ("symmetry: time reversal without conjugation", "    if time_reversal:\n        C = np.conj(C)\n", "", 1),
    ("symmetry: projector rotation transposed", "@ np.asarray(D[a]).T", "@ np.asarray(D[a])", 1),
    # dielectric matrix
    ("epsilon^-1: Coulomb sandwich dropped",
     "M = sv[:, None] * chi[j] * sv[None, :]\n        out[j] = np.linalg.inv(np.eye(len(sv)) - M)",
     "M = chi[j]\n        out[j] = np.linalg.inv(np.eye(len(sv)) - M)", 1),
    # gradient (adjoint of Eqs. 1-6)
    ("gradient: dE/dchi sign", "G = sv[:, None] * (eye - inv) * sv[None, :]",
     "G = sv[:, None] * (inv - eye) * sv[None, :]", 1),
    ("gradient: factor 2 of the pair-density adjoint dropped", "nbar += 2.0 * np.einsum",
     "nbar += np.einsum", 1),
    ("gradient: conjugate dropped in the occupied-band adjoint",
     "gC[ik][np.ix_(nsel, ok)] += np.conj(nb_g) @ skp.C[np.ix_(msel, pos[ok])]",
     "gC[ik][np.ix_(nsel, ok)] += nb_g @ skp.C[np.ix_(msel, pos[ok])]", 1),
    ("gradient: conjugate of Q dropped in the PAW adjoint", '"gnm,ni,ijg->mj", nbar, Pn, np.conj(Qa))',
     '"gnm,ni,ijg->mj", nbar, Pn, Qa)', 1),
    ("gradient: optical head adjoint sign", "bmat = 1j * nbar[ig0] / dlt", "bmat = -1j * nbar[ig0] / dlt", 1),
    ("gradient: umklapp shift dropped in the adjoint", "tgt = millk + G + np.asarray(G0, dtype=np.int64)",
     "tgt = millk + G", 2),
    ("gradient: Q_ij transposed in the PAW adjoint", '"gnm,mj,ijg->ni", np.conj(nbar), Pm, Qa)',
     '"gnm,mj,jig->ni", np.conj(nbar), Pm, Qa)', 1),
    # further slips in the inputs of the method
    ("quadrature: omega0 ignored in the nodes", "omega = omega0 * (1.0 + x) / (1.0 - x)",
     "omega = (1.0 + x) / (1.0 - x)", 1),
    ("quadrature: omega0 ignored in the weights", "W = wx * 2.0 * omega0 / (1.0 - x) ** 2",
     "W = wx * 2.0 / (1.0 - x) ** 2", 1),
    ("Coulomb: v_G = 0 at G = 0 for every q", "nz = np.any(qg != 0.0, axis=1)",
     "nz = np.any(np.asarray(gmiller) != 0, axis=1)", 1),
    ("sphere: q ignored", "v = (np.array([g1, g2, g3], dtype=np.float64) + q) @ B",
     "v = np.array([g1, g2, g3], dtype=np.float64) @ B", 1),
    ("PAW: Q block offset not advanced", "        off += ni\n        qoff += ni * ni * ng\n    return out",
     "        off += ni\n    return out", 1),
    ("chi0: only the first transition summed", "    for t in range(len(qp.k_of)):\n        ik, ikp, G0 = int(qp.k_of[t])",
     "    for t in range(1):\n        ik, ikp, G0 = int(qp.k_of[t])", 1),
    ("optical: q direction not normalised", "    qhat = qhat / np.linalg.norm(qhat)\n    B = reciprocal(cell)",
     "    B = reciprocal(cell)", 1),
    ("symmetry: k not rotated", "kr = M @ np.asarray(oset.k_red, dtype=np.float64)",
     "kr = np.asarray(oset.k_red, dtype=np.float64)", 1),
    ("symmetry: plane waves rotated by M^T", "Qr = np.asarray(oset.miller, dtype=np.int64) @ M.T",
     "Qr = np.asarray(oset.miller, dtype=np.int64) @ M", 1),
    ("symmetry: projections not conjugated under time reversal", "            P = np.conj(P)\n",
     "            pass\n", 1),
    ("weight: energy difference not squared in the denominator", "om[None, None, :] ** 2 + d[:, :, None] ** 2",
     "om[None, None, :] ** 2 + d[:, :, None]", 1),
    ("PAW: Q block read with G slowest", "Qa = Qflat[qoff:qoff + ni * ni * ng].reshape(ni * ni, ng)",
     "Qa = Qflat[qoff:qoff + ni * ni * ng].reshape(ng, ni * ni).T", 1),
    ("optical: sign of the head", "return -1j * D / (np.asarray(eps_m)[None, :] - np.asarray(eps_n)[:, None])",
     "return 1j * D / (np.asarray(eps_m)[None, :] - np.asarray(eps_n)[:, None])", 1),
    ("gradient: Hermitian part not halved", "out[j] = (wq * omega_weights[j] / TWO_PI) * 0.5 * (G + G.conj().T)",
     "out[j] = (wq * omega_weights[j] / TWO_PI) * (G + G.conj().T)", 1),
    ("sphere: reciprocal basis transposed", "v = (np.array([g1, g2, g3], dtype=np.float64) + q) @ B",
     "v = (np.array([g1, g2, g3], dtype=np.float64) + q) @ B.T", 1),
    ("Coulomb: reciprocal basis transposed", "c = qg @ B", "c = qg @ B.T", 1),
    ("optical: k dropped from the dipole", "kQ = (np.asarray(oset.k_red, dtype=np.float64)[None, :] + "
     "np.asarray(oset.miller, dtype=np.float64)) @ B", "kQ = np.asarray(oset.miller, dtype=np.float64) @ B", 1),
    ("gradient: Gamma transposed", 'np.einsum("gh,hab->gab", Gam[j], n)', 'np.einsum("gh,hab->gab", Gam[j].T, n)', 1),
    ("pair density: plane waves on the box edge dropped", "inside = np.all((tgt >= lo) & (tgt <= hi), axis=1)",
     "inside = np.all((tgt > lo) & (tgt <= hi), axis=1)", 1),
    ("gradient: optical energy difference reversed", "dlt = sk.eps[msel][None, :] - sk.eps[nsel][:, None]",
     "dlt = sk.eps[nsel][:, None] - sk.eps[msel][None, :]", 1),
    ("gradient: optical plane-wave adjoint sign", "gC[ik][msel] += (-1j * bmat.T @ sk.C[nsel]) * sv[None, :]",
     "gC[ik][msel] += (1j * bmat.T @ sk.C[nsel]) * sv[None, :]", 1),
    ("gradient: optical PAW adjoint conjugate dropped", "gP[ik][np.ix_(msel, cols)] += bmat.T @ Pn @ np.conj(Qd)",
     "gP[ik][np.ix_(msel, cols)] += bmat.T @ Pn @ Qd", 1),
    ("PAW: projector offset of the k+q band ignored", "Pa_m = Pm[:, off:off + ni]", "Pa_m = Pm[:, :ni]", 1),
    ("symmetry: atom map ignored", "src = atom_map[a]", "src = a", 1),
    ("chi0 sampled: G sorted", "gm = gm_all[gidx]", "gm = gm_all[np.sort(gidx)]", 1),
    ("chi0 sampled: Q block stride of the sample", "off += ni * ni * ng_all", "off += ni * ni * len(gidx)", 1),
    ("E_c: Hermitian part taken with a transpose", "M = 0.5 * (M + M.conj().T)", "M = 0.5 * (M + M.T)", 1),
    ("gradient: projections of the k set on the k+q side", "Pm = skp.P[msel, off:off + ni]",
     "Pm = sk.P[msel, off:off + ni]", 1),
]


def _mutant(old, new, occurrence):
    with open(base.__file__) as f:
        src = f.read()
    assert src.count(old) >= occurrence, f"mutation site not in the oracle: {old!r}"
    at = -1
    for _ in range(occurrence):
        at = src.index(old, at + 1)
    src = src[:at] + new + src[at + len(old):]
    mod = types.ModuleType("oracle_mutant")
    exec(compile(src, os.path.basename(base.__file__) + " (mutant)", "exec"), mod.__dict__)
    return mod


def _pin_calls():
    """(name, zero-argument callable) for every pin, parametrised cases expanded,
    the slow ones last; the sampled pins get the mesh case built by the module
    under test."""
    calls, slow = [], []
    cache = {}

    def mesh():
        if "mesh" not in cache:
            cache["mesh"] = test_oracle_sampled._mesh_case()
        return cache["mesh"]

    for mod in PIN_MODULES:
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_") or name in NOT_PINS or fn.__module__ != mod.__name__:
                continue
            params = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
            cases = [{}]
            for m in params:
                argname, values = m.args[0], m.args[1]
                assert "," not in argname
                cases = [dict(c, **{argname: v}) for c in cases for v in values]
            for kw in cases:
                def call(fn=fn, kw=kw):
                    if "mesh_case" in inspect.signature(fn).parameters:
                        return fn(mesh_case=mesh(), **kw)
                    return fn(**kw)
                (slow if name in SLOW_LAST else calls).append((f"{mod.__name__}.{name}{kw or ''}", call))
    return calls + slow


def test_pins_pass_on_the_oracle_itself():
    # the harness runs the real pins: every one passes on the unmodified oracle
    calls = _pin_calls()
    assert len(calls) >= 30
    for _, call in calls:
        call()


@pytest.mark.parametrize("name,old,new,occurrence", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(monkeypatch, name, old, new, occurrence):
    mutant = _mutant(old, new, occurrence)
    for mod in PIN_MODULES:
        monkeypatch.setattr(mod, "o", mutant)
    for pin, call in _pin_calls():
        try:
            call()
        except Exception:  # an assertion of the pin, or the mutant breaking its arithmetic
            return
    pytest.fail(f"no pin fails with the planted mistake: {name}")
