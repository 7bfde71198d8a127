"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle on
the same seeded inputs."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu

# Tolerances.  E_c: 1e-10 relative in FP64, 1e-6 relative in the FP32 and
# split-bfloat16 modes.  chi0: elementwise, relative to its largest element.
# Per-frequency terms e(w): the E_c bound, except bf16x2 where a two-term
# bfloat16 split represents each operand to 2^-16 relative; on the 240-pair
# tiny case that averages down only to ~1.5e-6 per term, so the per-term bound
# there is 5e-6 (the summed E_c still has to meet 1e-6).
TOL = {
    "fp64": dict(chi=1e-11, ec=1e-10, term=1e-10),
    "fp32": dict(chi=4e-6, ec=1e-6, term=1e-6),
    "bf16x2": dict(chi=2e-5, ec=1e-6, term=5e-6),
    "bf16x3": dict(chi=4e-6, ec=1e-6, term=1e-6),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build()
    b.load()


def _ctx(p, precision, iqs=None, with_paw=True):
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    qf = (lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm)) if (with_paw and p.paw) else None
    b.load_problem(ctx, p, qs=iqs, paw_Q=qf)
    return ctx


def _oracle_Q(p, iq):
    if p.paw is None:
        return None
    gm = o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi)
    return syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm)


def _rel(a, b_):
    return np.abs(a - b_).max() / np.abs(b_).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x2", "bf16x3"])
def test_config0_chi_and_energy(precision):
    p = syn.config0()
    om, W = o.frequency_grid(p.nw)
    ctx = _ctx(p, precision)
    try:
        gm = b.rpa_gvectors(ctx, 0)
        assert np.array_equal(gm, o.g_sphere(p.cell, p.qpoints[0].q_red, p.ecut_chi))
        chi = b.rpa_chi0(ctx, 0, om)
        ref = o.chi0(p, 0, om)
        assert _rel(chi, ref) < TOL[precision]["chi"]
        E, terms = b.rpa_energy(ctx, [0], [1.0], om, W)
        Er, tr = o.energy(p, om, W)
        assert abs(E - Er) < TOL[precision]["ec"] * abs(Er)
        assert np.abs(terms[0] - tr[0]).max() < TOL[precision]["term"] * np.abs(tr).max()
    finally:
        b.rpa_destroy(ctx)


def test_config0_matches_stored_terms():
    """The FP64 path against the stored oracle terms of tests/golden/."""
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config0_terms.txt")) as f:
        rows = [[float(x) for x in ln.split()] for ln in f if ln.strip() and not ln.startswith("#")]
    t = np.array(rows)
    p = syn.config0()
    ctx = _ctx(p, "fp64")
    try:
        _, terms = b.rpa_energy(ctx, [0], [1.0], t[:, 1], t[:, 2])
    finally:
        b.rpa_destroy(ctx)
    assert np.max(np.abs(terms[0] - t[:, 3])) <= TOL["fp64"]["term"] * np.max(np.abs(t[:, 3]))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x2", "bf16x3"])
def test_small_mesh_umklapp_paw_all_q(precision):
    """2x1x1 mesh (umklapp at q = 1/2), ragged Miller boxes, two PAW atoms."""
    p = syn.small_problem()
    om, W = o.frequency_grid(p.nw)
    ctx = _ctx(p, precision)
    try:
        Qs = [_oracle_Q(p, iq) for iq in range(len(p.qpoints))]
        for iq in range(len(p.qpoints)):
            chi = b.rpa_chi0(ctx, iq, om)
            ref = o.chi0(p, iq, om, Qs[iq])
            assert _rel(chi, ref) < TOL[precision]["chi"], iq
        iqs = list(range(len(p.qpoints)))
        wq = [qp.weight for qp in p.qpoints]
        E, _ = b.rpa_energy(ctx, iqs, wq, om, W)
        Er, _ = o.energy(p, om, W, Qs)
        assert abs(E - Er) < TOL[precision]["ec"] * abs(Er)
    finally:
        b.rpa_destroy(ctx)


def test_device_pointers_match_host():
    import torch
    p = syn.small_problem(config_tag=94)
    om, _ = o.frequency_grid(4)
    ctx_h = _ctx(p, "fp64")
    ctx_d = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, "fp64")
    try:
        for i, s in enumerate(p.sets):
            Cd = torch.from_numpy(s.C).cuda()
            b.rpa_set_orbitals(ctx_d, i, s.k_red, s.miller, Cd, s.eps, s.f)
            b.rpa_set_paw(ctx_d, i, p.paw.nproj, torch.from_numpy(s.P).cuda())
        qp = p.qpoints[1]
        b.rpa_set_qpoint(ctx_d, 1, qp.q_red, qp.k_of, qp.kq_of, qp.G0)
        gm = b.rpa_gvectors(ctx_d, 1)
        b.rpa_set_paw_Q(ctx_d, 1, p.paw.nproj, torch.from_numpy(syn.paw_Q(p.paw, p.cell, qp.q_red, gm)).cuda())
        ng = len(gm)
        out = torch.zeros((len(om), ng, ng), dtype=torch.complex128, device="cuda")
        b.rpa_chi0(ctx_d, 1, om, out)
        torch.cuda.synchronize()
        host = b.rpa_chi0(ctx_h, 1, om)
        assert np.array_equal(out.cpu().numpy(), host)
    finally:
        b.rpa_destroy(ctx_h)
        b.rpa_destroy(ctx_d)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x2", "bf16x3"])
def test_config1_geometry_two_transitions(precision):
    """Full config-1 geometry (9 bohr box, 40^3 grid, 20 Ha orbitals, NG ~ 1200,
    3 x 13 projectors) with a band subset and two transitions of q = (0, 1/2, 1/2),
    one of them with an umklapp vector."""
    full = syn.config1()
    nsub = 2 + 150
    sets = []
    for s in full.sets:
        keep = np.r_[np.arange(14, 16), np.arange(16, 16 + 150)]
        sets.append(syn.OrbitalSet(s.k_red, s.miller, s.C[keep], s.eps[keep], s.f[keep], s.P[keep]))
    qp0 = full.qpoints[3]
    trans = [0, 3]
    qp = syn.QPoint(qp0.q_red, qp0.k_of[trans], qp0.kq_of[trans], qp0.G0[trans], 1.0)
    assert np.abs(qp.G0).sum() > 0
    p = syn.Problem(full.name, 1, full.cell, full.grid, full.ecut_wf, full.ecut_chi, full.spin_factor,
                    full.nk_bz, sets, [qp], 16, full.paw)
    assert sets[0].C.shape[0] == nsub
    om, W = o.frequency_grid(16)
    ctx = _ctx(p, precision)
    try:
        chi = b.rpa_chi0(ctx, 0, om)
        ref = o.chi0(p, 0, om, _oracle_Q(p, 0))
        assert _rel(chi, ref) < TOL[precision]["chi"]
        # the log-det of the GPU's own chi0 (NG ~ 1200: 38 panels, ragged last
        # tile) against FP64 eigenvalues of the same matrix; in the FP32 and
        # BF16X2 modes with every trailing-update choice: float-float with the
        # look-ahead (default), float-float on one stream (the same tiles in
        # the same order, so bit-identical), FP64
        v = o.coulomb(p.cell, qp.q_red, b.rpa_gvectors(ctx, 0))
        want = o.ec_terms(chi, v)
        _, t = b.rpa_energy(ctx, [0], [1.0], om, W)
        assert np.abs(t[0] - want).max() / np.abs(want).max() < (1e-11 if precision == "fp64" else 1e-10)
        if precision != "fp64":
            b.rpa_set_tuning(ctx, b.RPA_TUNE_LOGDET, 1)
            _, t1 = b.rpa_energy(ctx, [0], [1.0], om, W)
            assert np.array_equal(t1, t)
            b.rpa_set_tuning(ctx, b.RPA_TUNE_LOGDET, 0)
            _, t64 = b.rpa_energy(ctx, [0], [1.0], om, W)
            assert np.abs(t64[0] - want).max() / np.abs(want).max() < 1e-11
            with pytest.raises(b.RpaError):
                b.rpa_set_tuning(ctx, b.RPA_TUNE_LOGDET, 3)
    finally:
        b.rpa_destroy(ctx)


@pytest.fixture(scope="module")
def full_size_case():
    """The bench's bulk workload at full size (all 8 k, 16 occupied x 1200 empty
    bands, 3 x 13 PAW projectors, 16 frequencies) at q = (0, 1/2, 1/2), and the
    oracle at 23 sampled G indices: both ragged edges (0, 1, NG-2, NG-1), the last
    row of every 128-row tile of the rank-k kernel and one random row inside each
    tile, in shuffled order, so every row and column tile of the lower-triangle
    grid and both of its ragged edges are checked."""
    p = syn.config1()
    iq = 3
    om, _ = o.frequency_grid(16)
    ng = len(o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi))
    rng = np.random.default_rng(11)
    g = {0, 1, ng - 2, ng - 1}
    for t in range((ng + 127) // 128):
        lo, hi = 128 * t, min(ng, 128 * t + 128)
        g.add(int(rng.integers(lo, hi)))
        g.add(hi - 1)
    gidx = np.array(sorted(g))
    rng.shuffle(gidx)
    ref = o.chi0_sampled(p, iq, om, gidx, _oracle_Q(p, iq))
    return p, iq, om, gidx, ref


@pytest.mark.parametrize("precision", ["bf16x2", "fp64"])
def test_config1_full_size_sampled(full_size_case, precision):
    """Full-size chi0 in the bench's launch configuration (bf16x2) and in the plain
    FP64 mode: elements on the sampled G rows/columns against the oracle
    evaluated at those G only, plus properties that hold at any size (Hermitian,
    non-positive diagonal)."""
    p, iq, om, gidx, ref = full_size_case
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, qs=[iq], paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))
        chi = b.rpa_chi0(ctx, iq, om)
    finally:
        b.rpa_destroy(ctx)
    ng = chi.shape[1]
    assert ng > 1100 and ng % 128 != 0 and max(gidx) == ng - 1
    got = chi[:, gidx][:, :, gidx]
    assert np.abs(got - ref).max() / np.abs(ref).max() < TOL[precision]["chi"]
    assert np.array_equal(chi[3], chi[3].conj().T)
    assert np.all(np.einsum("wii->wi", chi).real <= 0)


@pytest.fixture(scope="module")
def slab_case():
    """Slab geometry (9.4 x 8.1 x 40 bohr, 48 x 40 x 200 grid, 13039 plane waves,
    NG = 3058, 16 x 18 + 2 x 8 projectors) on a band subset: k = Gamma and
    (0, 1/2, 0), q = (0, 1/2, 0) with one umklapp transition, 8 frequencies."""
    p = syn.config2(nocc=3, nunocc=40, kidx=[0, 1])
    iq = 1
    assert np.abs(p.qpoints[iq].G0).sum() > 0
    om, _ = o.frequency_grid(8)
    return p, iq, om, o.chi0(p, iq, om, _oracle_Q(p, iq))


@pytest.mark.parametrize("precision", ["fp64", "bf16x2"])
def test_config2_slab_geometry(slab_case, precision):
    p, iq, om, ref = slab_case
    ctx = _ctx(p, precision, iqs=[iq])
    try:
        chi = b.rpa_chi0(ctx, iq, om)
    finally:
        b.rpa_destroy(ctx)
    assert chi.shape == ref.shape and ref.shape[1] > 3000
    assert _rel(chi, ref) < TOL[precision]["chi"]


def test_tuning_knobs_change_rounding_only():
    p = syn.small_problem(config_tag=95)
    om, _ = o.frequency_grid(4)
    ctx = _ctx(p, "bf16x2")
    try:
        a = b.rpa_chi0(ctx, 1, om)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FOLD, 4)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PAIR_CHUNK, 7)
        c = b.rpa_chi0(ctx, 1, om)
        assert _rel(c, a) < TOL["bf16x2"]["chi"]
        # 32-element K stages x 4 with the 64-byte swizzle
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FOLD, 1)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PIPE, 1)
        d = b.rpa_chi0(ctx, 1, om)
        assert _rel(d, a) < TOL["bf16x2"]["chi"]
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FOLD, 0)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)


@pytest.mark.parametrize("precision", ["bf16x2", "bf16x3"])
def test_paw_product_on_tensor_cores(precision):
    """The opt-in tensor-core PAW product (Eq. 6 with the per-band factor R)
    against the oracle: chi0 and the energy terms within the mode's bounds, and
    the projector count (9) far from a K tile so the zero padding of K is
    exercised; out-of-range choices are rejected."""
    p = syn.small_problem(config_tag=95)
    iq = 1
    om, W = o.frequency_grid(6)
    ref = o.chi0(p, iq, om, _oracle_Q(p, iq))
    v = o.coulomb(p.cell, p.qpoints[iq].q_red, o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi))
    want = o.ec_terms(ref, v)
    ctx = _ctx(p, precision)
    try:
        plain = b.rpa_chi0(ctx, iq, om)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PAW_TC, 1)
        chi = b.rpa_chi0(ctx, iq, om)
        _, t = b.rpa_energy(ctx, [iq], [1.0], om, W)
        assert _rel(chi, ref) < TOL[precision]["chi"]
        assert np.abs(t[0] - want).max() <= TOL[precision]["term"] * np.abs(want).max()
        assert abs(np.dot(W, t[0]) - np.dot(W, want)) <= TOL[precision]["ec"] * abs(np.dot(W, want))
        assert 0 < _rel(chi, plain) < TOL[precision]["chi"]
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_PAW_TC, 2)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)


def test_minimal_transform_grid_equals_caller_grid():
    """The alias-free minimal transform grid and the caller's full grid give the
    same chi0 (both equal the plane-wave sums of Eq. 4)."""
    p = syn.small_problem(config_tag=96, grid=(20, 22, 18))
    om, _ = o.frequency_grid(3)
    ctx = _ctx(p, "fp64")
    try:
        a = b.rpa_chi0(ctx, 1, om)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_GRID, 1)
        c = b.rpa_chi0(ctx, 1, om)
    finally:
        b.rpa_destroy(ctx)
    assert _rel(a, c) < 1e-12
    assert _rel(a, o.chi0(p, 1, om, _oracle_Q(p, 1))) < TOL["fp64"]["chi"]


def test_qpoint_sphere_is_the_host_sphere():
    """rpa_set_qpoint's G list, read back through rpa_gvectors, is the sphere
    rpa_response_sphere plans without a context (tested on the CPU against the
    oracle), at every q-point of a mesh with umklapp."""
    p = syn.small_problem(config_tag=95)
    ctx = _ctx(p, "fp64", with_paw=False)
    try:
        for iq, qp in enumerate(p.qpoints):
            gm, _ = b.rpa_response_sphere(p.cell, qp.q_red, p.ecut_chi)
            assert np.array_equal(b.rpa_gvectors(ctx, iq), gm)
    finally:
        b.rpa_destroy(ctx)


def test_not_hpd_is_reported_not_trapped():
    """Mirrored band energies (occupied above empty by the same gaps) flip the sign
    of chi0, so 1 - v^1/2 chi0 v^1/2 has eigenvalues below zero: the Cholesky
    flag must come back as a status."""
    p = syn.config0()
    for s in p.sets:
        s.eps = -s.eps
    om, W = o.frequency_grid(4)
    ctx = _ctx(p, "fp64")
    try:
        with pytest.raises(b.RpaError) as e:
            b.rpa_energy(ctx, [0], [1.0], om, W)
        assert e.value.status == b.RPA_ERR_NOT_HPD
        # the context stays usable
        chi = b.rpa_chi0(ctx, 0, om)
        assert np.isfinite(chi).all()
    finally:
        b.rpa_destroy(ctx)


def test_device_allocation_failure_is_a_status_and_the_context_recovers():
    """A chi0 that cannot fit in device memory (4096 frequencies x NG^2 x 16 B,
    0.6 TB at NG 3042) makes the allocation fail before any kernel runs:
    RPA_ERR_OOM, not a crash, and the same context then evaluates the q-point
    at two frequencies exactly as a fresh context does."""
    cell = np.eye(3) * 20.0
    q = np.array([0.25, 0.0, 0.0])
    sets = [syn.make_orbitals(81, i, cell, k, 0.5, 1, 2) for i, k in enumerate([np.zeros(3), q])]
    qp = syn.QPoint(q, np.array([0]), np.array([1]), np.zeros((1, 3), np.int32), 1.0)
    p = syn.Problem("oom", 81, cell, (24, 24, 24), 0.5, 4.0, 2.0, 1, sets, [qp], 2, None)
    om, W = o.frequency_grid(2)
    ctx = _ctx(p, "fp64")
    try:
        ng = len(b.rpa_gvectors(ctx, 0))
        assert ng > 3000 and 4096 * ng * ng * 16 > 2 * 288e9
        with pytest.raises(b.RpaError) as e:
            b.rpa_energy(ctx, [0], [1.0], np.linspace(0.1, 10.0, 4096), np.ones(4096))
        assert e.value.status == b.RPA_ERR_OOM
        E1, t1 = b.rpa_energy(ctx, [0], [1.0], om, W)
    finally:
        b.rpa_destroy(ctx)
    ctx = _ctx(p, "fp64")
    try:
        E2, t2 = b.rpa_energy(ctx, [0], [1.0], om, W)
    finally:
        b.rpa_destroy(ctx)
    assert np.array_equal(t1, t2) and E1 == E2 and E1 < 0


def test_state_and_argument_errors():
    p = syn.config0()
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, "fp64")
    try:
        with pytest.raises(b.RpaError) as e:
            b.rpa_chi0(ctx, 0, [1.0])
        assert e.value.status == b.RPA_ERR_STATE
        s = p.sets[0]
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_orbitals(ctx, 0, s.k_red, np.concatenate([s.miller[:1], s.miller[:-1]]), s.C, s.eps, s.f)
        assert e.value.status == b.RPA_ERR_ARG
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_orbitals(ctx, 0, s.k_red, s.miller, s.C, s.eps, s.f * 2)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)
    # a grid too small for the orbital spheres must be rejected (aliasing)
    ctx = b.rpa_create(p.cell, (12, 12, 12), p.ecut_chi, p.spin_factor, p.nk_bz, "fp64")
    try:
        for i, s in enumerate(p.sets):
            b.rpa_set_orbitals(ctx, i, s.k_red, s.miller, s.C, s.eps, s.f)
        qp = p.qpoints[0]
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_qpoint(ctx, 0, qp.q_red, qp.k_of, qp.kq_of, qp.G0)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)


def test_device_memory_in_host_arguments_is_an_argument_error():
    """Frequencies, weights, index lists, small parameter arrays and scalar
    outputs are read or written by the host: device memory there is
    RPA_ERR_ARG (not a crash of the process), and the context stays usable."""
    import ctypes as ct
    import torch
    p = syn.config0()
    om, W = o.frequency_grid(4)
    ctx = _ctx(p, "fp64")
    try:
        lib = b.lib()

        def hp(a):
            return a.ctypes.data_as(b._P)

        def dp(t):
            return ct.c_void_p(t.data_ptr())

        om_h, W_h = np.ascontiguousarray(om), np.ascontiguousarray(W)
        iq_h, wq_h = np.zeros(1, np.int32), np.ones(1)
        om_d = torch.from_numpy(om_h).cuda()
        iq_d = torch.zeros(1, dtype=torch.int32, device="cuda")
        one_d = torch.ones(1, dtype=torch.float64, device="cuda")
        ng = len(b.rpa_gvectors(ctx, 0))
        out = np.zeros((len(om), ng, ng), dtype=np.complex128)
        E = ct.c_double()
        s, qp = p.sets[0], p.qpoints[0]
        k_h = np.ascontiguousarray(s.k_red, dtype=np.float64)
        m_h = np.ascontiguousarray(s.miller, dtype=np.int32)
        C_h = np.ascontiguousarray(s.C, dtype=np.complex128)
        e_h, f_h = np.ascontiguousarray(s.eps, dtype=np.float64), np.ascontiguousarray(s.f, dtype=np.float64)
        q_h = np.ascontiguousarray(qp.q_red, dtype=np.float64)
        ko_h, kq_h = np.ascontiguousarray(qp.k_of, dtype=np.int32), np.ascontiguousarray(qp.kq_of, dtype=np.int32)
        G0_h = np.ascontiguousarray(np.asarray(qp.G0).reshape(-1, 3), dtype=np.int32)
        nb, npw = C_h.shape
        e_d, m_d, ko_d = (torch.from_numpy(a).cuda() for a in (e_h, m_h, ko_h))
        st = {
            "chi0 omega": lib.rpa_chi0(ctx, 0, len(om), dp(om_d), hp(out)),
            "energy iqs": lib.rpa_energy(ctx, 1, dp(iq_d), hp(wq_h), len(om), hp(om_h), hp(W_h), ct.byref(E),
                                         None),
            "energy wq": lib.rpa_energy(ctx, 1, hp(iq_h), dp(one_d), len(om), hp(om_h), hp(W_h), ct.byref(E),
                                        None),
            "energy Ec": lib.rpa_energy(ctx, 1, hp(iq_h), hp(wq_h), len(om), hp(om_h), hp(W_h), dp(one_d), None),
            "frequencies": lib.rpa_set_frequencies(ctx, len(om), dp(om_d)),
            "orbitals eps": lib.rpa_set_orbitals(ctx, 7, hp(k_h), nb, npw, hp(m_h), hp(C_h), dp(e_d), hp(f_h)),
            "orbitals miller": lib.rpa_set_orbitals(ctx, 7, hp(k_h), nb, npw, dp(m_d), hp(C_h), hp(e_h), hp(f_h)),
            "qpoint k_of": lib.rpa_set_qpoint(ctx, 3, hp(q_h), len(ko_h), dp(ko_d), hp(kq_h), hp(G0_h), None),
            "gvectors ng": lib.rpa_gvectors(ctx, 0, dp(iq_d), None),
        }
        assert all(v == b.RPA_ERR_ARG for v in st.values()), st
        # nothing was changed, and device memory where the header allows it still works
        with pytest.raises(b.RpaError) as e:
            b.rpa_gvectors(ctx, 3)
        assert e.value.status == b.RPA_ERR_STATE
        Ed, _ = b.rpa_energy(ctx, [0], [1.0], om, W)
        Er, _ = o.energy(p, om, W)
        assert abs(Ed - Er) < TOL["fp64"]["ec"] * abs(Er)
        chi_d = torch.zeros((len(om), ng, ng), dtype=torch.complex128, device="cuda")
        b.rpa_chi0(ctx, 0, om, chi_d)
        torch.cuda.synchronize()
        assert _rel(chi_d.cpu().numpy(), o.chi0(p, 0, om)) < TOL["fp64"]["chi"]
    finally:
        b.rpa_destroy(ctx)
