"""The tensor-core rank-k update (Eq. 17) through the C ABI: the fused
frequency weighting against the form that stores weighted operands for every
frequency, the paired launch (two frequencies per cluster sharing the
unweighted operand tiles by TMA multicast) against the unpaired one, and the
bounded-wait failure path.

The fused form (converter warps scale the staged FP32 pair densities by
w_p(w) of Eq. 16 and split them inside the kernel) performs the same FP32
product and bfloat16 split as the stored form, in the same order, so chi0 must
be bit-identical.  The timeout test makes the load role of every CTA withhold
one K stage (a test hook of the kernel), so every consumer's bounded wait runs
out: the call must return RPA_ERR_TIMEOUT, and the same context must then give
the oracle's result again.
"""
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


def _ctx(p, precision):
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    qf = (lambda iq, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm)) if p.paw else None
    b.load_problem(ctx, p, paw_Q=qf)
    return ctx


def _rel(a, ref):
    return np.abs(a - ref).max() / np.abs(ref).max()


def _case(case):
    # config 0: NG 139 (two row tiles, ragged), 240 pairs (not a multiple of 32);
    # a small mesh with umklapp and PAW; the bulk geometry (NG ~ 1200, ten row
    # tiles) on a band subset with two transitions
    if case == "config0":
        return syn.config0(), 0, 8
    if case == "mesh_umklapp_paw":
        return syn.small_problem(config_tag=95), 1, 5
    p = syn.config1(nocc=3, nunocc=70)
    p.qpoints = [p.qpoints[3]]
    p.qpoints[0].k_of, p.qpoints[0].kq_of = p.qpoints[0].k_of[:2], p.qpoints[0].kq_of[:2]
    p.qpoints[0].G0 = p.qpoints[0].G0[:2]
    return p, 0, 16


@pytest.mark.parametrize("case", ["config0", "mesh_umklapp_paw", "bulk_subset"])
def test_fused_weighting_bit_identical(case):
    p, iq, nw = _case(case)
    om, W = o.frequency_grid(nw)
    ctx = _ctx(p, "bf16x2")
    try:
        fused = b.rpa_chi0(ctx, iq, om)
        Ef, tf = b.rpa_energy(ctx, [iq], [1.0], om, W)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FUSE, 0)
        stored = b.rpa_chi0(ctx, iq, om)
        Es, ts = b.rpa_energy(ctx, [iq], [1.0], om, W)
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FUSE, 2)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)
    assert np.array_equal(fused, stored)
    assert np.array_equal(tf, ts) and Ef == Es
    if case != "bulk_subset":
        Q = None
        if p.paw is not None:
            gm = o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi)
            Q = syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm)
        assert _rel(fused, o.chi0(p, iq, om, Q)) < 2e-5


@pytest.mark.parametrize("pair", [1, 2])
@pytest.mark.parametrize("case", ["config0", "mesh_umklapp_paw", "bulk_subset"])
def test_paired_launch_bit_identical(case, pair):
    # pair 1: 8 and 16 frequencies run paired, 5 (odd) falls back to the
    # unpaired launch; pair 2: two-SM products over row-tile pairs (config 0:
    # one pair; the bulk subset: ten row tiles, five pairs)
    p, iq, nw = _case(case)
    om, W = o.frequency_grid(nw)
    ctx = _ctx(p, "bf16x2")
    try:
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FUSE, 0)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PAIR, 0)
        single = b.rpa_chi0(ctx, iq, om)
        Es, ts = b.rpa_energy(ctx, [iq], [1.0], om, W)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PAIR, pair)
        paired = b.rpa_chi0(ctx, iq, om)
        Ep, tp = b.rpa_energy(ctx, [iq], [1.0], om, W)
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PAIR, 3)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)
    assert np.array_equal(paired, single)
    assert np.array_equal(tp, ts) and Ep == Es


@pytest.mark.parametrize("precision,fuse,pair", [("bf16x2", 1, 0), ("bf16x2", 0, 0), ("bf16x2", 0, 1),
                                                ("bf16x2", 0, 2), ("bf16x3", 0, 0)])
def test_bounded_wait_timeout_leaves_context_usable(precision, fuse, pair):
    p = syn.config0()
    om, W = o.frequency_grid(p.nw)
    ref = o.chi0(p, 0, om)
    E_ref, _ = o.energy(p, om, W)
    ctx = _ctx(p, precision)
    try:
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FUSE, fuse)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PAIR, pair)
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_WAIT_US, 999)
        assert e.value.status == b.RPA_ERR_ARG
        # 20 ms waits; every CTA withholds its second K stage
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_WAIT_US, 20000)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_STALL, 2)
        with pytest.raises(b.RpaError) as e:
            b.rpa_energy(ctx, [0], [1.0], om, W)
        assert e.value.status == b.RPA_ERR_TIMEOUT
        with pytest.raises(b.RpaError) as e:
            b.rpa_chi0(ctx, 0, om)
        assert e.value.status == b.RPA_ERR_TIMEOUT
        # the same context, knobs back to their defaults
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_STALL, 0)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_WAIT_US, 4000000)
        chi = b.rpa_chi0(ctx, 0, om)
        E, _ = b.rpa_energy(ctx, [0], [1.0], om, W)
    finally:
        b.rpa_destroy(ctx)
    tol = 2e-5 if precision == "bf16x2" else 4e-6
    assert _rel(chi, ref) < tol
    assert abs(E - E_ref) <= 1e-6 * abs(E_ref)
