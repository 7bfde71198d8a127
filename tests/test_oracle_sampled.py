"""Pins of ``oracle.chi0_sampled``, the reference of the full-size parity test.

``chi0_sampled`` evaluates Eq. 3 with the pair densities (Eq. 4 plus the PAW
term of Eq. 6) computed at a chosen subset of the response sphere only, so it
slices the flattened per-atom Q^a_ij(G) array and the k-sum on its own.  These
tests hold it to the full ``chi0`` (itself pinned by the discrete Lindhard sum,
the literal complex Eq. 3 and brute force in ``test_oracle_pins.py``) restricted
to the same rows and columns: a wrong Q-slice axis, a wrong atom offset, a lost
umklapp shift or a wrong transition subset each changes the sampled block.
"""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import synthetic as syn


def _Q(p, iq):
    gm = o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi)
    return syn.paw_Q(p.paw, p.cell, p.qpoints[iq].q_red, gm), len(gm)


def _subset_filter(ts):
    keep = set(ts)

    def f(t, nsel, msel):
        if t in keep:
            return np.arange(len(nsel)), np.arange(len(msel))
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return f


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _mesh_case():
    # two k-points along x: q = (1/2, 0, 0) maps k = 1/2 onto k' = 0 with the
    # umklapp G0 = (1, 0, 0); two PAW atoms with 4 and 5 projectors
    p = syn.small_problem(config_tag=97, nocc=3, nunocc=14, nproj=(4, 5), nw=3)
    iq = 1
    assert np.abs(p.qpoints[iq].G0).sum() > 0
    assert len(set(p.paw.nproj.tolist())) == 2
    om, _ = o.frequency_grid(p.nw)
    Q, ng = _Q(p, iq)
    full = o.chi0(p, iq, om, Q)
    return p, iq, om, Q, ng, full


@pytest.fixture(scope="module")
def mesh_case():
    return _mesh_case()


def test_sampled_equals_full_on_unsorted_gaps(mesh_case):
    p, iq, om, Q, ng, full = mesh_case
    rng = np.random.default_rng(5)
    gidx = rng.permutation(ng)[:11]          # unsorted, non-contiguous
    assert not np.all(np.diff(gidx) > 0)
    got = o.chi0_sampled(p, iq, om, gidx, Q)
    want = full[:, gidx][:, :, gidx]
    assert got.shape == (len(om), len(gidx), len(gidx))
    assert _rel(got, want) < 1e-14


def test_sampled_edges_and_repeats(mesh_case):
    p, iq, om, Q, ng, full = mesh_case
    gidx = np.array([ng - 1, 0, ng // 2, ng - 1, 1])   # both ends, a repeated index
    got = o.chi0_sampled(p, iq, om, gidx, Q)
    assert _rel(got, full[:, gidx][:, :, gidx]) < 1e-14
    assert np.array_equal(got[:, 0, 0], got[:, 3, 3])


@pytest.mark.parametrize("ts", [[0], [1]])
def test_sampled_transition_subset(mesh_case, ts):
    p, iq, om, Q, ng, _ = mesh_case
    part = o.chi0(p, iq, om, Q, pair_filter=_subset_filter(ts))
    gidx = np.array([3, ng - 2, 0, 7, ng // 3])
    got = o.chi0_sampled(p, iq, om, gidx, Q, transitions=ts)
    assert _rel(got, part[:, gidx][:, :, gidx]) < 1e-14
    # the two transitions add up to the full sum
    other = o.chi0_sampled(p, iq, om, gidx, Q, transitions=[1 - ts[0]])
    full = o.chi0_sampled(p, iq, om, gidx, Q)
    assert _rel(got + other, full) < 1e-14


def test_sampled_paw_term_is_sliced_per_atom(mesh_case):
    # the PAW term changes the sampled block, and the per-atom slicing of the
    # flattened Q array matches the full evaluation atom by atom
    p, iq, om, Q, ng, full = mesh_case
    gidx = np.array([ng - 3, 2, 9])
    no_paw = o.chi0_sampled(p, iq, om, gidx, None)
    with_paw = o.chi0_sampled(p, iq, om, gidx, Q)
    assert _rel(no_paw, with_paw) > 1e-3
    n0 = int(p.paw.nproj[0]) ** 2 * ng
    for keep in (0, 1):   # zero one atom's Q block at a time
        Qa = Q.copy()
        if keep == 0:
            Qa[n0:] = 0
        else:
            Qa[:n0] = 0
        ref = o.chi0(p, iq, om, Qa)[:, gidx][:, :, gidx]
        assert _rel(o.chi0_sampled(p, iq, om, gidx, Qa), ref) < 1e-14


def test_sampled_bulk_geometry_band_subset():
    # the bulk geometry of the full-size test (40^3 grid, 3 x 13 projectors) on a
    # band subset: the same code path chi0_sampled takes at full size
    p = syn.config1(nocc=2, nunocc=12)
    iq = 3
    om, _ = o.frequency_grid(4)
    Q, ng = _Q(p, iq)
    full = o.chi0(p, iq, om, Q)
    gidx = np.array([ng - 1, 0, 128, 127, 640, ng - 129, 5])
    got = o.chi0_sampled(p, iq, om, gidx, Q)
    assert _rel(got, full[:, gidx][:, :, gidx]) < 1e-14
