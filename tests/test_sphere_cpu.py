"""The response sphere of Sec. 2.1 as the library plans it on the host, without
a GPU: rpa_response_sphere is the routine rpa_set_qpoint builds every q-point's
G list and Coulomb kernel with.  Checked against lattice-point counts, the
Coulomb kernel's closed form, the umklapp shift of the definition and the
oracle's sphere on the cells of the synthetic workloads."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300.build import build


@pytest.fixture(scope="module", autouse=True)
def lib():
    build()
    return b.load()


def _tri():
    return np.array([[7.0, 0.0, 0.0], [2.1, 6.4, 0.0], [-1.3, 1.7, 8.2]])


# (cell, q_red, ecut_chi): the tiny cubic, bulk and slab workloads, the
# anisotropic small cell of the tests, and a triclinic cell at a general q
CASES = [
    ("tiny-cubic", np.eye(3) * 10.0, (0.1, 0.0, 0.0), 2.0),
    ("bulk-q0", np.eye(3) * 9.0, (0.0, 0.0, 0.0), 10.5),
    ("bulk-zone-edge", np.eye(3) * 9.0, (0.5, 0.5, 0.0), 10.5),
    ("slab", np.diag([9.4, 8.1, 40.0]), (0.25, -0.5, 0.0), 7.55),
    ("small-aniso", np.diag([5.0, 5.5, 4.5]), (0.5, 0.0, 0.0), 1.5),
    ("triclinic", _tri(), (0.25, -0.125, 1.0 / 3.0), 3.0),
]


def _k2(cell, q, gm):
    c = (np.asarray(gm, dtype=np.float64) + np.asarray(q, dtype=np.float64)) @ o.reciprocal(cell)
    return np.einsum("ij,ij->i", c, c)


def _boundary_margin(cell, q, ecut):
    # smallest | |q+G|^2/2 - ecut | over a box that holds the sphere with room
    # to spare: with a margin well above rounding, membership is decided the
    # same way in any summation order
    ext = int(np.ceil(np.sqrt(2 * ecut) * np.abs(np.linalg.inv(o.reciprocal(cell))).sum(axis=0).max())) + 3
    r = np.arange(-ext, ext + 1)
    box = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    return np.abs(0.5 * _k2(cell, q, box) - ecut).min() / ecut


def test_lattice_point_counts():
    # a = 2 pi makes B the identity: |G|^2 = m.m, and the counts of integer
    # points with m.m <= n for n = 0..8 are 1, 7, 19, 27, 33, 57, 81, 81, 93
    cell = np.eye(3) * 2 * np.pi
    counts = [len(b.rpa_response_sphere(cell, (0, 0, 0), 0.5 * n + 1e-9)[0]) for n in range(9)]
    assert counts == [1, 7, 19, 27, 33, 57, 81, 81, 93]


def test_coulomb_closed_form():
    cell = np.eye(3) * 10.0
    gm, v = b.rpa_response_sphere(cell, (0, 0, 0), 1.0)
    zero = np.flatnonzero(~gm.any(axis=1))
    assert len(zero) == 1 and v[zero[0]] == 0.0
    assert np.all(np.delete(v, zero) > 0)
    # the six nearest vectors have |G| = 2 pi / 10, so v = 100 / pi
    six = np.flatnonzero(np.abs(gm).sum(axis=1) == 1)
    assert len(six) == 6
    assert np.allclose(v[six], 100.0 / np.pi, rtol=1e-14, atol=0)
    # away from q = 0 no G is excluded and v = 4 pi / |q+G|^2 throughout
    q = (0.1, 0.0, 0.0)
    gm, v = b.rpa_response_sphere(cell, q, 1.0)
    assert np.all(v > 0)
    assert np.allclose(v, 4 * np.pi / _k2(cell, q, gm), rtol=1e-14, atol=0)


@pytest.mark.parametrize("name,cell,q,ecut", CASES, ids=[c[0] for c in CASES])
def test_sphere_matches_oracle(name, cell, q, ecut):
    assert _boundary_margin(cell, q, ecut) > 1e-9, "case sits on the cutoff: membership is not well posed"
    gm, v = b.rpa_response_sphere(cell, q, ecut)
    ref = o.g_sphere(cell, q, ecut)
    assert gm.shape == ref.shape and np.array_equal(gm, ref), name
    assert np.allclose(v, o.coulomb(cell, q, ref), rtol=1e-13, atol=0)
    # every vector inside, lexicographic and unique
    assert np.all(0.5 * _k2(cell, q, gm) <= ecut)
    key = [tuple(r) for r in gm]
    assert key == sorted(set(key))


@pytest.mark.parametrize("name,cell,q,ecut", CASES, ids=[c[0] for c in CASES])
def test_umklapp_shift(name, cell, q, ecut):
    # q -> q + G0 moves the sphere by -G0 and leaves v unchanged: the same
    # set {G : |q+G|^2/2 <= ecut} written in other Miller indices
    G0 = np.array([1, 0, -1])
    gm, v = b.rpa_response_sphere(cell, q, ecut)
    gs, vs = b.rpa_response_sphere(cell, np.asarray(q) + G0, ecut)
    assert np.array_equal(gs, gm - G0)
    assert np.allclose(vs, v, rtol=1e-13, atol=0)


def test_rejects_bad_arguments():
    cell, q = np.eye(3) * 6.0, (0.0, 0.0, 0.0)
    for c, qq, e in ((np.zeros((3, 3)), q, 1.0), (np.ones((3, 3)), q, 1.0), (cell, q, 0.0), (cell, q, -2.0),
                     (cell, q, np.nan), (cell, q, np.inf), (cell, (np.nan, 0.0, 0.0), 1.0),
                     (cell, (0.0, np.inf, 0.0), 1.0), (cell, q, 1e9)):
        with pytest.raises(b.RpaError) as err:
            b.rpa_response_sphere(c, qq, e)
        assert err.value.status == b.RPA_ERR_ARG
    lib = b.lib()
    import ctypes as ct
    pc = np.ascontiguousarray(cell.reshape(9))
    pq = np.zeros(3)
    ng = ct.c_int32(-1)
    assert lib.rpa_response_sphere(pc.ctypes.data_as(b._P), pq.ctypes.data_as(b._P), 1.0, 0, None, None,
                                   None) == b.RPA_ERR_ARG
    assert lib.rpa_response_sphere(pc.ctypes.data_as(b._P), pq.ctypes.data_as(b._P), 1.0, 0, ct.byref(ng), None,
                                   None) == b.RPA_OK
    n = ng.value
    assert n == len(o.g_sphere(cell, q, 1.0))
    out = np.zeros((n, 3), dtype=np.int32)
    # an output one entry too short is refused, with NG still reported
    ng.value = -1
    assert lib.rpa_response_sphere(pc.ctypes.data_as(b._P), pq.ctypes.data_as(b._P), 1.0, n - 1, ct.byref(ng),
                                   out.ctypes.data_as(b._P), None) == b.RPA_ERR_ARG
    assert ng.value == n and not out.any()


def test_empty_sphere_is_a_valid_answer():
    # at the zone corner with a cutoff below |q|^2/2 no G qualifies
    cell = np.eye(3) * 2 * np.pi
    gm, v = b.rpa_response_sphere(cell, (0.5, 0.5, 0.5), 0.3)
    assert gm.shape == (0, 3) and v.shape == (0,)
