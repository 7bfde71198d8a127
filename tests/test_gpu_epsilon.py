"""GPU parity of rpa_epsilon_inv: (1 - v^1/2 chi0 v^1/2)^-1 against the oracle
in every mode, including a q = 0 point with the optical limit."""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 4e-6, "bf16x2": 2e-5, "bf16x3": 4e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()


@pytest.fixture(scope="module")
def case():
    p = syn.small_problem(config_tag=87)
    om, _ = o.frequency_grid(p.nw)
    refs = {}
    Qn = syn.paw_Qnabla(p.paw, 87)
    qdir = [0.0, 0.6, 0.8]
    for iq, qp in enumerate(p.qpoints):
        gm = o.g_sphere(p.cell, qp.q_red, p.ecut_chi)
        Q = syn.paw_Q(p.paw, p.cell, qp.q_red, gm)
        opt = (qdir, Qn) if iq == 0 else None
        chi = o.chi0(p, iq, om, Q, optical=opt)
        refs[iq] = o.epsilon_inv(chi, o.coulomb(p.cell, qp.q_red, gm, optical=opt is not None))
    return p, om, refs, qdir, Qn


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x2", "bf16x3"])
def test_epsilon_inverse(case, precision):
    p, om, refs, qdir, Qn = case
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))
        b.rpa_set_optical(ctx, 0, qdir, p.paw.nproj, Qn)
        for iq, ref in refs.items():
            e = b.rpa_epsilon_inv(ctx, iq, om)
            # eps^-1 - 1 carries the chi0 error; the identity part is exact
            d = ref - np.eye(ref.shape[1])[None]
            assert np.abs(e - ref).max() <= TOL[precision] * np.abs(d).max(), iq
            assert np.abs(e - np.conj(np.transpose(e, (0, 2, 1)))).max() <= 1e-10 * np.abs(d).max()
    finally:
        b.rpa_destroy(ctx)
