"""The slowest and middle pair-density axes as two-level pruned DFTs (Eq. 10,
the N-point axis split as (N / L) x L) against the direct sums: the same
transform with other roundings, so chi0 agrees to the working precision's
rounding (FP64: 1e-13 relative; FP32 pair densities: 2e-6), and the FP64 mode
still matches the oracle.  Geometries: the bulk box (40-point axes, L = 4),
the slab geometry and a small mesh with umklapp and PAW."""
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


def _cases():
    bulk = syn.config1(nocc=2, nunocc=30)
    bulk.qpoints = [bulk.qpoints[3]]
    slab = syn.config2(nocc=2, nunocc=12, kidx=[0, 1])
    slab.qpoints = [slab.qpoints[1]]
    return {"bulk": bulk, "slab": slab, "mesh": syn.small_problem(config_tag=95)}


@pytest.mark.parametrize("case", ["bulk", "slab", "mesh"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("bf16x2", 2e-6)])
def test_factorised_axes_match_direct(case, precision, tol):
    p = _cases()[case]
    iq = 1 if case == "mesh" else 0
    om, _ = o.frequency_grid(4)
    Q = lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm)
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, paw_Q=Q)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_FACT, 1)
        fact = b.rpa_chi0(ctx, iq, om)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_FACT, 0)
        direct = b.rpa_chi0(ctx, iq, om)
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_FACT, 2)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)
    scale = np.abs(direct).max()
    assert scale > 0
    assert np.abs(fact - direct).max() <= tol * scale
    if precision == "fp64" and case != "slab":
        gm = o.g_sphere(p.cell, p.qpoints[iq].q_red, p.ecut_chi)
        ref = o.chi0(p, iq, om, Q(iq, gm))
        assert np.abs(fact - ref).max() <= 1e-11 * np.abs(ref).max()
