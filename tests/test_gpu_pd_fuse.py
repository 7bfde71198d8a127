"""The fused middle/fastest-axis pair-density kernel (stages B and C of the
pruned transform of Eq. 10 in one kernel through shared memory) against the
two-kernel form through global memory: the same products in the same order,
so chi0 must be bit-identical, in FP64 and in the mixed modes, on geometries
where a whole pair fits in one block (bulk), where the first axis is split
into several slabs (slab geometry, 200-point third axis) and with umklapp."""
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
@pytest.mark.parametrize("precision", ["fp64", "bf16x2"])
def test_fused_pair_density_stages_bit_identical(case, precision):
    p = _cases()[case]
    iq = 1 if case == "mesh" else 0
    om, _ = o.frequency_grid(4)
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, precision)
    try:
        b.load_problem(ctx, p, paw_Q=lambda i, gm: syn.paw_Q(p.paw, p.cell, p.qpoints[i].q_red, gm))
        # direct middle axis in both forms (the factorised one is a different sum)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_FACT, 0)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_FUSE, 1)
        fused = b.rpa_chi0(ctx, iq, om)
        b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_FUSE, 0)
        split = b.rpa_chi0(ctx, iq, om)
        with pytest.raises(b.RpaError) as e:
            b.rpa_set_tuning(ctx, b.RPA_TUNE_PD_FUSE, 2)
        assert e.value.status == b.RPA_ERR_ARG
    finally:
        b.rpa_destroy(ctx)
    assert np.array_equal(fused, split)
    assert np.abs(fused).max() > 0
