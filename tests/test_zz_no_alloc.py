"""rpa_logdet_noalloc: the log-det terms of the energy path computed with a
static device scratch array instead of allocations, for callers that may not
allocate device memory.  Its output must match the terms rpa_energy reports for
the same chi0, on two calls in a row (the scratch keeps the previous call's
contents, which must not leak into the next result).

This file is named to be collected last.
"""
import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300 import synthetic as syn
from paper_1307_8052_gb300.build import build

pytestmark = pytest.mark.gpu


def test_logdet_noalloc_matches_energy_terms_twice():
    import torch
    assert torch.cuda.is_available()
    build()
    b.load()
    p = syn.config0()
    om, W = o.frequency_grid(p.nw)
    ctx = b.rpa_create(p.cell, p.grid, p.ecut_chi, p.spin_factor, p.nk_bz, "fp64")
    try:
        b.load_problem(ctx, p)
        E, terms = b.rpa_energy(ctx, [0], [1.0], om, W)
        gm = b.rpa_gvectors(ctx, 0)
        ng = len(gm)
        chi = torch.zeros((len(om), ng, ng), dtype=torch.complex128, device="cuda")
        b.rpa_chi0(ctx, 0, om, chi)
        torch.cuda.synchronize()
    finally:
        b.rpa_destroy(ctx)
    v = torch.from_numpy(o.coulomb(p.cell, p.qpoints[0].q_red, gm)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full((len(om),), float("nan"), dtype=torch.float64, device="cuda")
        b.rpa_logdet_noalloc(chi, v, out, stream)
        got = out.cpu().numpy()
        # FP64 mode tolerance of the parity tests
        assert np.abs(got - terms[0]).max() < 1e-10 * np.abs(terms[0]).max(), call
    # a different, smaller problem in between must not disturb the next result
    small = chi[:2, :50, :50].contiguous()
    out2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    b.rpa_logdet_noalloc(small, v[:50].contiguous(), out2, stream)
    out = torch.zeros(len(om), dtype=torch.float64, device="cuda")
    b.rpa_logdet_noalloc(chi, v, out, stream)
    assert np.abs(out.cpu().numpy() - terms[0]).max() < 1e-10 * np.abs(terms[0]).max()


def test_logdet_noalloc_rejects_oversize_and_host_pointers():
    import torch
    build()
    b.load()
    big = torch.zeros((17, 256, 256), dtype=torch.complex128, device="cuda")   # 17 * 256^2 > 2^20
    v = torch.ones(256, dtype=torch.float64, device="cuda")
    out = torch.zeros(17, dtype=torch.float64, device="cuda")
    with pytest.raises(b.RpaError) as e:
        b.rpa_logdet_noalloc(big, v, out)
    assert e.value.status == b.RPA_ERR_ARG
    with pytest.raises(b.RpaError) as e:
        b.rpa_logdet_noalloc(big[:1].cpu(), v.cpu(), out[:1].cpu())
    assert e.value.status == b.RPA_ERR_ARG


def test_logdet_noalloc_rejects_memory_of_another_device():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second visible GPU")
    build()
    b.load()
    torch.cuda.set_device(0)
    chi = torch.zeros((1, 8, 8), dtype=torch.complex128, device="cuda:1")
    v = torch.ones(8, dtype=torch.float64, device="cuda:1")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:1")
    with pytest.raises(b.RpaError) as e:
        b.rpa_logdet_noalloc(chi, v, out)
    assert e.value.status == b.RPA_ERR_ARG
