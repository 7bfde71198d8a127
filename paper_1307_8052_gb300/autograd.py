"""torch.autograd.Function around rpa_energy / rpa_energy_backward.

``RpaEnergy.apply(engine, C_0, ..., C_{n-1}, P_0, ..., P_{n-1})`` returns E_c as
a 0-d float64 tensor; its backward runs the library's adjoint kernels (no
autograd graph through the CUDA path) and returns dE/dC and dE/dP in the
PyTorch complex convention (the library's convention).  Tensors may live on
the host or on the GPU; gradients come back on the same device as the inputs.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as b


class RpaEngine:
    """A library context with the fixed part of a problem: k-points, Miller
    indices, band energies, occupations, q-points and PAW functions Q."""

    def __init__(self, problem, precision="fp64", device=0, paw_Q=None):
        self.p = problem
        self.ctx = b.rpa_create(problem.cell, problem.grid, problem.ecut_chi, problem.spin_factor, problem.nk_bz,
                                precision, device=device)
        self.paw_Q = paw_Q
        b.load_problem(self.ctx, problem, paw_Q=paw_Q)
        self.iqs = list(range(len(problem.qpoints)))
        self.wq = [qp.weight for qp in problem.qpoints]
        self.omega, self.W = b.rpa_gauss_legendre(problem.nw, 1.0)

    def upload(self, Cs, Ps):
        p = self.p
        Cs = [c.detach().contiguous() for c in Cs]
        Ps = [q.detach().contiguous() for q in Ps] if Ps is not None else None
        if Cs[0].is_cuda:
            # the library reads on its own stream: torch's pending work must be done
            torch.cuda.synchronize()
        for i, s in enumerate(p.sets):
            b.rpa_set_orbitals(self.ctx, i, s.k_red, s.miller, Cs[i], s.eps, s.f)
            if Ps is not None and p.paw is not None:
                b.rpa_set_paw(self.ctx, i, p.paw.nproj, Ps[i])

    def close(self):
        if self.ctx is not None:
            b.rpa_destroy(self.ctx)
            self.ctx = None


class RpaEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, engine: RpaEngine, *tensors):
        n = len(engine.p.sets)
        Cs = list(tensors[:n])
        Ps = list(tensors[n:]) if len(tensors) > n else None
        engine.upload(Cs, Ps)
        E, _ = b.rpa_energy(engine.ctx, engine.iqs, engine.wq, engine.omega, engine.W)
        fctx.engine = engine
        fctx.n = n
        fctx.has_P = Ps is not None
        fctx.save_for_backward(*tensors)
        return torch.tensor(E, dtype=torch.float64, device=Cs[0].device)

    @staticmethod
    def backward(fctx, grad_E):
        engine = fctx.engine
        tensors = fctx.saved_tensors
        n = fctx.n
        Cs = list(tensors[:n])
        Ps = list(tensors[n:]) if fctx.has_P else None
        engine.upload(Cs, Ps)
        dC = [torch.empty_like(c) for c in Cs]
        dP = [torch.empty_like(q) for q in Ps] if Ps is not None else None
        if dC[0].is_cuda:
            torch.cuda.synchronize()
        # the library writes every output element and synchronises its stream before returning
        b.rpa_energy_backward(engine.ctx, engine.iqs, engine.wq, engine.omega, engine.W, float(grad_E.item()),
                              list(range(n)), dC, dP)
        grads = [None] + dC + (dP if dP is not None else [])
        return tuple(grads)
