"""One k-block-sized case of the bulk workload, for kernel profiling.

q = (0, 1/2, 1/2) of the 9-bohr bulk box with the two k-transitions
Gamma -> (0, 1/2, 1/2) (no umklapp) and (0, 1/2, 1/2) -> Gamma (umklapp (0, 1, 1)),
16 occupied + 1200 empty bands per set, 3 x 13 PAW projectors, 16 frequencies:
each launch of the rank-k kernel is exactly one launch of the bench's workload.

Usage: python -m paper_1307_8052_gb300.profile_case [fold] [reps] [chi|energy] [precision] [fuse] [pair] [pipe]
"""
from __future__ import annotations

import sys

import numpy as np

from . import binding as b
from . import synthetic as syn


def main(argv):
    fold = int(argv[1]) if len(argv) > 1 else 1
    reps = int(argv[2]) if len(argv) > 2 else 1
    mode = argv[3] if len(argv) > 3 else "chi"
    precision = argv[4] if len(argv) > 4 else "bf16x2"
    fuse = int(argv[5]) if len(argv) > 5 else 1
    pair = int(argv[6]) if len(argv) > 6 else 0
    pipe = int(argv[7]) if len(argv) > 7 else 0
    b.load()
    cell = np.eye(3) * 9.0
    ks = {0: np.zeros(3), 3: np.array([0.0, 0.5, 0.5])}
    sets = {i: syn.make_orbitals(1, i, cell, k, 20.0, 16, 1200) for i, k in ks.items()}
    paw = syn.make_paw_setup(1, [13, 13, 13])
    ctx = b.rpa_create(cell, (40, 40, 40), 10.5, 2.0, 8, precision)
    for i, s in sets.items():
        b.rpa_set_orbitals(ctx, i, s.k_red, s.miller, s.C, s.eps, s.f)
        b.rpa_set_paw(ctx, i, paw.nproj, syn.make_projections(1, i, 1216, 39))
    q = np.array([0.0, 0.5, 0.5])
    b.rpa_set_qpoint(ctx, 0, q, [0, 3], [3, 0], [[0, 0, 0], [0, 1, 1]])
    b.rpa_set_paw_Q(ctx, 0, paw.nproj, syn.paw_Q(paw, cell, q, b.rpa_gvectors(ctx, 0)))
    b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FOLD, fold)
    b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_FUSE, fuse)
    b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PAIR, pair)
    b.rpa_set_tuning(ctx, b.RPA_TUNE_TC_PIPE, pipe)
    om, W = b.rpa_gauss_legendre(16)
    b.rpa_set_profiling(ctx, True)
    for _ in range(reps):
        if mode == "energy":
            b.rpa_energy(ctx, [0], [1.0], om, W)
        else:
            b.rpa_chi0(ctx, 0, om)
        ms, _ = b.rpa_get_profile(ctx)
        print(f"{precision} fold {fold} fuse {fuse} pair {pair} pipe {pipe} stage ms {np.round(ms, 2).tolist()}", flush=True)
    b.rpa_destroy(ctx)


if __name__ == "__main__":
    main(sys.argv)
