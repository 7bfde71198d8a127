"""The multi-process path on CPU: two gloo ranks shard the q-points of one
problem, evaluate their share with the oracle, and the summed E_c equals the
single-process result; the step-time reduction takes the maximum."""
import os
import socket

import numpy as np
import pytest

from paper_1307_8052_gb300 import shard


def test_shard_assigns_every_q_once_and_balances():
    costs = [5.0, 1.0, 4.0, 2.0, 3.0, 3.0, 1.0, 9.0]
    for world in (1, 2, 3, 8, 11):
        parts = shard.shard_qpoints(costs, world)
        assert len(parts) == world
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in shard.shard_qpoints(costs, 2)]
    assert max(loads) - min(loads) <= max(costs)
    assert shard.shard_qpoints(costs, 2) == shard.shard_qpoints(costs, 2)
    with pytest.raises(ValueError):
        shard.shard_qpoints(costs, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import oracle as o
    from paper_1307_8052_gb300 import synthetic as syn
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        p = syn.small_problem(config_tag=97, nunocc=8, nw=4)
        om, W = o.frequency_grid(p.nw)
        Qs = {}
        for iq, qp in enumerate(p.qpoints):
            gm = o.g_sphere(p.cell, qp.q_red, p.ecut_chi)
            Qs[iq] = syn.paw_Q(p.paw, p.cell, qp.q_red, gm)
        costs = [len(o.g_sphere(p.cell, qp.q_red, p.ecut_chi)) ** 2 * len(qp.k_of) for qp in p.qpoints]
        wq = [qp.weight for qp in p.qpoints]

        def evaluate(iqs, wqs):
            # the oracle's energy with the weights the step hands over
            sub = [p.qpoints[i].weight for i in iqs]
            assert np.allclose(sub, wqs)
            E, _ = o.energy(p, om, W, Qs=Qs, iqs=iqs)
            return E

        E = shard.sharded_energy(evaluate, costs, wq, rank, world)
        # the step function the bench runs, over the q-points in a permuted
        # order (costs and weights aligned with that order)
        order = list(range(len(p.qpoints)))[::-1]
        E_step = shard.sharded_step(evaluate, order, [costs[i] for i in order], [wq[i] for i in order], rank, world)
        mine = shard.partition(order, [costs[i] for i in order], world)[rank]
        E_rep = shard.sharded_step(evaluate, order, [costs[i] for i in order], [wq[i] for i in order], rank, world,
                                   replicas=True)
        t = shard.max_over_ranks(1.0 + rank)
        out[rank] = (E, t, E_step, mine, E_rep)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_sharded_energy():
    import multiprocessing as mp
    import oracle as o
    from paper_1307_8052_gb300 import synthetic as syn
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=240)
        codes = [pr.exitcode for pr in procs]
        for pr in procs:
            if pr.is_alive():
                pr.kill()
        assert codes == [0, 0], codes
        res = dict(out)
    p = syn.small_problem(config_tag=97, nunocc=8, nw=4)
    om, W = o.frequency_grid(p.nw)
    Qs = {iq: syn.paw_Q(p.paw, p.cell, qp.q_red, o.g_sphere(p.cell, qp.q_red, p.ecut_chi))
          for iq, qp in enumerate(p.qpoints)}
    E_ref, _ = o.energy(p, om, W, Qs=Qs)
    shares = []
    for r in range(2):
        E, t, E_step, mine, E_rep = res[r]
        assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
        assert abs(E_step - E_ref) <= 1e-12 * abs(E_ref)
        assert abs(E_rep - E_ref) <= 1e-12 * abs(E_ref)
        assert t == 2.0
        shares.append(mine)
    # the two ranks' shares cover every q-point once
    assert sorted(shares[0] + shares[1]) == list(range(len(p.qpoints)))
    assert shares[0] and shares[1]
