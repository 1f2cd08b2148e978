"""The multi-GPU layout of bench.py on CPU: ranks develop disjoint ranges of
global shower ids with no data exchange (the random streams are keyed by
the global id), and only the timing is reduced across ranks (max).  Two
gloo ranks must reproduce a single run exactly."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_per_rank, out_q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2202_05012_gb300 import inputs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, p = inputs.workload_plain10(n_per_rank * world)
        mine = p[rank * n_per_rank:(rank + 1) * n_per_rank]
        r = oracle.simulate(g, mine, seed=0, shower_id_base=rank * n_per_rank)
        ls = torch.from_numpy(np.ascontiguousarray(r["layer_sum"]))
        hits = torch.tensor([len(r["E"])], dtype=torch.int64)
        gathered = [torch.zeros_like(ls) for _ in range(world)]
        dist.all_gather(gathered, ls)
        dist.all_reduce(hits)
        elapsed = torch.tensor([10.0 + rank], dtype=torch.float64)  # stand-in for a rank's timed region
        dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
        if rank == 0:
            out_q.put((torch.cat(gathered).numpy(), int(hits.item()), float(elapsed.item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_reproduce_one_run():
    import multiprocessing as mp

    import oracle
    from paper_2202_05012_gb300 import inputs

    world, n = 2, 150
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    ls, hits, tmax = q.get(timeout=240)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    g, p = inputs.workload_plain10(n * world)
    full = oracle.simulate(g, p, seed=0)
    assert np.array_equal(ls, full["layer_sum"])
    assert hits == len(full["E"])
    assert tmax == 11.0
