"""Multi-rank host logic on CPU (gloo, world size 2): sharding balance and the
gather of per-rank results; no GPU involved."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2303_08123_b300 import parallel
from synth import workloads


def _fake_sim(protocols, L, R):
    # stands in for the simulator: a deterministic function of the inputs
    return [sum(d) * 10.0 + float(l) + 0.5 * float(r) for (d, _), l, r in zip(protocols, L, R)]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, R, prot = workloads.ragged_batch(37, seed=11)
    res = parallel.evaluate(prot, L, R, _fake_sim, rank, world)
    out[rank] = res.tolist()
    dist.barrier()
    dist.destroy_process_group()


def test_shard_balances_cost_and_covers_everything():
    L, R, prot = workloads.ragged_batch(200, seed=1)
    cost = parallel.protocol_cost(L, prot)
    shards, loads = parallel.shard(cost, 3)
    assert sorted(i for s in shards for i in s) == list(range(200))
    assert loads.max() - loads.min() <= cost.max()  # greedy bound: within one job of balance


def test_two_gloo_ranks_gather_the_full_result():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    manager = mp.Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    L, R, prot = workloads.ragged_batch(37, seed=11)
    want = np.array(_fake_sim(prot, L, R))
    for r in range(2):
        np.testing.assert_array_equal(np.array(out[r]), want)
