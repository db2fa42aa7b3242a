"""Multi-rank path on CPU: subtree sharding of the DFS order across ranks
with one FP64 sum-reduce (gloo, world size 2).  Each rank's engine here is
the oracle (the CUDA engine needs a GPU); the test pins the sharding and
the reduction, which are the only multi-rank logic."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import paper_2508_04880_b300 as T
import tusq_workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        circ = W.random_layers(5, 10, 1, 2e-2, 5e-2)
        plan = T.plan(circ, 5000, 3, prune=False)
        part = plan.shard(rank, world)
        inst, counts, w, lcp = part.instances()
        local = oracle.run_instances(circ, inst, w) if inst else np.zeros(1 << circ.n_qubits)
        t = torch.from_numpy(local)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        if rank == 0:
            np.save(out_path, t.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_subtree_shard_reduce(tmp_path):
    out = str(tmp_path / "sum.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    circ = W.random_layers(5, 10, 1, 2e-2, 5e-2)
    ref, _ = oracle.run(circ, 5000, 3, prune=False)
    np.testing.assert_allclose(np.load(out), ref, atol=1e-13)


@pytest.mark.parametrize("world", [1, 2, 3, 7, 500])
def test_shards_partition_the_dfs_order(world):
    circ = W.random_layers(6, 12, 2, 1e-2, 3e-2)
    plan = T.plan(circ, 4000, 1, prune=False)
    inst, counts, w, lcp = plan.instances()
    got_inst, got_w = [], []
    for r in range(world):
        i2, c2, w2, l2 = plan.shard(r, world).instances()
        got_inst += i2
        got_w += list(w2)
        # branch slots inside a chunk are the original ones
        k = len(got_inst) - len(i2)
        assert list(l2) == list(lcp[k:k + max(len(i2) - 1, 0)])
    assert got_inst == inst
    assert np.array_equal(np.array(got_w), w)
