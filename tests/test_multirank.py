"""The multi-rank path on CPU: two gloo ranks shard an uneven batch with no
data exchange; every rank derives the same partition on its own."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1605_01800_gb300 import inputs
from paper_1605_01800_gb300.sharding import lpt_partition, shard


def test_lpt_partition_properties():
    sizes = [inputs.laplace_box(R) ** 2 for R in inputs.laplace_radii()]
    for n in (1, 2, 3, 4, 8):
        parts = lpt_partition(sizes, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert lpt_partition([5, 5, 5], 2) == [[0, 2], [1]]
    assert lpt_partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        lpt_partition([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = inputs.laplace_batch()
    mine = shard(specs, rank, world)
    ids = torch.tensor(sorted(int(round(s.meta["R"] * 1000)) for s in mine) + [-1] * (48 - len(mine)))
    nodes = torch.tensor([sum(s.nodes for s in mine)], dtype=torch.int64)
    all_ids = [torch.zeros_like(ids) for _ in range(world)]
    all_nodes = [torch.zeros_like(nodes) for _ in range(world)]
    # the gathers check the partition; the data path itself exchanges nothing
    dist.all_gather(all_ids, ids)
    dist.all_gather(all_nodes, nodes)
    if rank == 0:
        out.put(([t.tolist() for t in all_ids], [int(t) for t in all_nodes]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_disjointly():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    ids, nodes = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(i for r in ids for i in r if i >= 0)
    want = sorted(int(round(R * 1000)) for R in inputs.laplace_radii())
    assert got == want
    total = sum(s.nodes for s in inputs.laplace_batch())
    assert sum(nodes) == total
    assert abs(nodes[0] - nodes[1]) <= 320 * 320
