"""The multi-rank paths on CPU, as gloo ranks:
  - batches of independent lattices are split by node count (LPT) with no
    data exchange; every rank derives the same partition on its own, and the
    ranks' shares, stepped through the oracle, gather to the unsharded result
    bit for bit;
  - one lattice split into x-slabs exchanges, per face and step, the nine
    populations of its edge column and the density of the next column, and
    equals the single-domain oracle bit for bit."""
import os
import socket

import numpy as np
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


# ------------------------------------------------------------- sharded batch

def _uneven_batch():
    from tests.cases import small_spec
    shapes = [(40, 24), (17, 9), (33, 20), (24, 24), (9, 31), (28, 12)]
    return [small_spec(nx, ny, seed=100 + i, walls=(i % 3 == 0)) for i, (nx, ny) in enumerate(shapes)]


def _oracle_densities(specs, steps):
    from tests.cases import oracle_from_spec
    out = {}
    for s in specs:
        L = oracle_from_spec(s)
        L.step(steps)
        out[id(s)] = L.moments()[0]
    return out


def _shard_worker(rank, world, port, q, steps):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = _uneven_batch()
    parts = lpt_partition([s.nodes for s in specs], world)
    dens = _oracle_densities([specs[i] for i in parts[rank]], steps)
    # one flat vector per rank, lattices in ascending index order, padded to
    # the batch's total size so that every rank sends the same shape
    total = sum(s.nodes for s in specs)
    flat = torch.full((total,), float("nan"), dtype=torch.float64)
    pos = 0
    for i in parts[rank]:
        v = torch.from_numpy(dens[id(specs[i])].ravel())
        flat[pos:pos + v.numel()] = v
        pos += v.numel()
    got = [torch.zeros_like(flat) for _ in range(world)]
    dist.all_gather(got, flat)   # the read-out gather; stepping exchanged nothing
    if rank == 0:
        q.put([g.numpy() for g in got])
    dist.barrier()
    dist.destroy_process_group()


def _spawn(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


def test_sharded_batch_gathers_the_unsharded_result_bitwise():
    """Each gloo rank advances only its LPT share of an uneven batch (walled
    and periodic lattices) through the oracle; the gathered densities equal
    the run of the whole batch in one process, bit for bit."""
    world, steps = 2, 6
    got = _spawn(_shard_worker, world, steps)
    specs = _uneven_batch()
    ref = _oracle_densities(specs, steps)
    parts = lpt_partition([s.nodes for s in specs], world)
    assert all(parts)
    for r in range(world):
        pos = 0
        for i in parts[r]:
            n = specs[i].nodes
            assert np.array_equal(got[r][pos:pos + n], ref[id(specs[i])].ravel()), (r, i)
            pos += n


# ------------------------------------------------------------- x-slab split

def _slab_spec():
    """One lattice for the x-slab split: a bubble between two walls, with
    noise, so that every column differs."""
    from tests.cases import small_spec
    return small_spec(48, 22, tr=0.6, walls=True, seed=314, shape="bubble")


def _slab_bounds(nx, world):
    cuts = [round(nx * r / world) + (3 if r == 1 else 0) for r in range(world + 1)]
    cuts[-1] = nx
    return cuts


def _xslab_worker(rank, world, port, q, steps):
    """Rank `rank` owns columns [x0, x1) of the lattice. Every step it sends
    its two edge columns' halo to each neighbour: the full nine populations of
    the outermost column and the density of the next one (the pull of the
    neighbour's edge node needs the first, its psi ring the second), runs one
    oracle step on its columns plus two halo columns on each side (a periodic
    lattice of width w + 4; the wrap only touches the halo, which is dropped),
    and keeps its own columns."""
    from oracle import d2q9
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = _slab_spec()
    cuts = _slab_bounds(spec.nx, world)
    x0, x1 = cuts[rank], cuts[rank + 1]
    w, ny = x1 - x0, spec.ny
    full = d2q9.Lattice(spec.nx, spec.ny, a=spec.a, b=spec.b, R=spec.R, T=spec.T, G=spec.G, s=spec.s,
                        eps=spec.eps, solid=spec.solid)
    full.init(spec.rho)
    f = full.f[:, :, x0:x1].copy()          # this rank's state, (9, ny, w)
    solid_ext = np.concatenate([spec.solid[:, :2], spec.solid[:, :w], spec.solid[:, :2]], axis=1)
    ext = d2q9.Lattice(w + 4, ny, a=spec.a, b=spec.b, R=spec.R, T=spec.T, G=spec.G, s=spec.s,
                       eps=spec.eps, solid=solid_ext)
    left, right = (rank - 1) % world, (rank + 1) % world

    def halo(col_outer, col_inner):
        # 9 populations of the outer column, then the density of the inner one
        return torch.from_numpy(np.concatenate([f[:, :, col_outer].ravel(), f[:, :, col_inner].sum(axis=0)]))

    def as_columns(msg):
        m = msg.numpy()
        outer = m[:9 * ny].reshape(9, ny)
        inner = np.zeros((9, ny))
        inner[0] = m[9 * ny:]               # rho as f_0 alone: the oracle's sum9 returns it exactly
        return outer, inner

    for _ in range(steps):
        to_r, to_l = halo(w - 1, w - 2), halo(0, 1)
        from_l, from_r = torch.zeros_like(to_r), torch.zeros_like(to_l)
        reqs = [dist.isend(to_r, right), dist.isend(to_l, left), dist.irecv(from_l, left), dist.irecv(from_r, right)]
        for r_ in reqs:
            r_.wait()
        lo, li = as_columns(from_l)         # left neighbour's columns w_l - 1 (outer) and w_l - 2
        ro, ri = as_columns(from_r)         # right neighbour's columns 0 (outer) and 1
        ext.f[:] = np.concatenate([li[:, :, None], lo[:, :, None], f, ro[:, :, None], ri[:, :, None]], axis=2)
        ext.step(1)
        f = ext.f[:, :, 2:2 + w].copy()
    got = [torch.zeros(9 * ny * spec.nx, dtype=torch.float64) for _ in range(world)]
    mine = torch.zeros(9 * ny * spec.nx, dtype=torch.float64)
    mine.view(9, ny, spec.nx)[:, :, x0:x1] = torch.from_numpy(f)
    dist.all_gather(got, mine)
    if rank == 0:
        q.put(sum(g.numpy() for g in got))
    dist.barrier()
    dist.destroy_process_group()


def test_xslab_split_with_halo_exchange_equals_one_domain_bitwise():
    """Two gloo ranks hold x-slabs of one walled lattice (uneven widths) and
    exchange one population column and one density column per face per step;
    after the steps the gathered distributions equal the single-domain oracle
    bit for bit."""
    from oracle import d2q9
    world, steps = 2, 12
    got = _spawn(_xslab_worker, world, steps).reshape(9, _slab_spec().ny, _slab_spec().nx)
    spec = _slab_spec()
    L = d2q9.Lattice(spec.nx, spec.ny, a=spec.a, b=spec.b, R=spec.R, T=spec.T, G=spec.G, s=spec.s,
                     eps=spec.eps, solid=spec.solid)
    L.init(spec.rho)
    L.step(steps)
    assert np.array_equal(got, L.f)
