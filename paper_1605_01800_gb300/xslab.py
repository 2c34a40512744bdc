"""One lattice split into x-slabs, one context per slab (``include/lbm.h``:
``lbm_set_open_x``, ``lbm_halo_pack``, ``lbm_halo_unpack``).

A step reads a node's neighbours up to two columns away, so the slabs of a
lattice exchange, per face and step, 12 values per row (the halo the library
packs). This module only orchestrates: it cuts the slab specs out of a
whole-lattice spec and moves the packed halos, either between contexts on one
device (``LocalSlabs``, device-to-device through buffers on the contexts'
common stream) or between ranks, one slab per rank in rank order along x
(``RankSlab``, ``torch.distributed`` point-to-point: device buffers under
NCCL, host copies under gloo). Every arithmetic step runs in the library's
kernels.

With ``overlap=True`` each step is split (``lbm_step_part``): the tiles
next to the cuts first, then the halo is packed, exchanged and unpacked on a
stream of its own while the rest of the step runs; the next step waits for
the unpack. The result is bitwise the same.
"""
from dataclasses import replace
from typing import List, Optional, Sequence

import numpy as np

from . import lbm


def cut(spec, x0: int, x1: int):
    """The slab [x0, x1) of a lattice that is periodic in x.

    Returns (slab spec, initial density of (ny, x1 - x0 + 2) values: the
    slab's columns with the neighbouring edge columns x0 - 1 and x1 on either
    side, halo mask of (4, ny) bytes for columns x0 - 2, x0 - 1, x1, x1 + 1 or
    None without walls)."""
    nx = spec.nx
    if not 0 <= x0 < x1 <= nx:
        raise ValueError(f"slab [{x0}, {x1}) is not inside 0 .. {nx}")
    cols = np.arange(x0 - 1, x1 + 1) % nx
    rho_ext = np.ascontiguousarray(spec.rho[:, cols])
    solid = None if spec.solid is None else np.ascontiguousarray(spec.solid[:, x0:x1])
    halo = None
    if spec.solid is not None:
        hc = [(x0 - 2) % nx, (x0 - 1) % nx, x1 % nx, (x1 + 1) % nx]
        halo = np.ascontiguousarray(spec.solid[:, hc].T, dtype=np.uint8)
    slab = replace(spec, nx=x1 - x0, rho=np.ascontiguousarray(spec.rho[:, x0:x1]), solid=solid)
    return slab, rho_ext, halo


def even_cuts(nx: int, n: int) -> List[int]:
    """Column boundaries of n slabs of nearly equal width."""
    return [round(nx * k / n) for k in range(n + 1)]


class _Slab:
    def __init__(self, spec, x0, x1, precision, stream):
        import torch
        self.slab, rho_ext, halo = cut(spec, x0, x1)
        self.x0, self.x1 = x0, x1
        self.batch = lbm.Batch([self.slab], precision, stream=stream)
        lbm.lbm_set_open_x(self.batch.ctx, 0, halo)
        self.batch.init([rho_ext])
        dtype = torch.float64 if self.batch.precision == lbm.LBM_FP64 else torch.float32
        n = lbm.LBM_HALO_ROWS * self.slab.ny
        self.out = [torch.empty(n, dtype=dtype, device="cuda") for _ in range(2)]   # packed for side 0, 1
        self.inc = [torch.empty(n, dtype=dtype, device="cuda") for _ in range(2)]   # received from side 0, 1

    def pack(self, stream=None):
        h = stream.cuda_stream if stream is not None else 0
        for side in (0, 1):
            lbm.lbm_halo_pack(self.batch.ctx, 0, side, self.out[side].data_ptr(), h)

    def unpack(self, stream=None):
        h = stream.cuda_stream if stream is not None else 0
        for side in (0, 1):
            lbm.lbm_halo_unpack(self.batch.ctx, 0, side, self.inc[side].data_ptr(), h)


class LocalSlabs:
    """The slabs of one lattice as contexts on the current device, stepped
    together; halos move by device copies on the contexts' common stream."""

    def __init__(self, spec, cuts: Sequence[int], precision="fp32_dev", stream=None, overlap=False):
        import torch
        self.spec = spec
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.overlap = overlap
        self.comm = torch.cuda.Stream() if overlap else self.stream
        self.slabs = [_Slab(spec, a, b, precision, self.stream) for a, b in zip(cuts[:-1], cuts[1:])]
        self.exchange(self.stream)

    def exchange(self, stream):
        import torch
        n = len(self.slabs)
        with torch.cuda.stream(stream):
            for s in self.slabs:
                s.pack(stream)
            for k, s in enumerate(self.slabs):
                s.inc[0].copy_(self.slabs[(k - 1) % n].out[1])   # the left neighbour's right side
                s.inc[1].copy_(self.slabs[(k + 1) % n].out[0])   # the right neighbour's left side
            for s in self.slabs:
                s.unpack(stream)

    def step(self, n: int = 1):
        import torch
        for _ in range(n):
            if not self.overlap:
                for s in self.slabs:
                    s.batch.step(1)
                self.exchange(self.stream)
                continue
            for s in self.slabs:
                lbm.lbm_step_part(s.batch.ctx, lbm.LBM_STEP_EDGE)
            edge_done = torch.cuda.Event()
            edge_done.record(self.stream)
            self.comm.wait_event(edge_done)
            self.exchange(self.comm)                       # runs beside the interior tiles
            for s in self.slabs:
                lbm.lbm_step_part(s.batch.ctx, lbm.LBM_STEP_INTERIOR)
            unpacked = torch.cuda.Event()
            unpacked.record(self.comm)
            self.stream.wait_event(unpacked)               # the next step reads the frames

    def moments(self, allow_flags=False):
        """(rho, ux, uy, p) of the whole lattice, (ny, nx) each."""
        parts = [s.batch.moments(0, allow_flags=allow_flags) for s in self.slabs]
        return tuple(np.concatenate([p[k] for p in parts], axis=1) for k in range(4))

    def close(self):
        for s in self.slabs:
            s.batch.close()


class RankSlab:
    """This rank's slab of a lattice split across the ranks of the default
    process group, one slab per rank in rank order along x. exchange() sends
    the packed halos to both neighbours and unpacks theirs: device buffers
    under NCCL, host copies under gloo. The sends and receives are posted in
    an order that pairs them correctly also when both neighbours are the same
    rank (two ranks)."""

    def __init__(self, spec, precision="fp32_dev", cuts: Optional[Sequence[int]] = None, stream=None,
                 overlap=False):
        import torch
        import torch.distributed as dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        cuts = list(cuts) if cuts is not None else even_cuts(spec.nx, self.world)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.overlap = overlap
        self.comm = torch.cuda.Stream() if overlap else self.stream
        self.slab = _Slab(spec, cuts[self.rank], cuts[self.rank + 1], precision, self.stream)
        self.host = dist.get_backend() != "nccl"
        self.exchange(self.stream)

    def exchange(self, stream, before_wait=None):
        """Pack, send and receive, unpack, all on `stream`; `before_wait`
        (if given) is called once the sends and receives are posted, before
        anything waits for them."""
        import torch
        import torch.distributed as dist
        s = self.slab
        left, right = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        # everything on `stream`: under NCCL the sends read the packed
        # buffers after the pack, and wait() orders the unpack after the
        # receives; under gloo the copies to the host synchronise it
        with torch.cuda.stream(stream):
            s.pack(stream)
            if before_wait is not None and self.host:
                before_wait()    # the copies to the host below block this thread
                before_wait = None
            if self.host:
                out = [t.cpu() for t in s.out]
                inc = [torch.empty_like(t) for t in out]
            else:
                out, inc = s.out, s.inc
            ops = [dist.P2POp(dist.isend, out[1], right, tag=1), dist.P2POp(dist.irecv, inc[0], left, tag=1),
                   dist.P2POp(dist.isend, out[0], left, tag=0), dist.P2POp(dist.irecv, inc[1], right, tag=0)]
            reqs = dist.batch_isend_irecv(ops)
            if before_wait is not None:
                before_wait()
            for r in reqs:
                r.wait()
            if self.host:
                s.inc[0].copy_(inc[0])
                s.inc[1].copy_(inc[1])
            s.unpack(stream)

    def step(self, n: int = 1):
        import torch
        ctx = self.slab.batch.ctx
        for _ in range(n):
            if not self.overlap:
                self.slab.batch.step(1)
                self.exchange(self.stream)
                continue
            lbm.lbm_step_part(ctx, lbm.LBM_STEP_EDGE)
            edge_done = torch.cuda.Event()
            edge_done.record(self.stream)
            self.comm.wait_event(edge_done)
            # the interior tiles are launched before anything waits for the
            # messages, so they run while the halo travels
            self.exchange(self.comm, before_wait=lambda: lbm.lbm_step_part(ctx, lbm.LBM_STEP_INTERIOR))
            unpacked = torch.cuda.Event()
            unpacked.record(self.comm)
            self.stream.wait_event(unpacked)

    def moments(self, allow_flags=False):
        return self.slab.batch.moments(0, allow_flags=allow_flags)

    def close(self):
        self.slab.batch.close()
