"""One lattice split into x-slabs on the GPU (lbm_set_open_x, lbm_halo_pack,
lbm_halo_unpack): the slabs, stepped with a halo exchange after every step,
equal the undivided lattice bit for bit, in FP32 deviation storage and FP64,
with walls along the cut and slab widths that do not fill whole tiles.

The exchange runs between contexts of one process (device copies) and
between two gloo ranks sharing the one GPU (host copies and point-to-point
messages; the ranks' kernels never wait on each other: every wait is on the
host)."""
import os
import socket

import numpy as np
import pytest

from paper_1605_01800_gb300 import lbm, xslab
from tests.cases import small_spec

pytestmark = pytest.mark.gpu

STEPS = 25


def _spec():
    # a vapour bubble between two walls (rows 0 and ny - 1), with noise
    return small_spec(96, 40, tr=0.6, walls=True, seed=271, shape="bubble", R=12.0)


def _whole(spec, precision, steps, momentum=False):
    b = lbm.Batch([spec], precision)
    b.init()
    b.step(steps)
    out = b.moments(0)
    mass = b.mass(0)
    mom = b.momentum(0)
    b.close()
    return (out, mass, mom) if momentum else (out, mass)


def _first_of(kind):
    return next(t for t in range(lbm.lbm_tile_count()) if lbm.lbm_tile_kind(t) == kind)


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("precision,kind", [("fp32_dev", lbm.LBM_TILE_PLAIN), ("fp32_dev", lbm.LBM_TILE_TMA),
                                            ("fp32_dev", lbm.LBM_TILE_PIPELINED), ("fp64", lbm.LBM_TILE_PLAIN)])
def test_slabs_in_one_process_equal_the_whole_lattice(precision, kind, overlap):
    """Every step-kernel kind on the slabs (the TMA and pipelined kernels take
    the slabs' interior tiles, the plain kernel's general path the tiles
    along the cuts); with overlap, each step split into the tiles along the
    cuts and the rest, the exchange on a second stream beside the rest."""
    spec = _spec()
    ref, mass, mom = _whole(spec, precision, STEPS, momentum=True)
    slabs = xslab.LocalSlabs(spec, [0, 37, 59, 96], precision, overlap=overlap)   # widths 37, 22, 37
    tile = 1 if kind == lbm.LBM_TILE_PLAIN else _first_of(kind)
    for s in slabs.slabs:
        lbm.lbm_set_tile(s.batch.ctx, tile)
    slabs.step(STEPS)
    got = slabs.moments()
    for name, a, b in zip(("rho", "ux", "uy", "p"), got, ref):
        assert np.array_equal(a, b), name
    # the mass of the stored state adds up across the slabs
    assert sum(s.batch.mass(0) for s in slabs.slabs) == pytest.approx(mass, rel=1e-12)
    # and so does the momentum, the force at the cut taken from the halo
    for k in range(2):
        assert sum(s.batch.momentum(0)[k] for s in slabs.slabs) == pytest.approx(mom[k], abs=1e-12 * mass)
    slabs.close()


@pytest.mark.parametrize("overlap", [False, True])
def test_narrow_slabs_equal_the_whole_lattice(overlap):
    """Five slabs, two of them at the minimum width of 2 columns and one of
    3: every node of those slabs is an edge node whose pulls and psi ring
    reach into both neighbours' halos (with overlap their whole step is the
    edge part)."""
    spec = _spec()
    ref, _ = _whole(spec, "fp32_dev", STEPS)
    slabs = xslab.LocalSlabs(spec, [0, 2, 5, 40, 42, 96], "fp32_dev", overlap=overlap)
    slabs.step(STEPS)
    for name, a, b in zip(("rho", "ux", "uy", "p"), slabs.moments(), ref):
        assert np.array_equal(a, b), name
    slabs.close()


def test_open_lattice_rules():
    spec = _spec()
    slab, rho_ext, halo = xslab.cut(spec, 0, 48)
    b = lbm.Batch([slab], "fp32_dev")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_halo_pack(b.ctx, 0, 0, 1)           # not open yet
    assert e.value.code == lbm.LBM_EINVAL
    lbm.lbm_set_open_x(b.ctx, 0, halo)
    b.init([rho_ext])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_step(b.ctx, 2)                      # a halo exchange is due after every step
    with pytest.raises(lbm.LbmError):
        lbm.lbm_init_fields_all(b.ctx, np.ascontiguousarray(slab.rho.ravel()))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_halo_pack(b.ctx, 0, 2, 1)           # side 0 or 1
    lbm.lbm_step(b.ctx, 1)
    b.close()
    auto = small_spec(16, 8, seed=3)
    auto.rho_ref = -1.0                             # automatic reference: refused for a slab
    b = lbm.Batch([auto], "fp32_dev")
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_open_x(b.ctx, 0, None)
    b.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_step_equals_one_step():
    """lbm_step_part on a batch with and without x-slabs: both orders of the
    parts give lbm_step's result bit for bit; the rules of a split step."""
    specs = [small_spec(70, 45, walls=True, seed=81), small_spec(33, 20, seed=82)]
    ref = lbm.Batch(specs, "fp32_dev")
    ref.init()
    ref.step(6)
    want = [ref.moments(i) for i in range(2)]
    ref.close()
    for order in ((lbm.LBM_STEP_EDGE, lbm.LBM_STEP_INTERIOR), (lbm.LBM_STEP_INTERIOR, lbm.LBM_STEP_EDGE)):
        b = lbm.Batch(specs, "fp32_dev")
        b.init()
        for _ in range(6):
            for part in order:
                lbm.lbm_step_part(b.ctx, part)
        assert b.info()["steps"] == 6
        for i in range(2):
            for x, y in zip(b.moments(i), want[i]):
                assert np.array_equal(x, y)
        lbm.lbm_step_part(b.ctx, lbm.LBM_STEP_EDGE)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step_part(b.ctx, lbm.LBM_STEP_EDGE)       # the same part twice
        assert e.value.code == lbm.LBM_EINVAL
        with pytest.raises(lbm.LbmError):
            lbm.lbm_step(b.ctx, 1)                           # a split step is half done
        with pytest.raises(lbm.LbmError):
            lbm.lbm_step_part(b.ctx, 3)
        for call in (lambda: lbm.lbm_set_tile(b.ctx, 1), lambda: lbm.lbm_save_state(b.ctx),
                     lambda: lbm.lbm_autotune(b.ctx, 1), lambda: b.init()):
            with pytest.raises(lbm.LbmError) as e:
                call()                                       # state and tiles wait for the second part
            assert e.value.code == lbm.LBM_EINVAL
        lbm.lbm_step_part(b.ctx, lbm.LBM_STEP_INTERIOR)
        lbm.lbm_step(b.ctx, 1)
        b.close()
    # a pack during a split step needs its edge part first
    slab, rho_ext, halo = xslab.cut(_spec(), 0, 48)
    b = lbm.Batch([slab], "fp32_dev")
    lbm.lbm_set_open_x(b.ctx, 0, halo)
    b.init([rho_ext])
    torch = pytest.importorskip("torch")
    buf = torch.empty(lbm.LBM_HALO_ROWS * slab.ny, dtype=torch.float32, device="cuda")
    lbm.lbm_step_part(b.ctx, lbm.LBM_STEP_INTERIOR)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_halo_pack(b.ctx, 0, 0, buf.data_ptr())
    assert e.value.code == lbm.LBM_EINVAL
    lbm.lbm_step_part(b.ctx, lbm.LBM_STEP_EDGE)
    lbm.lbm_halo_pack(b.ctx, 0, 0, buf.data_ptr())
    b.close()


def _rank(rank, world, port, q, steps, overlap=False):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    spec = _spec()
    cuts = [0, 41, 96]
    mine = xslab.RankSlab(spec, "fp32_dev", cuts=cuts, overlap=overlap)
    mine.step(steps)
    # each rank's columns in a whole-lattice array, zero elsewhere (equal
    # shapes for the gather; the sum over ranks is exact)
    full = torch.zeros((spec.ny, spec.nx), dtype=torch.float64)
    full[:, cuts[rank]:cuts[rank + 1]] = torch.from_numpy(mine.moments()[0].copy())
    got = [torch.zeros_like(full) for _ in range(world)]
    dist.all_gather(got, full)
    if rank == 0:
        q.put(sum(g.numpy() for g in got))
    mine.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("overlap", [False, True])
def test_two_gloo_ranks_on_one_gpu_equal_the_whole_lattice(overlap):
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, STEPS, overlap)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (ref, _, _, _), _ = _whole(_spec(), "fp32_dev", STEPS)
    assert np.array_equal(got, ref)
