"""The FP32 step kernel's L2 prefetch of later tiles changes no result.

A context whose two distribution arrays exceed the device's L2 streams every
step from DRAM, and its step kernel prefetches, about 7 MB ahead, the
populations of the tiles that later CTAs take; a smaller context does not.
Results never depend on it: the same lattices stepped in one large batch
(prefetching) and each in a context of its own (not prefetching) agree bit for
bit, on every plain tile shape, with walls and with ragged tiles."""
import numpy as np
import pytest

from paper_1605_01800_gb300 import lbm
from tests.cases import small_spec

pytestmark = pytest.mark.gpu


def lattices():
    # four lattices of about 1M nodes: 75 MB of distributions each, 300 MB together
    return [small_spec(1024, 1024, seed=71),
            small_spec(1024, 1024, walls=True, seed=72, shape="bubble", R=200.0),
            small_spec(1000, 1030, seed=73),                  # ragged tiles in x and y
            small_spec(1056, 992, walls=True, seed=74)]


def run(specs, tile, steps, precision="fp32_dev"):
    b = lbm.Batch(specs, precision)
    lbm.lbm_set_tile(b.ctx, tile)
    b.init()
    b.step(steps)
    out = [b.moments(i, allow_flags=True) for i in range(len(specs))]
    info = b.info()
    tot = b.totals(allow_flags=True)
    b.close()
    return out, info, tot


@pytest.mark.parametrize("tile", [1, 3, 5])
def test_prefetching_batch_equals_lattices_alone(tile):
    specs = lattices()
    steps = 37   # one CUDA-graph chunk and five single launches
    batch, info, _ = run(specs, tile, steps)
    assert info["l2_prefetch"] == 1
    for i, spec in enumerate(specs):
        alone, info1, _ = run([spec], tile, steps)
        assert info1["l2_prefetch"] == 0
        for name, a, c in zip(("rho", "ux", "uy", "p"), batch[i], alone[0]):
            assert np.array_equal(a, c), (tile, i, name)


def test_prefetch_rule():
    small = lbm.Batch([small_spec(256, 64, seed=75)], "fp32_dev")
    assert small.info()["l2_prefetch"] == 0
    small.close()
    for precision, expect in (("fp32_dev", 1), ("fp32", 1), ("fp32_dev_inplace", 0), ("fp64", 0)):
        b = lbm.Batch(lattices(), precision)
        assert b.info()["l2_prefetch"] == expect, precision
        b.close()


def test_regular_tile_grid_changes_no_result():
    """Lattices alike in size, without walls and covered by whole tiles form a
    regular grid of tiles: the 32 x 16 shapes (four nodes per thread) then
    find their own tile and the tile they prefetch by arithmetic instead of
    loading records. Bit for bit the two-node shapes' result (which load
    records), on an L2-resident batch and on a prefetching one, and the same
    lattices with walls (no grid) agree with themselves across shapes."""
    grid_tiles = [t for t in range(lbm.lbm_tile_count())
                  if lbm.lbm_tile_kind(t) == lbm.LBM_TILE_PLAIN and lbm.lbm_tile_shape(t) == (32, 16)]
    small = [small_spec(256, 64, seed=90 + i, shape="bubble" if i % 2 else "droplet", R=12.0 + i)
             for i in range(4)]
    big = [small_spec(1024, 1024, seed=95), small_spec(1024, 1024, seed=96, shape="bubble", R=150.0)]
    for specs, steps in ((small, 37), (big, 9)):
        ref, info, ref_tot = run(specs, 1, steps)
        assert info["tile_grid"] == 1
        for t in grid_tiles:
            got, info_t, tot = run(specs, t, steps)
            assert info_t["tile_grid"] == 1 and info_t["l2_prefetch"] == info["l2_prefetch"]
            assert np.array_equal(tot, ref_tot), t
            for i in range(len(specs)):
                for name, a, c in zip(("rho", "ux", "uy", "p"), got[i], ref[i]):
                    assert np.array_equal(a, c), (t, i, name)
    # no grid: lattices of different sizes, or walls
    _, info, _ = run([small_spec(256, 64, seed=97), small_spec(128, 64, seed=98)], 3, 2)
    assert info["tile_grid"] == 0
    _, info, _ = run([small_spec(256, 64, walls=True, seed=99)], 3, 2)
    assert info["tile_grid"] == 0
