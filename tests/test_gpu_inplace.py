"""In-place storage (LBM_INPLACE, the AA pattern) against two-buffer storage
and the oracle.

One array holds the distribution; the state alternates between the natural
layout (after an even number of steps) and the swapped one. The arithmetic
is that of the two-buffer kernels, so every field, every mass and momentum
total equals the two-buffer path's bit for bit, at odd and even step counts,
through CUDA-graph chunks, on walls, obstacles across periodic edges, tiny
lattices and every pseudopotential kind."""
import numpy as np
import pytest

from paper_1605_01800_gb300 import inputs, lbm
from tests.cases import abs_err, fluid, oracle_from_spec, rel_err, small_spec
from tests.test_gpu_eos_variants import spec_for
from tests.test_gpu_parity import obstacle_spec

pytestmark = pytest.mark.gpu


def mixed_batch():
    return [small_spec(70, 45, walls=True, seed=51),           # walls, partial tiles
            small_spec(33, 300, seed=52, shape="bubble"),       # tall, ragged in x
            obstacle_spec(),                                    # solid cells across the periodic edges
            small_spec(5, 3, seed=53),                          # smaller than a tile
            small_spec(1, 9, seed=54),                          # one column: its own x neighbours
            # every kind of psi: van der Waals, Eq. 12 (eps = 1/3), Peng-Robinson, Eq. 12 (eps = 0)
            spec_for("vdw", 40, 24, seed=55), spec_for("psi_exp1", 40, 24, seed=56),
            spec_for("pr", 40, 24, seed=57), spec_for("psi_exp0", 40, 24, seed=58)]


def run(specs, precision, steps, tile=None, stream=None):
    b = lbm.Batch(specs, precision, stream=stream)
    if tile is not None:
        lbm.lbm_set_tile(b.ctx, tile)
    b.init()
    b.step(steps)
    out = [b.moments(i, allow_flags=True) for i in range(len(specs))]
    tot = b.totals(allow_flags=True)
    b.close()
    return out, tot


@pytest.mark.parametrize("precision", ["fp32_dev", "fp32", "fp64"])
@pytest.mark.parametrize("steps", [1, 2, 5, 37])
def test_inplace_equals_two_buffers_bitwise(precision, steps):
    specs = mixed_batch()
    ref, ref_tot = run(specs, precision, steps)
    got, got_tot = run(specs, precision + "_inplace", steps)
    for i in range(len(specs)):
        for name, a, b in zip(("rho", "ux", "uy", "p"), got[i], ref[i]):
            assert np.array_equal(a, b), (i, name)
    # mass and momentum: the post-collision values gathered through the layout
    assert np.array_equal(got_tot, ref_tot)


def test_inplace_graph_replay_equals_two_buffers():
    torch = pytest.importorskip("torch")
    specs = mixed_batch()[:3]
    ref, ref_tot = run(specs, "fp32_dev", 69)
    got, got_tot = run(specs, "fp32_dev_inplace", 69, stream=torch.cuda.Stream())   # 2 chunks + 5 steps
    for i in range(len(specs)):
        for a, b in zip(got[i], ref[i]):
            assert np.array_equal(a, b)
    assert np.array_equal(got_tot, ref_tot)


@pytest.mark.parametrize("tile", [0, 1, 3, 5])
def test_inplace_plain_tiles_agree(tile):
    specs = mixed_batch()[:3]
    ref, _ = run(specs, "fp32_dev", 6)
    got, _ = run(specs, "fp32_dev_inplace", 6, tile=tile)
    for i in range(len(specs)):
        for a, b in zip(got[i], ref[i]):
            assert np.array_equal(a, b)


def test_inplace_matches_oracle():
    spec = small_spec(64, 40, walls=True, seed=57, shape="bubble", R=9.0)
    for steps in (3, 8):
        (rho, ux, uy, p), = run([spec], "fp64_inplace", steps)[0]
        L = oracle_from_spec(spec)
        L.step(steps)
        orho, oux, ouy, op = L.moments()
        m = fluid(spec)
        assert rel_err(rho, orho, m) < 1e-12
        assert abs_err(ux, oux, m) < 1e-13 and abs_err(uy, ouy, m) < 1e-13
        (frho, fux, fuy, _), = run([spec], "fp32_dev_inplace", steps)[0]
        uscale = max(np.abs(oux).max(), np.abs(ouy).max(), 1e-3)
        assert rel_err(frho, orho, m) < 1e-4
        assert abs_err(fux, oux, m) < 1e-4 * uscale and abs_err(fuy, ouy, m) < 1e-4 * uscale


def test_checkpoint_in_either_layout_and_one_lattice_reinitialised():
    specs = [small_spec(48, 40, walls=True, seed=58), small_spec(21, 13, seed=59)]
    other = small_spec(21, 13, seed=60).rho
    results = {}
    for prec in ("fp32_dev", "fp32_dev_inplace"):
        b = lbm.Batch(specs, prec)
        b.init()
        b.step(7)                                    # odd: in place, the swapped layout
        lbm.lbm_init_fields(b.ctx, 1, other)         # one lattice restarts in the current layout
        b.step(4)
        blob_odd = lbm.lbm_save_state(b.ctx) if prec.endswith("inplace") else None
        b.step(3)
        blob_even = lbm.lbm_save_state(b.ctx) if prec.endswith("inplace") else None
        b.step(5)
        results[prec] = [b.moments(i) for i in range(2)]
        b.close()
        if blob_odd is not None:
            for blob, more in ((blob_odd, 8), (blob_even, 5)):
                b2 = lbm.Batch(specs, prec)
                lbm.lbm_load_state(b2.ctx, blob)
                b2.step(more)
                for a, c in zip(results[prec], [b2.moments(i) for i in range(2)]):
                    for x, y in zip(a, c):
                        assert np.array_equal(x, y)
                b2.close()
            # a blob of in-place storage does not load into two-buffer storage
            b3 = lbm.Batch(specs, "fp32_dev")
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_load_state(b3.ctx, blob_odd)
            assert e.value.code == lbm.LBM_EINVAL
            b3.close()
    for a, c in zip(results["fp32_dev"], results["fp32_dev_inplace"]):
        for x, y in zip(a, c):
            assert np.array_equal(x, y)


def test_state_view_reports_the_layout():
    torch = pytest.importorskip("torch")
    spec = small_spec(40, 20, seed=61)
    b = lbm.Batch([spec], "fp32_dev_inplace")
    b.init()
    lbm.lbm_sync(b.ctx)
    arr = lbm.StateArray(b.ctx, 0)
    v = arr.view
    assert v.layout == 1
    # natural layout after init at rest: plane a at each node holds w_a (rho - rho_ref)
    t = torch.as_tensor(arr, device="cuda")[:, v.y0:v.y0 + spec.ny, v.x0:v.x0 + spec.nx].cpu().numpy()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    expect = (w[:, None, None] * (spec.rho - np.float32(spec.rho_ref))[None]).astype(np.float32)
    assert np.allclose(t, expect, rtol=0, atol=2e-8)
    b.step(1)
    assert lbm.lbm_get_state_view(b.ctx, 0).layout == 2
    b.step(1)
    assert lbm.lbm_get_state_view(b.ctx, 0).layout == 1
    b.close()
    b = lbm.Batch([spec], "fp32_dev")
    assert lbm.lbm_get_state_view(b.ctx, 0).layout == 0
    b.close()


def test_inplace_rules_and_memory():
    spec = small_spec(256, 128, seed=62)
    two = lbm.Batch([spec], "fp32_dev")
    one = lbm.Batch([spec], "fp32_dev_inplace")
    i2, i1 = two.info(), one.info()
    assert i1["inplace"] == 1 and i2["inplace"] == 0
    # one distribution array less: 9 planes of (ny + 4) x pitch floats
    pitch = -(-(spec.nx + 34) // 32) * 32
    assert i2["device_bytes"] - i1["device_bytes"] == 4 * ((9 * (spec.ny + 4) * pitch + 63) // 64 * 64)
    n = lbm.lbm_tile_count()
    non_plain = [t for t in range(n) if lbm.lbm_tile_kind(t) != lbm.LBM_TILE_PLAIN]
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_tile(one.ctx, non_plain[0])
    assert e.value.code == lbm.LBM_EINVAL
    one.init()
    best, ms = lbm.lbm_autotune(one.ctx, 2)
    assert lbm.lbm_tile_kind(best) == lbm.LBM_TILE_PLAIN
    assert all(ms[t] < 0 for t in non_plain)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_open_x(one.ctx, 0, None)
    assert e.value.code == lbm.LBM_EINVAL
    one.close()
    two.close()


def test_inplace_flags_psi_domain():
    from oracle import thermo
    Tc = inputs.critical_temperature()
    r0 = thermo.psi_root(0.5 * Tc)
    rho = np.full((8, 8), 0.45)
    rho[3:5, 3:5] = r0 * 1.01
    spec = inputs.LatticeSpec(8, 8, 0.5 * Tc, inputs.relax_rates(0.6), 1.86, rho, rho_ref=0.45)
    for prec in ("fp32_dev_inplace", "fp64_inplace"):
        b = lbm.Batch([spec], prec)
        b.init()
        b.step(1)
        assert b.status(0) & lbm.LBM_FLAG_PSI_CLAMPED
        b.close()
