"""Per-lattice FP64 totals on the GPU (lbm_total_momentum, lbm_totals_all)
against the oracle's sums of j + F/2 (Eq. 6, 7) and the context's own mass.

Tolerances: FP64 storage differs from the oracle only in rounding order, so
the totals agree to 1e-12 of the mass (the scale of the summed magnitudes).
For FP32 storage the bar is the pointwise velocity bar of the parity tests
(1e-4 of the velocity scale, at least 1e-3 in lattice units) summed over the
nodes: |dP| <= 1e-4 * mass * u_scale."""
import numpy as np
import pytest

from paper_1605_01800_gb300 import inputs, lbm
from tests.cases import oracle_from_spec, small_spec

pytestmark = pytest.mark.gpu


def stratified_channel(along_x=False):
    """Walls on two opposite edges, vapour along one and liquid along the
    other (a flat interface between them, parallel to the walls); the total
    momentum at rest is half the walls' reaction."""
    Tc = inputs.critical_temperature()
    c = inputs.coexistence(0.6)
    nx, ny = (64, 20) if along_x else (20, 64)
    n = nx if along_x else ny
    k = np.arange(n, dtype=float)
    prof = 0.5 * (c["rho_l"] + c["rho_g"]) + 0.5 * (c["rho_l"] - c["rho_g"]) * np.tanh((k - 0.4 * n) / 3.0)
    rho = np.tile(prof, (ny, 1)) if along_x else np.tile(prof[:, None], (1, nx))
    solid = np.zeros((ny, nx), np.uint8)
    if along_x:
        solid[:, 0] = solid[:, nx - 1] = 1
    else:
        solid[0, :] = solid[ny - 1, :] = 1
    return inputs.LatticeSpec(nx, ny, 0.6 * Tc, inputs.relax_rates(0.8), 1.86, np.ascontiguousarray(rho),
                              rho_ref=c["rho_g"], solid=solid)


CASES = {
    "droplet_periodic": lambda: small_spec(70, 45, seed=31),
    "bubble_walls": lambda: small_spec(66, 40, tr=0.6, walls=True, seed=32, shape="bubble", R=10.0),
    "channel_y": lambda: stratified_channel(False),
    "channel_x": lambda: stratified_channel(True),
}


def _oracle_totals(spec, steps):
    L = oracle_from_spec(spec)
    L.step(steps)
    _, ux, uy, _ = L.moments()
    return L.mass(), L.momentum(), max(np.abs(ux).max(), np.abs(uy).max(), 1e-3)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dev"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_momentum_matches_oracle(name, precision):
    spec = CASES[name]()
    steps = 60
    b = lbm.Batch([spec], precision)
    b.init()
    b.step(steps)
    px, py = b.momentum(0)
    mass = b.mass(0)
    b.close()
    omass, (opx, opy), uscale = _oracle_totals(spec, steps)
    tol = 1e-12 * omass if precision == "fp64" else 1e-4 * omass * uscale
    assert abs(px - opx) <= tol and abs(py - opy) <= tol, (px, opx, py, opy, tol)
    assert mass == pytest.approx(omass, rel=1e-12 if precision == "fp64" else 1e-6)


def test_channel_at_rest_matches_the_wall_reaction():
    # before any step j = 0, and the total is -G * lines * (psi_last^2 -
    # psi_first^2) / 4 along the channel's normal (the closed form the
    # oracle is pinned to), zero along the walls
    for along_x in (False, True):
        spec = stratified_channel(along_x)
        b = lbm.Batch([spec], "fp64")
        b.init()
        px, py = b.momentum(0)
        b.close()
        L = oracle_from_spec(spec)
        n = spec.nx if along_x else spec.ny
        prof = spec.rho[0, :] if along_x else spec.rho[:, 0]
        lines = spec.ny if along_x else spec.nx
        psi_first, _ = L.psi(prof[1])
        psi_last, _ = L.psi(prof[n - 2])
        normal = -spec.G * lines * (psi_last ** 2 - psi_first ** 2) / 4
        along, across = (px, py) if along_x else (py, px)
        assert along == pytest.approx(normal, rel=1e-12)
        assert abs(across) < 1e-14 * abs(normal)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dev"])
def test_totals_all_equal_the_per_lattice_calls(precision):
    specs = [small_spec(70, 45, walls=True, seed=41), small_spec(130, 9, seed=42), stratified_channel(True),
             small_spec(33, 300, seed=43, shape="bubble")]
    b = lbm.Batch(specs, precision)
    b.init()
    b.step(7)
    t = b.totals()
    assert t.shape == (4, 3)
    for i in range(len(specs)):
        assert t[i, 0] == b.mass(i)                    # bit for bit
        px, py = b.momentum(i)
        assert t[i, 1] == px and t[i, 2] == py
    b.close()


def test_momentum_without_walls_is_kept_with_a_drift():
    # a droplet moving diagonally across a periodic lattice: the total stays
    # at its initial value (Eq. 7 sums to zero, the collision adds F to j)
    spec = small_spec(128, 96, seed=44)
    ux = np.full_like(spec.rho, 0.02)
    uy = np.full_like(spec.rho, -0.01)
    b = lbm.Batch([spec], "fp32_dev")
    lbm.lbm_init_fields(b.ctx, 0, spec.rho, ux, uy)
    p0 = b.momentum(0)
    b.step(2000)
    p1 = b.momentum(0)
    mass = b.mass(0)
    b.close()
    assert p0[0] == pytest.approx(0.02 * mass, rel=2e-3)
    # FP32 rounding of j per node and step: bounded by 1e-4 of the velocity
    # scale summed over the nodes
    tol = 1e-4 * mass * 0.02
    assert abs(p1[0] - p0[0]) < tol and abs(p1[1] - p0[1]) < tol


def test_momentum_rejects_bad_arguments():
    b = lbm.Batch([small_spec(16, 8, seed=3)], "fp32_dev")
    b.init()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_total_momentum(b.ctx, 1)
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm._check(lbm.load().lbm_total_momentum(b.ctx, 0, None, None))
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm._check(lbm.load().lbm_totals_all(b.ctx, None))
    assert e.value.code == lbm.LBM_EINVAL
    b.close()


def test_staging_in_groups_changes_nothing(monkeypatch):
    """Init and read-outs stage a group of lattices at a time when the batch
    exceeds the staging buffers; with tiny buffers (every lattice a group of
    its own, or a few together) the results equal one-group staging bit for
    bit, also with velocities and for in-place storage."""
    specs = [small_spec(70, 45, walls=True, seed=71), small_spec(130, 9, seed=72), stratified_channel(True),
             small_spec(33, 300, seed=73, shape="bubble"), small_spec(5, 3, seed=74)]
    ux = [np.full_like(s.rho, 0.01) for s in specs]
    uy = [np.full_like(s.rho, -0.02) for s in specs]

    def run(precision):
        b = lbm.Batch(specs, precision)
        for i, s in enumerate(specs):
            lbm.lbm_init_fields(b.ctx, i, s.rho, ux[i], uy[i])
        rho_all = np.ascontiguousarray(np.concatenate([s.rho.ravel() for s in specs]))
        b.step(3)
        lbm.lbm_init_fields(b.ctx, 3, specs[3].rho)                    # one lattice again
        b.step(4)
        n = sum(s.nodes for s in specs)
        out = [np.empty(n) for _ in range(4)]
        lbm.lbm_read_moments_all(b.ctx, *out, allow_flags=True)
        dens = np.empty(n)
        lbm.lbm_read_moments_all(b.ctx, dens, allow_flags=True)       # density alone
        tot = b.totals(allow_flags=True)
        per = [b.moments(i, allow_flags=True) for i in range(len(specs))]
        b2 = lbm.Batch(specs, precision)
        lbm.lbm_init_fields_all(b2.ctx, rho_all)
        b2.step(2)
        out2 = np.empty(n)
        lbm.lbm_read_moments_all(b2.ctx, out2, allow_flags=True)
        b.close()
        b2.close()
        return out, dens, tot, per, out2

    for precision in ("fp32_dev", "fp64", "fp32_dev_inplace"):
        ref = run(precision)
        for nodes, cells in (("1", "1"), ("20000", "40000")):
            monkeypatch.setenv("LBM_STAGE_NODES", nodes)
            monkeypatch.setenv("LBM_STAGE_CELLS", cells)
            got = run(precision)
            monkeypatch.delenv("LBM_STAGE_NODES")
            monkeypatch.delenv("LBM_STAGE_CELLS")
            for a, b in zip(got[0], ref[0]):
                assert np.array_equal(a, b), precision
            assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
            for pa, pb in zip(got[3], ref[3]):
                for a, b in zip(pa, pb):
                    assert np.array_equal(a, b)
            assert np.array_equal(got[4], ref[4])
