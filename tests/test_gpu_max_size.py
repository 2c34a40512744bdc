"""The largest lattice the library accepts (9 stored planes just under 2^31
elements), twice in one batch, so that the second lattice starts past 2^31
elements of the distribution arrays. A field that varies along x only must
evolve identically in every row, and row for row as a one-row lattice of the
same width (which the oracle parity tests cover): any wrong 32-bit index or
offset at these sizes breaks one of the two."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1605_01800_gb300 import inputs, lbm  # noqa: E402

pytestmark = pytest.mark.gpu

NX = 15000
KGY, KGX = 2, 32  # the stored frame: rows above and below, left margin


def largest_ny(nx):
    """Largest ny with 9 * plane < 2^31, plane = (ny + 2 kGY) * round_up(nx + 34, 32)."""
    pitch = -(-(nx + KGX + 2) // 32) * 32
    ny = (2**31 - 1) // (9 * pitch) - 2 * KGY
    assert 9 * (ny + 2 * KGY) * pitch < 2**31 <= 9 * (ny + 1 + 2 * KGY) * pitch
    return ny


def x_profile(nx, tr=0.7):
    c = inputs.coexistence(tr)
    x = np.arange(nx, dtype=float)
    return c["rho_g"] + 0.5 * (c["rho_l"] - c["rho_g"]) * (
        np.tanh(2 * (x - nx / 4) / 4) - np.tanh(2 * (x - 3 * nx / 4) / 4)), c


def spec(nx, ny, prof, c, tr=0.7):
    Tc = inputs.critical_temperature()
    return inputs.LatticeSpec(nx, ny, tr * Tc, inputs.relax_rates(0.7), 1.86,
                              np.broadcast_to(prof, (ny, nx)), rho_ref=c["rho_g"])


def test_largest_lattices_past_2_31_elements_evolve_row_for_row():
    free, _ = torch.cuda.mem_get_info()
    if free < 64 * 2**30:
        pytest.skip("needs 64 GB of free device memory")
    ny = largest_ny(NX)
    prof, c = x_profile(NX)
    steps = 3
    # reference: one row of the same width
    ref = lbm.Batch([spec(NX, 1, prof, c)], "fp32_dev")
    ref.init()
    ref.step(steps)
    row = np.empty((1, NX))
    lbm.lbm_read_moments(ref.ctx, 0, row)
    ref.close()

    big = [spec(NX, ny, prof, c), spec(NX, ny, prof, c)]
    b = lbm.Batch(big, "fp32_dev")
    try:
        for i in range(2):
            lbm.lbm_init_fields(b.ctx, i, np.ascontiguousarray(big[i].rho, dtype=np.float64))
        b.step(steps)
        rows = [0, 1, 2, ny // 2, ny - 3, ny - 2, ny - 1]
        rows += list(np.random.default_rng(5).integers(0, ny, 8))
        for i in range(2):
            rho = np.empty((ny, NX))
            lbm.lbm_read_moments(b.ctx, i, rho)
            assert b.status(i) == 0
            for y in rows:
                assert np.array_equal(rho[y], row[0]), (i, y)
            del rho
    finally:
        b.close()
