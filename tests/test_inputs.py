"""The seeded input generators (paper_1605_01800_gb300/inputs.py), on the CPU:
SplitMix64 against its published first outputs, the uniform draws, and the
shapes of the workloads the tests and the benchmark use."""
import numpy as np

from paper_1605_01800_gb300 import inputs


def test_splitmix64_first_outputs_for_seed_zero():
    # the first three outputs of SplitMix64 from state 0 (Steele, Lea and
    # Flood 2014; the generator of java.util.SplittableRandom)
    assert [int(v) for v in inputs.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_form_is_a_prefix_of_longer_draws():
    a = inputs.splitmix64(1605019, 1000)
    b = inputs.splitmix64(1605019, 10)
    assert np.array_equal(a[:10], b)
    assert len(set(a.tolist())) == 1000


def test_uniform_draws():
    u = inputs.uniform01(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12) < 0.002
    v = inputs.uniform_pm1(7, 200000)
    assert np.array_equal(v, 2.0 * u - 1.0) and v.min() >= -1.0 and v.max() < 1.0


def test_workload_shapes():
    tc = inputs.critical_temperature()
    coex = inputs.coexistence_batch()
    assert len(coex) == 32 and all((s.nx, s.ny) == (256, 64) for s in coex)
    assert np.allclose([s.T / tc for s in coex], 0.5 + 0.45 * np.arange(32) / 31)
    assert sum(s.nodes for s in coex) == 524288

    lap = inputs.laplace_batch()
    sizes = sorted({s.nx for s in lap})
    assert len(lap) == 48 and all(s.nx == s.ny for s in lap)
    assert sizes[0] == 128 and sizes[-1] == 320 and all(L % 32 == 0 for L in sizes)
    assert sum(s.nodes for s in lap) == 2256896

    (cav,) = inputs.cavitation_1024()
    assert (cav.nx, cav.ny) == (1024, 1024) and cav.solid is None

    (col,) = inputs.collapse()
    assert (col.nx, col.ny) == (2048, 1024)
    assert col.solid[0].all() and col.solid[-1].all() and not col.solid[1:-1].any()


def test_noise_is_multiplicative_and_seeded():
    a = inputs.coexistence_batch()
    b = inputs.coexistence_batch()
    assert all(np.array_equal(x.rho, y.rho) for x, y in zip(a, b))
    assert not np.array_equal(a[0].rho, a[1].rho)
    assert all((s.rho > 0).all() for s in a)
