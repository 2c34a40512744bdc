"""The paper's dynamic cases at its geometry against the oracle, over a
window of their steps (Sec. 3.2, Fig. 4 and 5; Sec. 4.1, Fig. 7-9).

Tolerances:
- FP64 storage differs from the oracle in rounding order only. In the stable
  cases (the nucleus, the collapse) that stays below 1e-9 of the density over
  thousands of steps. Cavitation inception is an instability: the 1e-8
  perturbation of its initial row grows to order one by the separation near
  step 180, and rounding differences of order 1e-16 grow with it (measured
  7e-10 at step 150, 2e-6 at 250, 3e-4 at 400). So the fields are compared
  before the separation (1e-8), and after it what is unique: the step at which
  the perturbed row turns to vapour.
- FP32 storage against the FP64 oracle: 1e-4 of the density pointwise and 1%
  of the bubble radius, the bars stated for the FP32 path."""
import os

import numpy as np
import pytest

from oracle import d2q9, thermo
from paper_1605_01800_gb300 import experiments, inputs, lbm
from tests.cases import oracle_from_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def oracle_on_every_core():
    d2q9.set_threads(os.cpu_count() or 1)
    yield
    d2q9.set_threads(1)


def _rel(a, b, m):
    return float(np.max(np.abs(a[m] / b[m] - 1.0)))


def _gpu(spec, precision, steps):
    b = lbm.Batch([spec], precision)
    b.init()
    b.step(steps)
    out = b.moments(0, allow_flags=True)
    status = b.status(0)
    b.close()
    return out, status


def test_inception_separates_at_the_oracle_step():
    spec = experiments.inception_spec()
    n = spec.nx
    rho_c = thermo.critical_point(a=0.5)[1]
    b = lbm.Batch([spec], "fp64")
    b.init()
    L = oracle_from_spec(spec)
    t_gpu = t_orc = None
    for t in range(5, 301, 5):
        b.step(5)
        L.step(5)
        g = b.moments(0, allow_flags=True)[0]
        o = L.moments()[0]
        if t == 150:   # before the separation: rounding differences only
            assert _rel(g, o, np.ones_like(o, bool)) < 1e-8
        if t_gpu is None and g[(n - 1) // 2, (n - 1) // 2] < rho_c:
            t_gpu = t
        if t_orc is None and o[(n - 1) // 2, (n - 1) // 2] < rho_c:
            t_orc = t
    assert b.status(0) == 0 and L.flags == 0
    b.close()
    assert t_orc is not None and 0.7 * 180 <= t_orc <= 1.3 * 180
    assert t_gpu == t_orc


def _nucleus_liquid():
    """The stretched liquid of the critical-nucleus experiment: Eq. 18 with
    the printed sigma gives r* = 11.3."""
    import warnings
    from scipy.optimize import brentq
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        T = 0.5 * thermo.critical_point(a=0.5)[0]
        _, rho_l, p0 = thermo.maxwell(T, a=0.5)
        dP = 0.01051 / 11.3
        return brentq(lambda r: thermo.p_eos(r, T, a=0.5) - (p0 - dP), thermo.spinodals(T, a=0.5)[1], rho_l)


@pytest.mark.parametrize("R0", [9.0, 14.0])
def test_critical_nucleus_window_matches_oracle(R0):
    """401^2, 2000 steps: the bubble below r* condenses, the one above grows,
    in the GPU runs as in the oracle."""
    rho_L = _nucleus_liquid()
    (spec,) = experiments.nucleus_specs([R0], rho_L)
    steps = 2000
    L = oracle_from_spec(spec)
    L.step(steps)
    orho = L.moments()[0]
    m = np.ones_like(orho, bool)
    rho_g = inputs.coexistence(0.5)["rho_g"]
    r_orc = experiments.vapour_radius(orho, rho_L, rho_g)
    (g64, _, _, _), s64 = _gpu(spec, "fp64", steps)
    assert s64 == 0 and L.flags == 0
    assert _rel(g64, orho, m) < 1e-9
    (g32, _, _, _), s32 = _gpu(spec, "fp32_dev", steps)
    assert s32 == 0
    assert _rel(g32, orho, m) < 1e-4
    r32 = experiments.vapour_radius(g32, rho_L, rho_g)
    assert r32 == pytest.approx(r_orc, rel=0.01, abs=0.01 * R0)
    if R0 < 11.3:
        assert r_orc == 0.0
    else:
        assert r_orc > R0


def test_wall_collapse_window_matches_oracle():
    """1801 x 301 between two walls, R0 = 138, d = 150, liquid at 1.05 rho_l,
    tau_nu = 0.6 (at the paper's 0.51 the split diverges, in the oracle as on
    the GPU): 400 steps of the collapse."""
    spec = experiments.wall_collapse_spec(tau_nu=0.6, liquid_factor=1.05)
    steps = 400
    L = oracle_from_spec(spec)
    L.step(steps)
    orho, oux, ouy, _ = L.moments()
    m = spec.solid == 0
    uscale = max(np.abs(oux[m]).max(), np.abs(ouy[m]).max())
    thr = 0.5 * (spec.meta["rho_l"] + spec.meta["rho_g"])
    r_orc = np.sqrt(((orho < thr) & m).sum() / np.pi)
    for precision, tol in (("fp64", 1e-10), ("fp32_dev", 1e-4)):
        (rho, ux, uy, _), status = _gpu(spec, precision, steps)
        assert status == 0
        assert _rel(rho, orho, m) < tol, precision
        assert max(np.abs(ux - oux)[m].max(), np.abs(uy - ouy)[m].max()) < tol * uscale, precision
        r = np.sqrt(((rho < thr) & m).sum() / np.pi)
        assert r == pytest.approx(r_orc, rel=0.01)
