"""Pins of the oracle's thermodynamics (Eq. 9, 11, 13, 15) against the paper's
printed values and against closed forms that do not go through the oracle's
own quadrature."""
import json
import math
import os
import warnings

import numpy as np
import pytest

from oracle import thermo

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
warnings.filterwarnings("ignore", category=Warning, module="scipy")


def test_critical_temperature_matches_printed_a_b_relations():
    # Eq. 15 text: a = 0.4963 R^2 Tc^2/pc and b = 0.18727 R Tc/pc, so
    # Tc = (0.18727 / 0.4963) a / (b R). The printed coefficients have 4-5
    # significant figures.
    Tc, rho_c, p_c = thermo.critical_point(1.0, 4.0, 1.0)
    printed = GOLDEN["cs_b_coefficient"]["value"] / GOLDEN["cs_a_coefficient"]["value"]
    assert Tc * 4.0 / 1.0 == pytest.approx(printed, rel=1e-4)
    # and the same relations give a and b back from Tc and pc
    assert 0.4963 * Tc ** 2 / p_c == pytest.approx(1.0, rel=2e-4)
    assert 0.18727 * Tc / p_c == pytest.approx(4.0, rel=2e-4)


def test_critical_density_printed():
    _, rho_c, _ = thermo.critical_point()
    # Printed to 4 decimals; the exact CS value 0.130444 sits 0.56 units of
    # the last printed digit below it, so allow one unit.
    assert rho_c == pytest.approx(GOLDEN["rho_c"]["value"], abs=1e-4)


def test_critical_point_is_inflection_by_finite_differences():
    Tc, rho_c, _ = thermo.critical_point()
    h = 1e-5
    p = lambda r: thermo.p_eos(r, Tc)
    d1 = (p(rho_c + h) - p(rho_c - h)) / (2 * h)
    d2 = (p(rho_c + h) - 2 * p(rho_c) + p(rho_c - h)) / h ** 2
    assert abs(d1) < 1e-9
    assert abs(d2) < 1e-5


def test_g1_is_derivative_of_eta_z():
    for eta in (0.01, 0.1, 0.2, 0.35):
        h = 1e-6
        fd = ((eta + h) * thermo.z_cs(eta + h) - (eta - h) * thermo.z_cs(eta - h)) / (2 * h)
        assert thermo.g1(eta) == pytest.approx(fd, rel=1e-8)
        fd2 = (thermo.g1(eta + h) - thermo.g1(eta - h)) / (2 * h)
        assert thermo.g1_prime(eta) == pytest.approx(fd2, rel=1e-7)


def test_maxwell_at_half_tc_matches_printed_values():
    Tc, _, _ = thermo.critical_point()
    rg, rl, _ = thermo.maxwell(0.5 * Tc)
    assert rl == pytest.approx(GOLDEN["rho_l_0p5Tc"]["value"], abs=5e-5)
    assert rg == pytest.approx(GOLDEN["rho_g_0p5Tc"]["value"], abs=5e-7)
    assert rl / rg > GOLDEN["min_density_ratio_0p5Tc"]["value"]


def _mu_cs(rho, T, a=1.0, b=4.0, R=1.0):
    """Chemical potential of the CS fluid, mu = int dp / rho, in closed form:
    R T [ln rho + eta (8 - 9 eta + 3 eta^2) / (1 - eta)^3 + 1] - 2 a rho
    (constant terms drop out of differences)."""
    eta = b * rho / 4.0
    return R * T * (math.log(rho) + eta * (8 - 9 * eta + 3 * eta ** 2) / (1 - eta) ** 3) - 2 * a * rho


@pytest.mark.parametrize("tr", [0.5, 0.6, 0.8, 0.95])
def test_maxwell_is_equal_pressure_and_chemical_potential(tr):
    # Eq. 11 with p(rho_g) = p(rho_l) = p0 is equivalent to equal chemical
    # potentials; check with the closed-form mu, independent of the quadrature.
    Tc, _, _ = thermo.critical_point()
    T = tr * Tc
    rg, rl, p0 = thermo.maxwell(T)
    assert thermo.p_eos(rg, T) == pytest.approx(p0, rel=1e-9)
    assert thermo.p_eos(rl, T) == pytest.approx(p0, rel=1e-9)
    dmu = _mu_cs(rl, T) - _mu_cs(rg, T)
    assert abs(dmu) < 1e-9 * T


def test_mu_closed_form_derivative():
    T = 0.07
    for r in (0.01, 0.2, 0.4):
        h = 1e-6
        dmu = (_mu_cs(r + h, T) - _mu_cs(r - h, T)) / (2 * h)
        assert dmu == pytest.approx(thermo.dp_drho(r, T) / r, rel=1e-7)


def test_spinodal_zero_slope():
    Tc, _, _ = thermo.critical_point()
    for tr in (0.5, 0.6, 0.8):
        for r in thermo.spinodals(tr * Tc):
            h = 1e-7
            fd = (thermo.p_eos(r + h, tr * Tc) - thermo.p_eos(r - h, tr * Tc)) / (2 * h)
            assert abs(fd) < 1e-8


def test_eq9_with_eps_zero_reduces_to_psi_prime_over_psi():
    # At eps = 0 the weight psi'/psi integrates to ln psi; check one value of
    # the weighted area by direct integration of d(ln psi).
    Tc, _, _ = thermo.critical_point()
    T = 0.9 * Tc
    rg, rl, p0 = thermo.lb_coexistence(T, 0.0)
    assert thermo.p_eos(rg, T) == pytest.approx(p0, rel=1e-9)
    # integral of (p0 - p) dln(psi) via trapezoid in psi on a fine grid
    r = np.linspace(rg, rl, 400001)
    psi = np.sqrt(thermo.psi_sq(r, T))
    integrand = p0 - thermo.p_eos(r, T)
    lnpsi = np.log(psi)
    area = np.sum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(lnpsi))
    assert abs(area) < 1e-9


def test_psi_root_is_where_psi_vanishes():
    Tc, _, _ = thermo.critical_point()
    for tr in (0.5, 0.6, 0.8):
        r0 = thermo.psi_root(tr * Tc)
        assert abs(thermo.psi_sq(r0, tr * Tc)) < 1e-13
        assert thermo.psi_sq(r0 - 1e-3, tr * Tc) > 0 > thermo.psi_sq(r0 + 1e-3, tr * Tc)


def test_coexistence_table_regenerates_from_oracle():
    from paper_1605_01800_gb300 import inputs
    tab = inputs.coexistence_table()
    Tc, rho_c, _ = thermo.critical_point()
    assert tab["Tc"] == pytest.approx(Tc, rel=1e-14)
    assert tab["rho_c"] == pytest.approx(rho_c, rel=1e-14)
    for row in tab["rows"][::6]:
        rg, rl, p0 = thermo.maxwell(row["T_over_Tc"] * Tc)
        assert row["rho_g"] == pytest.approx(rg, rel=1e-10)
        assert row["rho_l"] == pytest.approx(rl, rel=1e-12)


def test_eos_constant_a_from_the_oracle_laplace_series():
    # Reading of Sec. 3.1's constants: with b = 4 (fixed by the printed
    # densities) the surface tension decides a. The oracle's own static-bubble
    # Laplace series at 0.5 Tc (tests/golden/write_oracle_laplace.py, FP64,
    # oracle only) gives sigma within 5% of the printed 0.01051 for a = 0.5
    # and 48% above it for a = 1 (where the smallest bubble also drives the
    # liquid past the psi root once: psi^2 clamped).
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_laplace_sigma.json")
    data = json.load(open(path))
    paper = data["paper_sigma_0p5Tc"]["value"]
    by_a = {s["a"]: s for s in data["series"]}
    assert all(b["flags"] == 0 for b in by_a[0.5]["bubbles"])
    for s in by_a.values():
        assert all(b["flags"] & 2 == 0 for b in s["bubbles"])   # nothing non-finite
        # every bubble kept its size: a settled series, not a shrinking one
        assert all(abs(b["r"] / b["R0"] - 1) < 0.1 for b in s["bubbles"])
    assert by_a[0.5]["sigma"] == pytest.approx(paper, rel=0.05)
    assert by_a[1.0]["sigma"] > 1.3 * paper
