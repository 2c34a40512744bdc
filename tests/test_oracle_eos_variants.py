"""Pins of the oracle's pseudopotentials beyond the paper's Carnahan-Starling
case: Eq. 13 with van der Waals and Peng-Robinson, and psi of Eq. 12.

Each check rests on something other than the oracle itself: the closed-form
van der Waals critical point, the Peng-Robinson critical compressibility
(0.3074, fixed by its two constants), the defining property of Eq. 12
(psi'/psi^(1+eps) = 1/rho^2, checked by finite differences of the C oracle),
the closed-form van der Waals chemical potential at coexistence, and the
identity of the Eq. 9 and Eq. 11 coexistence that Eq. 12 is built for.
"""
import math
import warnings

import numpy as np
import pytest

from oracle import d2q9, eos_variants as E

VDW = dict(a=0.3375, b=1.0 / 3.0, R=1.0)      # T_c = 0.3, rho_c = 1, p_c = 0.1125
PR = dict(a=2.0 / 49.0, b=2.0 / 21.0, R=1.0)  # T_c = 0.0729


@pytest.fixture(autouse=True)
def _quiet():
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        yield


def _lat(eos, **kw):
    return d2q9.Lattice(4, 4, eos=eos, **kw)


def test_c_oracle_eos_matches_the_written_formulas():
    # the C oracle's p for each kind at a few densities, against the
    # formulas written out here a second time
    T = 0.25
    L = _lat("vdw", T=T, **VDW)
    for r in (0.1, 0.7, 1.9):
        assert L.p_eos(r) == pytest.approx(r * T / (1 - VDW["b"] * r) - VDW["a"] * r * r, rel=1e-14)
    T2 = 0.06
    L = _lat("pr", T=T2, omega=0.344, **PR)
    al = E.pr_alpha(T2, PR["a"], PR["b"], 1.0, 0.344)
    for r in (0.1, 3.0, 7.0):
        b = PR["b"]
        ref = r * T2 / (1 - b * r) - PR["a"] * al * r * r / (1 + 2 * b * r - b * b * r * r)
        assert L.p_eos(r) == pytest.approx(ref, rel=1e-13)
    L = _lat("psi_exp", G=-3.0, eps=0.0)
    for r in (0.3, 1.0, 2.5):
        assert L.psi(r)[0] == pytest.approx(math.exp(-1.0 / r), rel=1e-15)


def test_vdw_critical_point_closed_form():
    Tc, rc, pc = E.critical_point("vdw", **VDW)
    a, b = VDW["a"], VDW["b"]
    assert Tc == pytest.approx(8 * a / (27 * b), rel=1e-5)
    assert rc == pytest.approx(1 / (3 * b), rel=1e-4)
    assert pc == pytest.approx(a / (27 * b * b), rel=1e-4)


def test_pr_critical_compressibility_and_temperature():
    Tc, rc, pc = E.critical_point("pr", omega=0.344, **PR)
    assert Tc == pytest.approx(0.0778 * PR["a"] / (0.45724 * PR["b"]), rel=1e-4)
    assert pc / (rc * Tc) == pytest.approx(0.3074, abs=2e-4)


@pytest.mark.parametrize("G,eps", [(-1.0, 0.0), (-1.0, 1.0), (-1.0, 1.86), (-3.0, 1.0 / 3.0), (-3.0, 0.5)])
def test_eq12_psi_has_the_defining_derivative(G, eps):
    # psi'/psi^(1+e) = 1/rho^2 with e = -G eps (Li's eps in Eq. 9 terms)
    e = -G * eps
    L = _lat("psi_exp", G=G, eps=eps)
    for r in (0.2, 0.8, 2.0, 5.0):
        h = 1e-6 * r
        d = (L.psi(r + h)[0] - L.psi(r - h)[0]) / (2 * h)
        assert d / L.psi(r)[0] ** (1 + e) == pytest.approx(1.0 / (r * r), rel=1e-7)


def test_eq12_small_eps_tends_to_the_exponential():
    L0 = _lat("psi_exp", G=-3.0, eps=0.0)
    L1 = _lat("psi_exp", G=-3.0, eps=1e-7)
    for r in (0.3, 1.0, 3.0):
        assert L1.psi(r)[0] == pytest.approx(L0.psi(r)[0], rel=1e-5)


def test_vdw_maxwell_has_equal_chemical_potential():
    # mu = R T ln(rho / (1 - b rho)) + R T b rho / (1 - b rho) - 2 a rho (+ const)
    a, b = VDW["a"], VDW["b"]
    for tr in (0.7, 0.9):
        T = tr * 0.3
        g, l, p0 = E.maxwell("vdw", T=T, **VDW)
        mu = lambda r: T * math.log(r / (1 - b * r)) + T * b * r / (1 - b * r) - 2 * a * r
        assert mu(g) == pytest.approx(mu(l), abs=1e-9)
        p, _, _ = E.eos("vdw", T=T, **VDW)
        assert p(g) == pytest.approx(p0, rel=1e-10) and p(l) == pytest.approx(p0, rel=1e-10)


@pytest.mark.parametrize("eps", [0.0, 1.0 / 3.0])
def test_eq12_mechanical_stability_equals_maxwell(eps):
    g9, l9, p9 = E.lb_coexistence("psi_exp", eps, G=-3.0)
    g11, l11, p11 = E.maxwell("psi_exp", G=-3.0, eps=eps)
    assert g9 == pytest.approx(g11, rel=1e-8) and l9 == pytest.approx(l11, rel=1e-8)


def test_eq9_for_vdw_depends_on_eps_as_for_cs():
    # Eq. 9 moves the vapour density up with eps and passes Maxwell between
    # eps = 1 and 1.5 at 0.7 Tc (the same trend as the paper's CS fluid)
    T = 0.7 * 0.3
    g11, _, _ = E.maxwell("vdw", T=T, **VDW)
    g = [E.lb_coexistence("vdw", e, T=T, **VDW)[0] for e in (0.0, 1.0, 1.5, 2.0)]
    assert g[0] < g[1] < g[2] < g[3]
    assert g[1] < g11 < g[2]
