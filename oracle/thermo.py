"""Thermodynamics of the Carnahan-Starling fluid of arXiv:1605.01800 (test infrastructure only).

- ``p_eos``           Eq. 15.
- ``critical_point``  T_c, rho_c from dp/drho = d2p/drho2 = 0 of Eq. 15.
- ``maxwell``         Maxwell equal-area coexistence, Eq. 11.
- ``lb_coexistence``  the pseudopotential mechanical-stability coexistence of
                      Eq. 9 with psi of Eq. 13 (p_EOS-PL = p_EOS, Eq. 10).
- ``spinodals``       the densities where dp/drho = 0.

All FP64 numpy / scipy. With eta = b rho / 4 the CS EOS reads
p = rho R T Z(eta) - a rho^2, Z = (1 + eta + eta^2 - eta^3) / (1 - eta)^3.
"""
import math
import warnings

import numpy as np
from scipy import integrate, optimize

CS2 = 1.0 / 3.0


def z_cs(eta):
    """Compressibility factor of Eq. 15."""
    return (1.0 + eta + eta ** 2 - eta ** 3) / (1.0 - eta) ** 3


def p_eos(rho, T, a=1.0, b=4.0, R=1.0):
    """Carnahan-Starling EOS, Eq. 15."""
    eta = b * rho / 4.0
    return rho * R * T * z_cs(eta) - a * rho * rho


def g1(eta):
    """d(eta Z)/d eta for the CS Z, written out: (1+4e+4e^2-4e^3+e^4)/(1-e)^4."""
    return (1.0 + 4.0 * eta + 4.0 * eta ** 2 - 4.0 * eta ** 3 + eta ** 4) / (1.0 - eta) ** 4


def g1_prime(eta):
    """Derivative of ``g1`` with respect to eta."""
    P = 1.0 + 4.0 * eta + 4.0 * eta ** 2 - 4.0 * eta ** 3 + eta ** 4
    dP = 4.0 + 8.0 * eta - 12.0 * eta ** 2 + 4.0 * eta ** 3
    return (dP * (1.0 - eta) + 4.0 * P) / (1.0 - eta) ** 5


def dp_drho(rho, T, a=1.0, b=4.0, R=1.0):
    """dp/drho of Eq. 15: R T d(eta Z)/d eta - 2 a rho."""
    return R * T * g1(b * rho / 4.0) - 2.0 * a * rho


def critical_point(a=1.0, b=4.0, R=1.0):
    """(T_c, rho_c, p_c) of Eq. 15.

    At the critical point dp/drho = 0 and d2p/drho2 = 0, i.e.
    R T g1(eta) = (8a/b) eta and R T g1'(eta) = 8a/b, so g1(eta) = eta g1'(eta).
    """
    eta_c = optimize.brentq(lambda e: g1(e) - e * g1_prime(e), 0.05, 0.3, xtol=1e-16, rtol=1e-15)
    Tc = (8.0 * a / b) * eta_c / (R * g1(eta_c))
    rho_c = 4.0 * eta_c / b
    return Tc, rho_c, p_eos(rho_c, Tc, a, b, R)


def spinodals(T, a=1.0, b=4.0, R=1.0):
    """(rho_spinodal_vapour, rho_spinodal_liquid) at T < T_c: zeros of dp/drho."""
    Tc, rho_c, _ = critical_point(a, b, R)
    if T >= Tc:
        raise ValueError("no spinodal above T_c")
    f = lambda r: dp_drho(r, T, a, b, R)
    # dp/drho > 0 at rho -> 0 and near close packing, < 0 around rho_c.
    r_min = optimize.minimize_scalar(f, bounds=(1e-6, 0.9 * 4.0 / b), method="bounded",
                                     options={"xatol": 1e-14}).x
    lo = optimize.brentq(f, 1e-12, r_min, xtol=1e-16, rtol=1e-15)
    hi = optimize.brentq(f, r_min, 0.999 * 4.0 / b, xtol=1e-16, rtol=1e-15)
    return lo, hi


def _branch_roots(p0, T, a, b, R):
    """Vapour and liquid densities with p_EOS(rho) = p0 (outside the spinodal)."""
    sv, sl = spinodals(T, a, b, R)
    g = lambda r: p_eos(r, T, a, b, R) - p0
    rg = optimize.brentq(g, 1e-300, sv, xtol=1e-300, rtol=1e-15, maxiter=500)
    rl = optimize.brentq(g, sl, 0.999 * 4.0 / b, xtol=1e-16, rtol=1e-15, maxiter=500)
    return rg, rl


def _coexistence(T, weight, a, b, R):
    """Solve int_{rho_g}^{rho_l} (p0 - p_EOS) weight(rho) drho = 0 with
    p_EOS(rho_g) = p_EOS(rho_l) = p0, scanning p0 between the spinodal
    pressures (a 1-D root find in p0)."""
    sv, sl = spinodals(T, a, b, R)
    p_hi = p_eos(sv, T, a, b, R)
    p_lo = max(p_eos(sl, T, a, b, R), 0.0)

    def area(p0):
        rg, rl = _branch_roots(p0, T, a, b, R)
        pts = [sv, sl]
        with warnings.catch_warnings():
            # quad reports round-off once the relative error nears 1e-13
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, _ = integrate.quad(lambda r: (p0 - p_eos(r, T, a, b, R)) * weight(r), rg, rl,
                                    points=pts, epsabs=0.0, epsrel=1e-11, limit=400)
        return val

    span = p_hi - p_lo
    lo = p_lo + 1e-12 * span
    hi = p_hi - 1e-12 * span
    p0 = optimize.brentq(area, lo, hi, xtol=1e-18, rtol=1e-15, maxiter=500)
    rg, rl = _branch_roots(p0, T, a, b, R)
    return rg, rl, p0


def maxwell(T, a=1.0, b=4.0, R=1.0):
    """Maxwell equal-area coexistence (rho_g, rho_l, p0), Eq. 11."""
    return _coexistence(T, lambda r: 1.0 / (r * r), a, b, R)


def psi_sq(rho, T, a=1.0, b=4.0, R=1.0, G=-1.0):
    """psi^2 of Eq. 13 (c = 1)."""
    return 2.0 * (p_eos(rho, T, a, b, R) - rho * CS2) / G


def lb_coexistence(T, eps, a=1.0, b=4.0, R=1.0, G=-1.0):
    """Coexistence (rho_g, rho_l, p0) of the pseudopotential model from the
    mechanical stability condition Eq. 9, with psi of Eq. 13 and
    p_EOS-PL = p_EOS. The weight psi'/psi^(1+e) is evaluated with
    psi' = (dp/drho - c_s^2) / (G psi), which follows from Eq. 13; the
    exponent e = -G eps is the one Li's term of Eq. 14 with coefficient eps
    produces (eps itself at the paper's G = -1)."""
    e = -G * eps

    def weight(r):
        s2 = psi_sq(r, T, a, b, R, G)
        psi = math.sqrt(s2)
        dpsi = (dp_drho(r, T, a, b, R) - CS2) / (G * psi)
        return dpsi / psi ** (1.0 + e)
    return _coexistence(T, weight, a, b, R)


def psi_root(T, a=1.0, b=4.0, R=1.0):
    """Liquid density above which psi^2 of Eq. 13 turns negative (G < 0)."""
    f = lambda r: p_eos(r, T, a, b, R) - r * CS2
    return optimize.brentq(f, 0.2, 0.999 * 4.0 / b, xtol=1e-16, rtol=1e-15)
