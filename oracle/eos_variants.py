"""Thermodynamics of the pseudopotentials beyond the paper's Carnahan-Starling
case (test infrastructure only): Eq. 13 with the van der Waals and
Peng-Robinson EOS, and psi of Eq. 12 (the first strategy) whose EOS is the
LB pressure of Eq. 10.

All FP64 numpy / scipy. An EOS is a pair of callables (p, dp/drho) on
(0, rho_max); the coexistence solvers scan them numerically, so they serve
every kind alike:

- ``eos``              (p, dp, rho_max) of a kind.
- ``critical_point``   (T_c, rho_c, p_c) from dp/drho = d2p/drho2 = 0 (Eq. 13 kinds).
- ``maxwell``          equal-area coexistence, Eq. 11 (weight 1/rho^2).
- ``lb_coexistence``   mechanical-stability coexistence, Eq. 9
                       (weight psi'/psi^(1+eps), psi of Eq. 13 or Eq. 12).
"""
import math
import warnings

from scipy import integrate, optimize

CS2 = 1.0 / 3.0


def pr_alpha(T, a, b, R, omega):
    """Peng-Robinson alpha(T) = (1 + k (1 - sqrt(T/Tc)))^2 with
    k = 0.37464 + 1.54226 omega - 0.26992 omega^2 and Tc from
    a = 0.45724 R^2 Tc^2 / pc, b = 0.0778 R Tc / pc."""
    Tc = (0.0778 / 0.45724) * a / (b * R)
    k = 0.37464 + 1.54226 * omega - 0.26992 * omega ** 2
    return (1.0 + k * (1.0 - math.sqrt(T / Tc))) ** 2


def psi_eq12(rho, e):
    """psi of Eq. 12 with exponent e: exp(-1/rho) for e = 0, else
    (rho/(e + rho))^(1/e)."""
    if e == 0.0:
        return math.exp(-1.0 / rho)
    return (rho / (e + rho)) ** (1.0 / e)


def mech_eps(G, eps):
    """The exponent of the mechanical stability condition (Eq. 9) that Li's
    term of Eq. 14 with coefficient eps yields: -G eps (Li et al. 2013,
    -16 G sigma with 0.75 eps = 12 sigma); eps itself at the paper's G = -1.
    Eq. 12's psi takes this exponent."""
    return -G * eps


def eos(kind, T=0.0, a=0.0, b=0.0, R=1.0, omega=0.0, G=-1.0, eps=0.0):
    """(p, dp/drho, rho_max) of a pseudopotential kind: "vdw", "pr" (T, a, b,
    R, omega) or "psi_exp" (G and Li's eps; psi of Eq. 12 with the exponent
    mech_eps(G, eps); p = rho c_s^2 + G psi^2 / 2, Eq. 10)."""
    if kind == "vdw":
        p = lambda r: r * R * T / (1.0 - b * r) - a * r * r
        dp = lambda r: R * T / (1.0 - b * r) ** 2 - 2.0 * a * r
        return p, dp, 1.0 / b
    if kind == "pr":
        aa = a * pr_alpha(T, a, b, R, omega)

        def p(r):
            return r * R * T / (1.0 - b * r) - aa * r * r / (1.0 + 2.0 * b * r - b * b * r * r)

        def dp(r):
            D = 1.0 + 2.0 * b * r - b * b * r * r
            dD = 2.0 * b - 2.0 * b * b * r
            return R * T / (1.0 - b * r) ** 2 - aa * (2.0 * r * D - r * r * dD) / (D * D)
        return p, dp, 1.0 / b
    if kind == "psi_exp":
        e = mech_eps(G, eps)

        def p(r):
            return r * CS2 + 0.5 * G * psi_eq12(r, e) ** 2

        def dp(r):  # dpsi/drho written out from Eq. 12
            s = psi_eq12(r, e)
            ds = s / (r * r) if e == 0.0 else s * (1.0 / r - 1.0 / (e + r)) / e
            return CS2 + G * s * ds
        return p, dp, 60.0
    raise ValueError(kind)


def _spinodals(dp, rho_max, n=4000):
    """The two zeros of dp/drho on (0, rho_max): a scan on a geometric grid,
    then bisection on each sign change."""
    lo = rho_max * 1e-6
    grid = [lo * (0.999 * rho_max / lo) ** (k / n) for k in range(n + 1)]
    vals = [dp(r) for r in grid]
    roots = []
    for i in range(n):
        if vals[i] == 0.0 or vals[i] * vals[i + 1] < 0.0:
            roots.append(optimize.brentq(dp, grid[i], grid[i + 1], xtol=1e-15, rtol=1e-14))
    if len(roots) < 2:
        raise ValueError("no two-phase region")
    return roots[0], roots[-1]


def _coexistence(p, dp, rho_max, weight):
    sv, sl = _spinodals(dp, rho_max)
    p_hi, p_lo = p(sv), p(sl)

    def roots(p0):
        rg = optimize.brentq(lambda r: p(r) - p0, rho_max * 1e-9, sv, xtol=1e-300, rtol=1e-14, maxiter=500)
        rl = optimize.brentq(lambda r: p(r) - p0, sl, 0.999 * rho_max, xtol=1e-15, rtol=1e-14, maxiter=500)
        return rg, rl

    def area(p0):
        rg, rl = roots(p0)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, _ = integrate.quad(lambda r: (p0 - p(r)) * weight(r), rg, rl, points=[sv, sl],
                                    epsabs=0.0, epsrel=1e-11, limit=400)
        return val

    span = p_hi - p_lo
    lo_p = max(p_lo, p(rho_max * 1e-9)) + 1e-12 * span
    p0 = optimize.brentq(area, lo_p, p_hi - 1e-12 * span, xtol=1e-18, rtol=1e-14, maxiter=500)
    rg, rl = roots(p0)
    return rg, rl, p0


def maxwell(kind, **kw):
    """Maxwell equal-area coexistence (rho_g, rho_l, p0), Eq. 11."""
    p, dp, rmax = eos(kind, **kw)
    return _coexistence(p, dp, rmax, lambda r: 1.0 / (r * r))


def lb_coexistence(kind, eps, **kw):
    """Mechanical-stability coexistence (rho_g, rho_l, p0), Eq. 9, with the
    exponent mech_eps(G, eps) of Li's term eps. For the Eq. 13 kinds
    psi' = (dp/drho - c_s^2) / (G psi); for Eq. 12 psi' comes from its
    definition (the weight is then 1/rho^2: Eq. 9 is Eq. 11)."""
    G = kw.get("G", -1.0)
    em = mech_eps(G, eps)
    p, dp, rmax = eos(kind, eps=eps, **kw) if kind == "psi_exp" else eos(kind, **kw)
    if kind == "psi_exp":
        def weight(r):
            s = psi_eq12(r, em)
            ds = s / (r * r) if em == 0.0 else s * (1.0 / r - 1.0 / (em + r)) / em
            return ds / s ** (1.0 + em)
    else:
        def weight(r):
            s = math.sqrt(2.0 * (p(r) - r * CS2) / G)
            return (dp(r) - CS2) / (G * s) / s ** (1.0 + em)
    return _coexistence(p, dp, rmax, weight)


def critical_point(kind, a, b, R=1.0, omega=0.0):
    """(T_c, rho_c, p_c) of an Eq. 13 kind from dp/drho = d2p/drho2 = 0: the
    temperature where the two zeros of dp/drho merge (bisection in T)."""
    def two_phase(T):
        try:
            _spinodals(eos(kind, T=T, a=a, b=b, R=R, omega=omega)[1], 1.0 / b)
            return True
        except ValueError:
            return False
    lo, hi = 1e-6 * a / (b * R), 10.0 * a / (b * R)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if two_phase(mid) else (lo, mid)
    Tc = 0.5 * (lo + hi)
    # rho_c: the minimum of dp/drho at Tc
    p, dp, rmax = eos(kind, T=Tc, a=a, b=b, R=R, omega=omega)
    rc = optimize.minimize_scalar(dp, bounds=(1e-6 * rmax, 0.99 * rmax), method="bounded",
                                  options={"xatol": 1e-13}).x
    return Tc, rc, p(rc)
