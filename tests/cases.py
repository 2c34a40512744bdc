"""Helpers shared by the GPU parity tests: oracle lattices built from the same
seeded ``inputs.LatticeSpec`` the CUDA path gets, and comparison utilities."""
import numpy as np

from oracle import d2q9
from paper_1605_01800_gb300 import inputs


def oracle_from_spec(spec) -> d2q9.Lattice:
    L = d2q9.Lattice(spec.nx, spec.ny, a=spec.a, b=spec.b, R=spec.R, T=spec.T, G=spec.G,
                     s=spec.s, eps=spec.eps, solid=spec.solid, eos=spec.eos, omega=spec.omega)
    L.init(spec.rho)
    return L


def fluid(spec):
    return np.ones((spec.ny, spec.nx), bool) if spec.solid is None else spec.solid == 0


def rel_err(a, b, mask=None):
    d = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    if mask is not None:
        d = d[mask]
    return float(d.max()) if d.size else 0.0


def abs_err(a, b, mask=None):
    d = np.abs(a - b)
    if mask is not None:
        d = d[mask]
    return float(d.max()) if d.size else 0.0


def small_spec(nx, ny, tr=0.7, eps=1.86, tau=0.6, walls=False, seed=7, R=None, shape="droplet"):
    """A small two-phase lattice: droplet (or bubble) of the Maxwell densities
    at T/Tc with a seeded 1e-3 multiplicative noise; optional solid rows."""
    Tc = inputs.critical_temperature()
    c = inputs.coexistence(tr)
    R = R if R is not None else 0.3 * min(nx, ny)
    if shape == "droplet":
        rho = inputs.tanh_profile(nx, ny, (nx - 1) / 2, (ny - 1) / 2, R, c["rho_g"], c["rho_l"], 3.0)
    else:
        rho = inputs.tanh_profile(nx, ny, (nx - 1) / 2, (ny - 1) / 2, R, c["rho_l"], c["rho_g"], 3.0)
    rho = rho * (1.0 + 1e-3 * inputs.uniform_pm1(seed, nx * ny).reshape(ny, nx))
    solid = None
    if walls:
        solid = np.zeros((ny, nx), np.uint8)
        solid[0, :] = 1
        solid[ny - 1, :] = 1
    return inputs.LatticeSpec(nx, ny, tr * Tc, inputs.relax_rates(tau), eps, rho,
                              rho_ref=c["rho_g"], solid=solid)
