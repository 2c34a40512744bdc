"""Seeded synthetic inputs shaped like the paper's workloads (arXiv:1605.01800, Sec. 3-4).

This module is shared by the CUDA path's tests and benchmark and by the
oracle's tests. It holds no arithmetic of the lattice Boltzmann step: it
draws random numbers, lays out initial density fields (the tanh profile of
Eq. 16, uniform fields with multiplicative noise) and fills in the parameter
sets of each workload. Coexistence densities come from
``cs_coexistence.json``, written by ``oracle/write_coexistence_table.py``.

Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter
form, x_i = mix(seed + (i + 1) * 0x9E3779B97F4A7C15); a uniform double in
[0, 1) is (x_i >> 11) * 2^-53.

Workloads (all a = 1, b = 4, R = 1, G = -1, c_s^2 = 1/3):
  droplet_128         128^2 periodic static droplet, R = 25, W = 2, T = 0.8 Tc,
                      s_nu = 1, eps = 1.6
  coexistence_batch   32 flat slabs 256x64 periodic, T/Tc = 0.5 + 0.45 i / 31,
                      liquid for 64 <= x < 192, W = 5, noise x(1 + 1e-3 U(-1,1)),
                      tau_nu = 0.6, eps = 1.86
  laplace_batch       48 static droplets R_i = 10 + 70 i / 47 on square periodic
                      boxes L_i = max(128, 32 ceil(4 R_i / 32)), T = 0.6 Tc, W = 5,
                      s_nu = 1, eps = 1.6
  cavitation_1024     1024^2 periodic, uniform 0.98 x spinodal liquid density at
                      0.6 Tc, noise x(1 + 0.01 U(-1,1)), tau_nu = 0.8, eps = 1.86
  collapse_2048x1024  2048x1024, solid rows y = 0 and y = 1023, periodic in x,
                      vapour bubble R0 = 200 at (1023.5, 300) in liquid at
                      1.05 x rho_l, W = 5, T = 0.5 Tc, tau_nu = 0.6, eps = 1.86
  roofline_4096       4096^2 periodic with the physics of cavitation_1024
                      (1.2 GB of distributions, ten times the L2)
  collapse_x8         eight collapse_2048x1024 lattices in one batch (1.2 GB)
"""
import json
import math
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_TABLE = None

SEED_BASE = 1605018
GOLDEN = np.uint64(0x9E3779B97F4A7C15)


# ---------------------------------------------------------------- random numbers

def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of SplitMix64 in counter form (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    return 2.0 * uniform01(seed, n) - 1.0


# ---------------------------------------------------------------- coexistence table

def coexistence_table() -> dict:
    global _TABLE
    if _TABLE is None:
        with open(os.path.join(_HERE, "cs_coexistence.json")) as fh:
            _TABLE = json.load(fh)
    return _TABLE


def coexistence(t_over_tc: float) -> dict:
    """Row of the table at T/Tc (Maxwell rho_g, rho_l, spinodals, psi root)."""
    for row in coexistence_table()["rows"]:
        if abs(row["T_over_Tc"] - t_over_tc) < 1e-9:
            return row
    raise KeyError(f"T/Tc = {t_over_tc} is not in cs_coexistence.json")


def critical_temperature() -> float:
    return coexistence_table()["Tc"]


# ---------------------------------------------------------------- fields

def tanh_profile(nx, ny, x0, y0, r0, rho_out, rho_in, width):
    """Eq. 16 around (x0, y0): rho_in inside radius r0, rho_out outside, with
    interface width W. Eq. 16 as printed is the bubble case (vapour inside);
    a droplet swaps the two densities."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    return 0.5 * (rho_out + rho_in) + 0.5 * (rho_out - rho_in) * np.tanh(2.0 * (r - r0) / width)


def slab_profile(nx, ny, x_lo, x_hi, rho_l, rho_g, width):
    """Flat liquid slab x_lo <= x < x_hi in vapour, tanh faces of width W."""
    x = np.arange(nx, dtype=np.float64)
    prof = rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (x - x_lo) / width)
                                            - np.tanh(2.0 * (x - x_hi) / width))
    return np.tile(prof, (ny, 1))


# ---------------------------------------------------------------- workloads

def relax_rates(tau_nu: float) -> List[float]:
    """Diagonal of Lambda (Eq. 2) in the order (rho, e, zeta, j, q, j, q, nu, nu):
    1/tau_rho = 1/tau_j = 1.0, 1/tau_e = 1/tau_zeta = 1/tau_q = 1.1 (Sec. 3.1),
    1/tau_nu for the two shear moments."""
    return [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0 / tau_nu, 1.0 / tau_nu]


@dataclass
class LatticeSpec:
    nx: int
    ny: int
    T: float
    s: List[float]
    eps: float
    rho: np.ndarray                       # (ny, nx) initial density, float64
    rho_ref: float = 0.0                  # deviation reference for FP32 storage (the vapour density)
    solid: Optional[np.ndarray] = None    # (ny, nx) uint8, 1 = solid
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    G: float = -1.0
    meta: dict = field(default_factory=dict)
    eos: str = "cs"                       # psi: "cs" (Eq. 13 with Eq. 15), "vdw", "pr" (Eq. 13), "psi_exp" (Eq. 12)
    omega: float = 0.0                    # Peng-Robinson acentric factor

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


def droplet_128() -> List[LatticeSpec]:
    Tc = critical_temperature()
    c = coexistence(0.8)
    nx = ny = 128
    rho = tanh_profile(nx, ny, (nx - 1) / 2, (ny - 1) / 2, 25.0, c["rho_g"], c["rho_l"], 2.0)
    return [LatticeSpec(nx, ny, 0.8 * Tc, relax_rates(1.0), 1.6, rho, rho_ref=c["rho_g"],
                        meta={"R": 25.0, "rho_l": c["rho_l"], "rho_g": c["rho_g"]})]


def coexistence_batch(n: int = 32, nx: int = 256, ny: int = 64, config_id: int = 1) -> List[LatticeSpec]:
    Tc = critical_temperature()
    out = []
    for i in range(n):
        tr = round(0.5 + 0.45 * i / 31, 12)
        c = coexistence(tr)
        rho = slab_profile(nx, ny, nx / 4, 3 * nx / 4, c["rho_l"], c["rho_g"], 5.0)
        noise = uniform_pm1(SEED_BASE + 1000 * config_id + i, nx * ny).reshape(ny, nx)
        rho = rho * (1.0 + 1e-3 * noise)
        out.append(LatticeSpec(nx, ny, tr * Tc, relax_rates(0.6), 1.86, rho, rho_ref=c["rho_g"],
                               meta={"T_over_Tc": tr, "rho_l": c["rho_l"], "rho_g": c["rho_g"]}))
    return out


def laplace_radii(n: int = 48) -> List[float]:
    return [10.0 + 70.0 * i / (n - 1) for i in range(n)]


def laplace_box(R: float) -> int:
    return max(128, 32 * math.ceil(4.0 * R / 32.0))


def laplace_batch(n: int = 48) -> List[LatticeSpec]:
    Tc = critical_temperature()
    c = coexistence(0.6)
    out = []
    for R in laplace_radii(n):
        L = laplace_box(R)
        rho = tanh_profile(L, L, (L - 1) / 2, (L - 1) / 2, R, c["rho_g"], c["rho_l"], 5.0)
        out.append(LatticeSpec(L, L, 0.6 * Tc, relax_rates(1.0), 1.6, rho, rho_ref=c["rho_g"],
                               meta={"R": R, "rho_l": c["rho_l"], "rho_g": c["rho_g"]}))
    return out


def cavitation_1024(n: int = 1024, config_id: int = 3) -> List[LatticeSpec]:
    Tc = critical_temperature()
    c = coexistence(0.6)
    rho0 = 0.98 * c["spinodal_liquid"]
    noise = uniform_pm1(SEED_BASE + 1000 * config_id, n * n).reshape(n, n)
    rho = rho0 * (1.0 + 0.01 * noise)
    return [LatticeSpec(n, n, 0.6 * Tc, relax_rates(0.8), 1.86, rho, rho_ref=c["rho_g"],
                        meta={"rho0": rho0, "rho_c": coexistence_table()["rho_c"]})]


def roofline_4096(n: int = 4096, config_id: int = 9) -> List[LatticeSpec]:
    """The cavitation workload's physics on a 4096^2 lattice: a working set
    far larger than L2, for the sustained-bandwidth measurement."""
    return cavitation_1024(n, config_id)


def collapse_x8() -> List[LatticeSpec]:
    return collapse() * 8


def collapse(nx: int = 2048, ny: int = 1024, R0: float = 200.0, yc: float = 300.0) -> List[LatticeSpec]:
    Tc = critical_temperature()
    c = coexistence(0.5)
    rho_liq = 1.05 * c["rho_l"]
    rho = tanh_profile(nx, ny, (nx - 1) / 2, yc, R0, rho_liq, c["rho_g"], 5.0)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    rho[solid == 1] = rho_liq
    return [LatticeSpec(nx, ny, 0.5 * Tc, relax_rates(0.6), 1.86, rho, rho_ref=c["rho_g"], solid=solid,
                        meta={"R0": R0, "yc": yc, "rho_l": rho_liq, "rho_g": c["rho_g"]})]


WORKLOADS = {
    "droplet_128": droplet_128,
    "coexistence_batch": coexistence_batch,
    "laplace_batch": laplace_batch,
    "cavitation_1024": cavitation_1024,
    "collapse_2048x1024": collapse,
    "roofline_4096": roofline_4096,
    "collapse_x8": collapse_x8,
}
