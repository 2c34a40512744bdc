"""The paper's static-bubble experiments (arXiv:1605.01800, Sec. 3.1-3.2) on the GPU path.

- ``bubble_batch``: static vapour bubbles (Eq. 16 with vapour inside) of several
  radii on periodic square lattices, one batch.
- ``laplace_fit`` / ``laplace_series``: run a batch of bubbles (or droplets)
  through the C ABI and fit the Laplace law, Eq. 17, |p_out - p_in| = sigma / r,
  with r the equivalent radius of the inner phase's area and p of Eq. 10
  averaged in the inner half of the bubble and in the far outer phase.
- ``vapour_fraction_history``: phi(t), the fraction of nodes below the
  critical density, for the homogeneous cavitation workload.

Eq. 17 is printed as p_out - p_in = sigma / r; a bubble's inside pressure is
the higher one, so the fit uses the magnitude. The coexistence densities the
bubbles start from are those of ``cs_coexistence.json``; for fixed b and T/Tc
they do not depend on a (p_EOS scales with a at fixed T/Tc), only T_c does.
"""
from typing import List, Sequence

import numpy as np

from . import inputs, lbm


def bubble_batch(radii: Sequence[float], t_over_tc: float, a: float = 1.0, n: int = 201,
                 tau_nu: float = 0.6, eps: float = 1.86, width: float = 5.0) -> List[inputs.LatticeSpec]:
    c = inputs.coexistence(t_over_tc)
    T = t_over_tc * inputs.critical_temperature() * a  # T_c is proportional to a
    specs = []
    for R in radii:
        rho = inputs.tanh_profile(n, n, (n - 1) / 2, (n - 1) / 2, R, c["rho_l"], c["rho_g"], width)
        specs.append(inputs.LatticeSpec(n, n, T, inputs.relax_rates(tau_nu), eps, rho, rho_ref=c["rho_g"],
                                        a=a, b=4.0, meta={"R0": R, "rho_l": c["rho_l"], "rho_g": c["rho_g"]}))
    return specs


def measure_bubbles(batch: "lbm.Batch") -> List[dict]:
    """Equivalent radius, inside/outside density and pressure of each bubble.
    Pressures are averaged over the inner half of the bubble and over the
    liquid more than 15 nodes outside its interface, which removes most of
    the node-to-node oscillation of p near a sharp interface."""
    out = []
    for i, s in enumerate(batch.specs):
        rho, ux, uy, p = batch.moments(i, allow_flags=True)
        cy, cx = s.ny // 2, s.nx // 2
        rin, rout = rho[cy, cx], rho[0, 0]
        frac = np.clip((rout - rho) / (rout - rin), 0.0, 1.0)
        r_eq = float(np.sqrt(frac.sum() / np.pi))
        yy, xx = np.mgrid[0:s.ny, 0:s.nx]
        d = np.hypot(xx - (s.nx - 1) / 2, yy - (s.ny - 1) / 2)
        inner, outer = d < 0.5 * r_eq, d > r_eq + 15.0

        def mean(a, sel):
            return float(a[sel].mean()) if sel.any() else float("nan")   # nan: a run that diverged
        out.append({"R0": s.meta.get("R0", s.meta.get("R")), "r": r_eq, "rho_in": mean(rho, inner), "rho_out": mean(rho, outer),
                    "p_in": mean(p, inner), "p_out": mean(p, outer),
                    "umax": float(max(np.abs(ux).max(), np.abs(uy).max())), "status": batch.status(i)})
    return out


def fit_laplace(rows: Sequence[dict]) -> dict:
    """Fit Eq. 17 to measured bubbles or droplets: `sigma` is the
    least-squares slope of |dp| = sigma / r (a line through the origin);
    `sigma_free`, `intercept` and `r2` are the fit |dp| = sigma / r + c, whose
    small intercept and r2 near 1 show that the series obeys the 1/r law."""
    inv_r = np.array([1.0 / r["r"] for r in rows])
    dp = np.array([abs(r["p_out"] - r["p_in"]) for r in rows])
    sigma = float(np.dot(inv_r, dp) / np.dot(inv_r, inv_r))
    A = np.vstack([inv_r, np.ones_like(inv_r)]).T
    (sigma_free, intercept), *_ = np.linalg.lstsq(A, dp, rcond=None)
    pred = A @ np.array([sigma_free, intercept])
    r2 = 1.0 - float(np.sum((dp - pred) ** 2) / np.sum((dp - dp.mean()) ** 2))
    return {"sigma": sigma, "sigma_free": float(sigma_free), "intercept": float(intercept), "r2": r2,
            "bubbles": list(rows)}


def laplace_series(specs: Sequence[inputs.LatticeSpec], steps: int, precision: str = "fp32_dev",
                   stream=None, window: int = 0, every: int = 50) -> dict:
    """Run static bubbles or droplets (one batch) for `steps` steps, measure
    each (``measure_bubbles``: the inner phase is the one at the centre) and
    fit the Laplace law (``fit_laplace``). With `window` > 0 the radius and
    the two pressures are averaged over samples taken every `every` steps in
    the last `window` steps, which removes the acoustic oscillation that a
    large drop or bubble still carries when it has not yet decayed."""
    b = lbm.Batch(list(specs), precision, stream=stream)
    b.init()
    b.step(steps - window)
    samples = [measure_bubbles(b)]
    done = steps - window
    while done < steps:
        k = min(every, steps - done)
        b.step(k)
        done += k
        samples.append(measure_bubbles(b))
    b.close()
    rows = []
    for i, r0 in enumerate(samples[0]):
        row = dict(r0)
        for key in ("r", "rho_in", "rho_out", "p_in", "p_out"):
            row[key] = float(np.mean([smp[i][key] for smp in samples]))
        row["umax"] = max(smp[i]["umax"] for smp in samples)
        row["status"] = samples[-1][i]["status"]
        rows.append(row)
    return fit_laplace(rows)


def laplace_fit(radii: Sequence[float], t_over_tc: float, steps: int, a: float = 1.0, tau_nu: float = 0.6,
                eps: float = 1.86, n: int = 201, stream=None, precision: str = "fp32_dev") -> dict:
    """Static bubbles of the given radii (``bubble_batch``) run for `steps`
    steps, and the Laplace fit of ``fit_laplace``."""
    specs = bubble_batch(radii, t_over_tc, a=a, n=n, tau_nu=tau_nu, eps=eps)
    return laplace_series(specs, steps, precision=precision, stream=stream)


def vapour_fraction(rho: np.ndarray, rho_c: float) -> float:
    """Fraction of the nodes whose density is below the critical density."""
    return float(np.count_nonzero(rho < rho_c)) / rho.size


def vapour_fraction_history(spec: inputs.LatticeSpec, steps: int, every: int, precision: str = "fp32_dev",
                            stream=None) -> dict:
    """phi(t), the vapour fraction of a lattice every `every` steps."""
    rho_c = inputs.coexistence_table()["rho_c"]
    b = lbm.Batch([spec], precision, stream=stream)
    b.init()
    t, phi = [], []
    done = 0
    while True:
        rho = b.moments(0, allow_flags=True)[0]
        t.append(done)
        phi.append(vapour_fraction(rho, rho_c))
        if done >= steps:
            break
        k = min(every, steps - done)
        b.step(k)
        done += k
    status = b.status(0)
    b.close()
    return {"t": t, "phi": phi, "status": status}


def coexistence_curve(t_over_tc: Sequence[float], eps: Sequence[float], tau_nu: Sequence[float], steps: int,
                      a: float = 0.5, n: int = 201, r0: float = 70.0, width: float = 5.0, stream=None) -> List[dict]:
    """Static bubbles of radius r0 (Sec. 3.1, Fig. 1 and 2): one lattice per
    (T/Tc, eps, tau_nu), all in one batch, run for `steps` steps; returns the
    vapour density (inner half of the bubble) and the liquid density (more
    than 15 nodes outside the interface) of each."""
    combos = [(t, e, tn) for t in t_over_tc for e in eps for tn in tau_nu]
    specs = []
    for t, e, tn in combos:
        specs += bubble_batch([r0], t, a=a, n=n, tau_nu=tn, eps=e, width=width)
    b = lbm.Batch(specs, "fp32_dev", stream=stream)
    b.init()
    b.step(steps)
    rows = measure_bubbles(b)
    b.close()
    out = []
    for (t, e, tn), r in zip(combos, rows):
        out.append({"t_over_tc": t, "eps": e, "tau_nu": tn, "rho_g": r["rho_in"], "rho_l": r["rho_out"],
                    "r": r["r"], "umax": r["umax"], "status": r["status"]})
    return out


# ---------------------------------------------------------------- dynamic cases (Sec. 3.2, Sec. 4)

def inception_spec(n: int = 201, rho_init: float = 0.2609, rel_perturbation: float = -1e-8, t_over_tc: float = 0.5,
                   a: float = 0.5, tau_nu: float = 0.6, eps: float = 1.86) -> inputs.LatticeSpec:
    """Homogeneous cavitation inception (Sec. 3.2, Fig. 4): uniform density
    rho_init inside the spinodal region, changed by rho_init * rel_perturbation
    on the row (ly - 1) / 2, periodic in x and y. The paper gives the size of
    the perturbation, not its sign; a deficit is the one that makes vapour
    appear first on that row, as the paper reports."""
    T = t_over_tc * inputs.critical_temperature() * a
    rho = np.full((n, n), rho_init)
    rho[(n - 1) // 2, :] += rho_init * rel_perturbation
    return inputs.LatticeSpec(n, n, T, inputs.relax_rates(tau_nu), eps, rho, rho_ref=float(rho.min()), a=a, b=4.0,
                              meta={"rho_init": rho_init})


def inception_run(steps: int, every: int = 10, precision: str = "fp64", stream=None, **kw) -> dict:
    """Density histories at the two probes of Fig. 4: the perturbed row's
    centre ((lx-1)/2, (ly-1)/2) and ((lx-1)/2, ly-1)."""
    spec = inception_spec(**kw)
    n = spec.nx
    b = lbm.Batch([spec], precision, stream=stream)
    b.init()
    t, centre, edge, rmin = [0], [], [], []
    rho = b.moments(0, allow_flags=True)[0]
    centre.append(float(rho[(n - 1) // 2, (n - 1) // 2]))
    edge.append(float(rho[n - 1, (n - 1) // 2]))
    rmin.append(float(rho.min()))
    done = 0
    while done < steps:
        k = min(every, steps - done)
        b.step(k)
        done += k
        rho = b.moments(0, allow_flags=True)[0]
        t.append(done)
        centre.append(float(rho[(n - 1) // 2, (n - 1) // 2]))
        edge.append(float(rho[n - 1, (n - 1) // 2]))
        rmin.append(float(rho.min()))
    status = b.status(0)
    b.close()
    return {"t": t, "centre": centre, "edge": edge, "min": rmin, "status": status}


def vapour_radius(rho: np.ndarray, rho_l: float, rho_g: float) -> float:
    """Equivalent radius sqrt(A / pi) of the vapour area A: the nodes below
    the mean of rho_l and rho_g (insensitive to small drifts of the liquid
    density far from the bubble)."""
    return float(np.sqrt(np.count_nonzero(rho < 0.5 * (rho_l + rho_g)) / np.pi))


def nucleus_specs(radii: Sequence[float], rho_liquid: float, n: int = 401, t_over_tc: float = 0.5, a: float = 0.5,
                  tau_nu: float = 0.6, eps: float = 1.86, width: float = 5.0) -> List[inputs.LatticeSpec]:
    """The lattices of nucleus_run: one n x n periodic lattice per radius, a
    vapour bubble at the coexistence vapour density centred in liquid of
    density rho_liquid."""
    c = inputs.coexistence(t_over_tc)
    T = t_over_tc * inputs.critical_temperature() * a
    specs = []
    for R in radii:
        rho = inputs.tanh_profile(n, n, (n - 1) / 2, (n - 1) / 2, R, rho_liquid, c["rho_g"], width)
        specs.append(inputs.LatticeSpec(n, n, T, inputs.relax_rates(tau_nu), eps, rho, rho_ref=c["rho_g"],
                                        a=a, b=4.0, meta={"R0": R}))
    return specs


def nucleus_run(radii: Sequence[float], rho_liquid: float, steps: int, every: int = 1000, n: int = 401,
                t_over_tc: float = 0.5, a: float = 0.5, tau_nu: float = 0.6, eps: float = 1.86, width: float = 5.0,
                stream=None) -> List[dict]:
    """Critical nucleus (Sec. 3.2, Eq. 18, Fig. 5): vapour bubbles of the given
    radii at the coexistence vapour density, centred in liquid of density
    rho_liquid on n x n periodic lattices; radius histories r(t)."""
    c = inputs.coexistence(t_over_tc)
    specs = nucleus_specs(radii, rho_liquid, n, t_over_tc, a, tau_nu, eps, width)
    b = lbm.Batch(specs, "fp32_dev", stream=stream)
    b.init()
    hist = [{"R0": R, "t": [], "r": [], "rho_centre": [], "rho_liquid": []} for R in radii]
    done = 0
    while True:
        for i in range(len(radii)):
            rho = b.moments(i, allow_flags=True)[0]
            h = hist[i]
            h["t"].append(done)
            h["r"].append(vapour_radius(rho, rho_liquid, c["rho_g"]))
            h["rho_centre"].append(float(rho[(n - 1) // 2, (n - 1) // 2]))
            h["rho_liquid"].append(float(rho[0, 0]))
        if done >= steps:
            break
        k = min(every, steps - done)
        b.step(k)
        done += k
    for i, h in enumerate(hist):
        h["status"] = b.status(i)
    b.close()
    return hist


def wall_collapse_spec(nx: int = 1801, ny: int = 301, R0: float = 138.0, d: float = 150.0,
                       liquid_factor: float = 1.02, t_over_tc: float = 0.5, a: float = 0.5, tau_nu: float = 0.51,
                       eps: float = 1.86, width: float = 5.0) -> inputs.LatticeSpec:
    """Bubble collapse between two parallel walls (Sec. 4.1, Eq. 19-20):
    solid rows y = 0 and y = ny - 1 (halfway bounce-back), periodic in x, a
    vapour bubble of radius R0 centred at height d above the lower wall in
    liquid at liquid_factor times the coexistence density (the overpressure)."""
    c = inputs.coexistence(t_over_tc)
    T = t_over_tc * inputs.critical_temperature() * a
    rho_liq = liquid_factor * c["rho_l"]
    rho = inputs.tanh_profile(nx, ny, (nx - 1) / 2, d, R0, rho_liq, c["rho_g"], width)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    rho[solid == 1] = rho_liq
    return inputs.LatticeSpec(nx, ny, T, inputs.relax_rates(tau_nu), eps, rho, rho_ref=c["rho_g"], solid=solid,
                              a=a, b=4.0, meta={"R0": R0, "d": d, "rho_l": rho_liq, "rho_g": c["rho_g"]})


def _vapour_components(vap: np.ndarray) -> int:
    """Number of 4-connected vapour regions (periodic in x)."""
    from scipy import ndimage
    lab, k = ndimage.label(vap)
    if k > 1:  # merge labels that touch across the periodic x boundary
        parent = list(range(k + 1))

        def find(i):
            while parent[i] != i:
                i = parent[i]
            return i
        for l0, l1 in zip(lab[:, 0], lab[:, -1]):
            if l0 and l1:
                parent[find(l0)] = find(l1)
        k = len({find(i) for i in range(1, k + 1)})
    return k


def wall_collapse_run(steps: int, every: int = 500, stream=None, precision: str = "fp32_dev", spec=None,
                      **kw) -> dict:
    """Shape history of the collapsing bubble: vapour area, its equivalent
    radius sqrt(area / pi), lateral and vertical extent, number of vapour
    regions and the largest speeds, every `every` steps. `spec` (a lattice
    with walls and meta rho_l, rho_g) replaces the Sec. 4.1 domain."""
    if spec is None:
        spec = wall_collapse_spec(**kw)
    rl, rg = spec.meta["rho_l"], spec.meta["rho_g"]
    thr = 0.5 * (rl + rg)
    b = lbm.Batch([spec], precision, stream=stream)
    b.init()
    rows = []
    done = 0
    while True:
        rho, ux, uy, _ = b.moments(0, allow_flags=True)
        vap = (rho < thr) & (spec.solid == 0)
        ys, xs = np.nonzero(vap)
        wall = np.abs(uy[1:21, :])   # the 20 fluid rows above the lower wall
        rows.append({"t": done, "area": int(vap.sum()), "r": float(np.sqrt(vap.sum() / np.pi)),
                     "uy_wall": float(wall.max()) if np.all(np.isfinite(wall)) else float("nan"),
                     "width": int(xs.max() - xs.min() + 1) if xs.size else 0,
                     "height": int(ys.max() - ys.min() + 1) if ys.size else 0,
                     "regions": _vapour_components(vap) if xs.size else 0,
                     "uy_max": float(np.abs(uy).max()), "ux_max": float(np.abs(ux).max())})
        if done >= steps or not xs.size:
            break
        k = min(every, steps - done)
        b.step(k)
        done += k
    status = b.status(0)
    b.close()
    return {"history": rows, "status": status}
