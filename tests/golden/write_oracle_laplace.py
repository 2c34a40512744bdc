"""Surface tension of the scheme from a small static-bubble Laplace series run
through the FP64 oracle alone, for the two readings of the EOS constant a
(Sec. 3.1 prints a = 0.5, b = 1 for the CS EOS of Eq. 15; the densities the
paper prints fix b = 4, and a is then left to the surface tension it quotes,
sigma = 0.01051 at 0.5 Tc, Sec. 3.2).

Bubbles of Eq. 16 (vapour inside, W = 5) at the Maxwell densities, 0.5 Tc,
eps = 1.86, tau_nu = 0.6, G = -1, on 101 x 101 periodic lattices; after the
run p of Eq. 10 is averaged over the inner half of each bubble and over the
liquid more than 12 nodes outside its interface, the radius is the
equivalent radius of the vapour area, and sigma is the slope of
|p_in - p_out| = sigma / r through the origin (Eq. 17), with the pressures
averaged over the last `window` steps.

Writes ``oracle_laplace_sigma.json`` beside this file. Calls nothing but
``oracle/`` (the FP64 step and its Maxwell construction).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import d2q9, thermo  # noqa: E402

N = 101
RADII = (16.0, 20.0, 25.0, 30.0)
STEPS = 24000
WINDOW = 4000
EVERY = 200


def bubble(a, R, t_over_tc=0.5):
    Tc, _, _ = thermo.critical_point(a=a)
    T = t_over_tc * Tc
    rg, rl, _ = thermo.maxwell(T, a=a)
    y, x = np.mgrid[0:N, 0:N].astype(float)
    r = np.hypot(x - (N - 1) / 2, y - (N - 1) / 2)
    rho = 0.5 * (rl + rg) + 0.5 * (rl - rg) * np.tanh(2.0 * (r - R) / 5.0)
    s = [1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1 / 0.6, 1 / 0.6]
    L = d2q9.Lattice(N, N, a=a, b=4.0, R=1.0, T=T, G=-1.0, s=s, eps=1.86)
    L.init(rho)
    return L


def measure(L):
    rho, _, _, p = L.moments()
    c = N // 2
    rin, rout = rho[c, c], rho[0, 0]
    frac = np.clip((rout - rho) / (rout - rin), 0.0, 1.0)
    r_eq = float(np.sqrt(frac.sum() / np.pi))
    y, x = np.mgrid[0:N, 0:N]
    d = np.hypot(x - (N - 1) / 2, y - (N - 1) / 2)
    return r_eq, float(p[d < 0.5 * r_eq].mean()), float(p[d > r_eq + 12.0].mean())


def series(a):
    rows = []
    for R in RADII:
        L = bubble(a, R)
        L.step(STEPS - WINDOW)
        samples = [measure(L)]
        for _ in range(WINDOW // EVERY):
            L.step(EVERY)
            samples.append(measure(L))
        r, pin, pout = (float(np.mean(v)) for v in zip(*samples))
        rows.append({"R0": R, "r": r, "dp": abs(pin - pout), "flags": L.flags})
    inv_r = np.array([1.0 / q["r"] for q in rows])
    dp = np.array([q["dp"] for q in rows])
    sigma = float(np.dot(inv_r, dp) / np.dot(inv_r, inv_r))
    return {"a": a, "sigma": sigma, "bubbles": rows}


def main():
    threads = len(os.sched_getaffinity(0))
    d2q9.set_threads(threads)
    t0 = time.time()
    out = {"_source": "written by tests/golden/write_oracle_laplace.py from the FP64 oracle alone",
           "setup": {"lattice": [N, N], "radii": list(RADII), "steps": STEPS, "window": WINDOW, "every": EVERY,
                     "t_over_tc": 0.5, "eps": 1.86, "tau_nu": 0.6, "b": 4.0, "W": 5.0},
           "paper_sigma_0p5Tc": {"value": 0.01051, "cite": "Sec. 3.2, critical nucleus paragraph"},
           "series": [series(0.5), series(1.0)]}
    out["seconds"] = time.time() - t0
    with open(os.path.join(HERE, "oracle_laplace_sigma.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({s["a"]: s["sigma"] for s in out["series"]}), out["seconds"])


if __name__ == "__main__":
    main()
