"""The paper's experiments reproduced through the CUDA path (a = 0.5, b = 4).

- Laplace law (Sec. 3.1, Eq. 17): the surface tension at 0.5 Tc the paper
  quotes, sigma = 0.01051 (Sec. 3.2), from static bubbles on 201^2 lattices.
  The printed coexistence densities fix b = 4 but not a; the printed sigma
  does: a = 0.5 (as printed) gives 0.0106, a = 1 gives 0.015. sigma barely
  depends on tau_nu (0.6 vs 0.8).
- Coexistence curves (Fig. 1 and 2): r0 = 70 bubbles against Maxwell and the
  oracle's Eq. 9 quadrature, for eps = 1.0, 1.86, 2.0 and tau_nu = 0.51 to 0.8.
- Cavitation inception (Fig. 4), the critical nucleus (Eq. 18, Fig. 5) and
  the collapse between two walls (Sec. 4, Fig. 7-9), qualitatively.
"""
import json
import os

import pytest

from paper_1605_01800_gb300 import experiments, inputs

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
RADII = [20, 25, 30, 40, 50]
STEPS = 60000


@pytest.fixture(scope="module")
def fits():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    return {tau: experiments.laplace_fit(RADII, 0.5, STEPS, a=0.5, tau_nu=tau, stream=s) for tau in (0.6, 0.8)}


def test_laplace_law_sigma_matches_paper(fits):
    f = fits[0.6]
    assert all(b["status"] == 0 for b in f["bubbles"])
    sigma_paper = GOLDEN["sigma_0p5Tc"]["value"]
    assert f["sigma"] == pytest.approx(sigma_paper, rel=0.06)
    # the 1/r law itself: a free linear fit in 1/r explains the data and
    # passes within 10% of the smallest bubble's dp from the origin
    assert f["r2"] > 0.97
    assert abs(f["intercept"]) < 0.1 * f["sigma"] / RADII[0]
    assert f["sigma_free"] == pytest.approx(f["sigma"], rel=0.1)


def test_sigma_independent_of_tau_nu(fits):
    assert fits[0.8]["sigma"] == pytest.approx(fits[0.6]["sigma"], rel=0.05)


def test_bubble_vapour_density_near_maxwell(fits):
    # the largest bubble's vapour within 30% of the Maxwell value the paper
    # prints (6.269e-4), far closer than the a = 1 reading (3x)
    big = max(fits[0.6]["bubbles"], key=lambda b: b["R0"])
    assert big["rho_in"] == pytest.approx(GOLDEN["rho_g_0p5Tc"]["value"], rel=0.3)


# ---------------------------------------------------------------- coexistence curves (Sec. 3.1, Fig. 1 and 2)

COEX_T = [0.6, 0.7, 0.8, 0.9]


@pytest.fixture(scope="module")
def coex():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    rows = experiments.coexistence_curve(COEX_T, [1.0, 1.86, 2.0], [0.6], 40000, stream=s)
    rows += experiments.coexistence_curve([0.5], [1.86], [0.6], 40000, stream=s)
    rows += experiments.coexistence_curve([0.5, 0.7, 0.9], [1.86], [0.51, 0.8], 40000, stream=s)
    return {(r["t_over_tc"], r["eps"], r["tau_nu"]): r for r in rows}


def _eq9(t_over_tc, eps):
    """Vapour and liquid densities of a flat interface from the oracle's
    quadrature of the mechanical-stability condition (Eq. 9), a = 0.5."""
    import warnings
    from oracle import thermo
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        Tc = thermo.critical_point(a=0.5)[0]
        g, l, _ = thermo.lb_coexistence(t_over_tc * Tc, eps, a=0.5)
    return g, l


def test_coexistence_eps_1p86_follows_maxwell(coex):
    # Fig. 1: with eps = 1.86 the simulated coexistence densities follow the
    # Maxwell construction (Eq. 11) down to 0.5 Tc
    for t in COEX_T + [0.5]:
        r = coex[(t, 1.86, 0.6)]
        assert r["status"] == 0
        c = inputs.coexistence(t)
        assert r["rho_l"] == pytest.approx(c["rho_l"], rel=5e-3)
        assert r["rho_g"] == pytest.approx(c["rho_g"], rel=0.08 if t >= 0.6 else 0.3)


def test_coexistence_vapour_follows_eq9_for_each_eps(coex):
    # the vapour densities of the GPU runs against the oracle's Eq. 9
    # quadrature (a flat interface; the r = 70 bubble's curvature lowers the
    # vapour density by a few per cent), and their order in eps
    for t in COEX_T:
        g = {e: coex[(t, e, 0.6)]["rho_g"] for e in (1.0, 1.86, 2.0)}
        for e in (1.86, 2.0):
            assert g[e] == pytest.approx(_eq9(t, e)[0], rel=0.08)
        if t >= 0.7:
            assert g[1.0] < g[1.86] < g[2.0]
        if t >= 0.8:
            assert g[1.0] == pytest.approx(_eq9(t, 1.0)[0], rel=0.08)
    # at 0.6 Tc Eq. 9 has no solution for eps = 1 (the vapour branch of the
    # quadrature runs into psi = 0) and the run leaves the EOS's domain
    with pytest.raises(ValueError):
        _eq9(0.6, 1.0)
    assert coex[(0.6, 1.0, 0.6)]["status"] != 0


def test_coexistence_independent_of_tau_nu(coex):
    # Fig. 2: tau_nu barely changes the coexistence densities
    for t, tol in ((0.7, 0.01), (0.9, 0.01), (0.5, 0.1)):
        ref = coex[(t, 1.86, 0.6)]
        for tau in (0.51, 0.8):
            r = coex[(t, 1.86, tau)]
            assert r["status"] == 0
            assert r["rho_g"] == pytest.approx(ref["rho_g"], rel=tol)
            assert r["rho_l"] == pytest.approx(ref["rho_l"], rel=1e-3)


# ---------------------------------------------------------------- cavitation inception (Sec. 3.2, Fig. 4)

def test_cavitation_inception_time_and_phases():
    """201^2 at rho_init = 0.2609, 0.5 Tc, a line perturbation of rho_init/1e8
    on row (ly-1)/2: the vapour separates there after about 180 steps and
    stays near the vapour density, run in FP64 (a 1e-8 relative seed is
    below what rho_ref + drho resolves in FP32)."""
    torch = pytest.importorskip("torch")
    h = experiments.inception_run(2000, every=5, precision="fp64", stream=torch.cuda.Stream())
    assert h["status"] == 0
    rho_c = GOLDEN["rho_c"]["value"]
    t_sep = next(t for t, c in zip(h["t"], h["centre"]) if c < rho_c)
    assert 0.7 * 180 <= t_sep <= 1.3 * 180
    assert h["centre"][h["t"].index(100)] == pytest.approx(0.2609, rel=1e-3)  # nothing visible before
    late = [c for t, c in zip(h["t"], h["centre"]) if t >= 1000]
    rho_g = GOLDEN["rho_g_0p5Tc"]["value"]
    assert max(late) < 2.5 * rho_g and min(late) > 0.5 * rho_g


# ---------------------------------------------------------------- critical nucleus (Sec. 3.2, Eq. 18, Fig. 5)

def test_critical_nucleus_radius():
    """Liquid stretched so that Eq. 18 with the printed sigma gives
    r* = 11.3: a bubble somewhat below r* condenses, one somewhat above grows
    (on 401^2, as in the paper)."""
    torch = pytest.importorskip("torch")
    import warnings
    from scipy.optimize import brentq
    from oracle import thermo
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        Tc = thermo.critical_point(a=0.5)[0]
        T = 0.5 * Tc
        _, rho_l, p0 = thermo.maxwell(T, a=0.5)
        dP = GOLDEN["sigma_0p5Tc"]["value"] / GOLDEN["critical_radius"]["value"]
        rho_L = brentq(lambda r: thermo.p_eos(r, T, a=0.5) - (p0 - dP), thermo.spinodals(T, a=0.5)[1], rho_l)
    hist = experiments.nucleus_run([9.0, 14.0], rho_L, 30000, every=10000, stream=torch.cuda.Stream())
    small, big = hist
    assert small["status"] == 0 and big["status"] == 0
    assert small["r"][-1] == 0.0                 # condensed
    assert big["r"][-1] > big["r"][0] + 1.5      # grew to a new equilibrium


# ---------------------------------------------------------------- collapse between two walls (Sec. 4, Fig. 7-9)

def test_bubble_collapse_between_walls():
    """1801 x 301, R0 = 138, d = 150 (lambda = 0.92, kappa = 0.5), 0.5 Tc,
    liquid at 1.05 rho_l: the bubble keeps its height while it shrinks
    sideways, splits into two bubbles, and the split drives jets towards the
    walls (wall-normal speed above the lateral one). Run with tau_nu = 0.6:
    at the paper's 0.51 this implementation diverges at the split, in FP64
    as in FP32."""
    torch = pytest.importorskip("torch")
    run = experiments.wall_collapse_run(3000, every=100, stream=torch.cuda.Stream(), tau_nu=0.6,
                                        liquid_factor=1.05)
    hist = run["history"]
    assert run["status"] == 0
    h0, w0 = hist[0]["height"], hist[0]["width"]
    split = next(h for h in hist if h["regions"] >= 2)
    before = [h for h in hist if h["t"] < split["t"]]
    assert all(h["regions"] == 1 and h["height"] >= 0.9 * h0 for h in before)
    assert before[-1]["width"] < 0.35 * w0
    assert split["regions"] == 2
    assert split["uy_max"] > 2.0 * split["ux_max"]
