"""The paper's static-bubble results reproduced through the CUDA path.

Sec. 3.2 quotes the surface tension at 0.5 Tc, sigma = 0.01051, obtained from
the Laplace-law runs of Sec. 3.1 (201^2 lattices, eps = 1.86, relaxation
rates of Sec. 3.1). The printed coexistence densities fix b = 4 but not a;
the printed sigma does: a = 0.5 (as printed) gives 0.0108, a = 1 gives 0.0153.
Sec. 3.1 also states that sigma barely depends on tau_nu (0.6 vs 0.8).
"""
import json
import os

import pytest

from paper_1605_01800_gb300 import experiments

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
