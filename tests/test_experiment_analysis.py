"""Host-side analysis of the paper's experiments (experiments.py), on the
CPU with synthetic fields: the equivalent vapour radius and the count of
separate vapour regions (periodic in x) that the bubble-collapse history
uses, and the wall-collapse geometry."""
import numpy as np
import pytest

pytest.importorskip("scipy")

from paper_1605_01800_gb300 import experiments, inputs  # noqa: E402


def disk(n, cx, cy, r, inside, outside):
    y, x = np.mgrid[0:n, 0:n]
    return np.where((x - cx) ** 2 + (y - cy) ** 2 < r * r, inside, outside)


@pytest.mark.parametrize("r", [10.0, 25.0, 60.0])
def test_vapour_radius_of_a_disk(r):
    rho = disk(201, 100, 100, r, 0.001, 0.45)
    assert experiments.vapour_radius(rho, 0.45, 0.001) == pytest.approx(r, rel=0.02)


def test_vapour_radius_ignores_small_liquid_drift():
    rho = disk(201, 100, 100, 30.0, 0.001, 0.45) * (1 + 0.01 * np.sin(np.arange(201) / 7.0))
    assert experiments.vapour_radius(rho, 0.45, 0.001) == pytest.approx(30.0, rel=0.02)


def test_vapour_components_count_separate_regions():
    vap = np.zeros((40, 100), bool)
    assert experiments._vapour_components(vap) == 0
    vap[10:15, 20:30] = True
    assert experiments._vapour_components(vap) == 1
    vap[25:30, 50:60] = True
    assert experiments._vapour_components(vap) == 2
    # touching only diagonally: still two regions (4-connectivity)
    vap2 = np.zeros((10, 10), bool)
    vap2[2, 2] = vap2[3, 3] = True
    assert experiments._vapour_components(vap2) == 2


def test_vapour_components_merge_across_the_periodic_x_edge():
    vap = np.zeros((40, 100), bool)
    vap[10:20, 0:5] = True     # one bubble split by the x = 0 / x = nx - 1 edge
    vap[10:20, 95:100] = True
    assert experiments._vapour_components(vap) == 1
    vap[30:35, 40:45] = True
    assert experiments._vapour_components(vap) == 2


def test_wall_collapse_geometry():
    spec = experiments.wall_collapse_spec(nx=301, ny=101, R0=30.0, d=50.0)
    assert spec.solid[0].all() and spec.solid[-1].all() and not spec.solid[1:-1].any()
    c = inputs.coexistence(0.5)
    # the bubble's centre is vapour, the corners are the raised liquid
    assert spec.rho[50, 150] == pytest.approx(c["rho_g"], rel=1e-3)
    assert spec.rho[50, 0] == pytest.approx(1.02 * c["rho_l"], rel=1e-6)
    assert experiments.vapour_radius(spec.rho[1:-1], spec.meta["rho_l"], spec.meta["rho_g"]) == \
        pytest.approx(30.0, rel=0.03)
