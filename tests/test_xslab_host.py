"""Host logic of the x-slab split (no GPU): the slab specs cut from a whole
lattice carry its columns, the neighbouring edge columns across each cut
(periodic in x) and the halo mask of the two columns beyond each edge."""
import numpy as np
import pytest

from paper_1605_01800_gb300 import xslab
from tests.cases import small_spec


def test_cut_takes_the_columns_across_each_edge_periodically():
    spec = small_spec(20, 9, walls=True, seed=5)
    spec.solid[4, 7] = 1   # a lone solid cell, to see which columns the halo mask takes
    slab, rho_ext, halo = xslab.cut(spec, 0, 8)
    assert slab.nx == 8 and slab.ny == 9
    assert np.array_equal(slab.rho, spec.rho[:, :8]) and np.array_equal(slab.solid, spec.solid[:, :8])
    assert rho_ext.shape == (9, 10)
    assert np.array_equal(rho_ext[:, 0], spec.rho[:, 19]) and np.array_equal(rho_ext[:, 9], spec.rho[:, 8])
    assert np.array_equal(rho_ext[:, 1:9], spec.rho[:, :8])
    assert halo.shape == (4, 9)
    for row, col in zip(halo, (18, 19, 8, 9)):
        assert np.array_equal(row, spec.solid[:, col])
    _, _, halo2 = xslab.cut(spec, 9, 20)
    assert np.array_equal(halo2[0], spec.solid[:, 7]) and halo2[0][4] == 1
    assert np.array_equal(halo2[2], spec.solid[:, 0]) and np.array_equal(halo2[3], spec.solid[:, 1])


def test_cut_without_walls_has_no_halo_mask_and_rejects_bad_bounds():
    spec = small_spec(16, 6, seed=6)
    _, _, halo = xslab.cut(spec, 3, 11)
    assert halo is None
    for a, b in ((0, 0), (5, 3), (-1, 4), (2, 17)):
        with pytest.raises(ValueError):
            xslab.cut(spec, a, b)


def test_even_cuts_cover_the_lattice():
    for nx, n in ((96, 2), (97, 3), (4, 2), (1801, 8)):
        c = xslab.even_cuts(nx, n)
        assert c[0] == 0 and c[-1] == nx and len(c) == n + 1
        w = np.diff(c)
        assert w.min() >= nx // n and w.max() <= nx // n + 1
