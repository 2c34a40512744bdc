"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/lbm.h declares; argument validation that runs before any
CUDA call. No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1605_01800_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_binding_names():
    assert sorted(lbm.EXPORTED) == declared_functions()


def test_library_exports_every_declared_symbol():
    lib = lbm.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_tile_table():
    n = lbm.lbm_tile_count()
    assert n >= 4
    shapes = [lbm.lbm_tile_shape(i) for i in range(n)]
    for tx, ty in shapes:
        assert tx % 32 == 0 and ty >= 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_tile_shape(n)
    assert e.value.code == lbm.LBM_EINVAL
    kinds = [lbm.lbm_tile_kind(i) for i in range(n)]
    assert kinds[0] == lbm.LBM_TILE_PLAIN and set(kinds) <= {0, 1, 2} and 2 in kinds
    with pytest.raises(lbm.LbmError):
        lbm.lbm_tile_kind(-1)


def _desc(**kw):
    d = lbm.lbm_lattice_desc()
    d.nx, d.ny = kw.get("nx", 8), kw.get("ny", 8)
    d.eos = lbm.lbm_eos_params(1.0, 4.0, 1.0, 0.05, kw.get("G", -1.0))
    d.s = (ctypes.c_double * 9)(*kw.get("s", [1.0] * 9))
    d.eps = 1.0
    d.rho_ref = 0.0
    d.wall_mask = None
    return d


@pytest.mark.parametrize("kw,fragment", [
    ({"nx": 0}, "nx=0"),
    ({"ny": -2}, "ny=-2"),
    ({"G": 1.0}, "G must be < 0"),
    ({"s": [1.0] * 8 + [2.0]}, "s[8]"),
    ({"nx": 60000, "ny": 60000}, "too large"),
])
def test_create_rejects_bad_parameters(kw, fragment):
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create_batch([_desc(**kw)], lbm.LBM_FP32_DEV)
    assert e.value.code == lbm.LBM_EINVAL
    assert fragment in str(e.value)


def test_precision_constants_match_the_header():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    for name in ("LBM_FP32_DEV", "LBM_FP32", "LBM_FP64", "LBM_INPLACE"):
        m = re.search(r"#define " + name + r"\s+(0x[0-9a-fA-F]+|\d+)", text)
        assert m and int(m.group(1), 0) == getattr(lbm, name), name


def test_create_rejects_an_unknown_precision():
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create_batch([_desc()], 3 | lbm.LBM_INPLACE)
    assert e.value.code == lbm.LBM_EINVAL
    assert "precision" in str(e.value)


def test_create_rejects_an_empty_batch():
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create_batch([], lbm.LBM_FP32_DEV)
    assert e.value.code == lbm.LBM_EINVAL


def test_state_view_rejects_null_arguments():
    lib = lbm.load()
    v = lbm.lbm_state_view()
    assert lib.lbm_get_state_view(None, 0, ctypes.byref(v)) == lbm.LBM_EINVAL


def test_create_rejects_unknown_precision():
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create_batch([_desc()], 7)
    assert e.value.code == lbm.LBM_EINVAL


def test_null_context_is_rejected():
    lib = lbm.load()
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert "null context" in lbm.lbm_last_error()
    assert lib.lbm_sync(None) == lbm.LBM_EINVAL
    lib.lbm_destroy(None)  # ignored


def test_binding_has_no_cpu_fallback():
    # the binding only marshals arguments: no numpy/torch arithmetic path
    src = open(os.path.join(ROOT, "paper_1605_01800_gb300", "lbm.py")).read()
    assert "oracle" not in src
