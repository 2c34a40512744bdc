"""The debug build of the library (-DLBM_DEBUG) against the release build.

In the debug build every population and wall-mask index the step kernels
touch is checked against its lattice (an index outside reads NaN, a store
outside is skipped) and every psi tile starts filled with NaN, so an offset
that strays or a psi cell that no thread writes changes the result. The debug
build must therefore give, on the parity cases (ragged, tiny, walled, batched;
every tile shape; FP32 deviation and FP64 storage), finite densities equal bit
for bit to the release build's. Each build runs in its own process (one
library per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, sys.argv[2]); sys.path.insert(0, sys.argv[3])
from paper_1605_01800_gb300 import lbm
from cases import small_spec
specs = [small_spec(70, 45, walls=True, seed=61), small_spec(19, 23, seed=62), small_spec(5, 3, seed=63),
         small_spec(130, 9, seed=64), small_spec(1, 1, seed=65), small_spec(256, 64, seed=66),
         small_spec(64, 48, walls=True, seed=67, shape="bubble")]
out = {}
for prec in ("fp32_dev", "fp64"):
    for t in range(lbm.lbm_tile_count()):
        if prec == "fp64" and lbm.lbm_tile_kind(t) != lbm.LBM_TILE_PLAIN:
            continue
        b = lbm.Batch(specs, prec)
        lbm.lbm_set_tile(b.ctx, t)
        b.init()
        b.step(7)
        n = sum(s.nodes for s in specs)
        rho = np.empty(n)
        lbm.lbm_read_moments_all(b.ctx, rho, allow_flags=True)
        out[f"{prec}_{t}"] = rho
        b.close()
np.savez(sys.argv[1], **out)
'''


def _run(lib, path):
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, path, ROOT, HERE], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(path)


def test_debug_build_matches_release_bitwise(tmp_path):
    from paper_1605_01800_gb300 import build
    debug_lib = build.build(debug=True)
    release_lib = build.build()
    dbg = _run(debug_lib, str(tmp_path / "debug.npz"))
    rel = _run(release_lib, str(tmp_path / "release.npz"))
    assert sorted(dbg.files) == sorted(rel.files) and len(rel.files) > 10
    for k in rel.files:
        assert np.all(np.isfinite(dbg[k])), k
        assert np.array_equal(dbg[k], rel[k]), k
