"""The mass entry point that allocates nothing, against the context's own.

lbm_total_mass_fp32_noalloc serves callers that cannot allocate device memory
when they need a mass check (under an allocator that owns all device memory,
in loops that must not wait on the allocator).
It takes the FP32 distribution by device pointer; here that distribution is
the one a context holds, taken from its checkpoint blob, and its result must
equal lbm_total_mass on the same state. The file is collected last so that a
run stopping at the first failure has run every other test first.
"""
import ctypes
import struct

import numpy as np
import pytest

from paper_1605_01800_gb300 import lbm
from tests.cases import small_spec

pytestmark = pytest.mark.gpu


def _device_state(torch, b):
    """The context's FP32 distribution (one lattice) and rho_ref, on the device."""
    blob = lbm.lbm_save_state(b.ctx)
    n_lat = struct.unpack_from("<I", blob, 8)[0]
    assert n_lat == 1
    head = 16 + 8
    rho_ref = struct.unpack_from("<d", blob, head)[0]
    f_host = np.frombuffer(blob, dtype=np.float32, offset=head + 8 * n_lat)
    return torch.from_numpy(f_host.copy()).cuda(), rho_ref


def _device_mask(torch, spec):
    if spec.solid is None:
        return None
    pitch = (spec.nx + 31) // 32 * 32
    m = np.zeros((spec.ny, pitch), np.uint8)
    m[:, :spec.nx] = spec.solid
    return torch.from_numpy(m).cuda()


def test_noalloc_mass_matches_context_mass_twice_in_a_row():
    torch = pytest.importorskip("torch")
    specs = [small_spec(70, 45, walls=True, seed=11), small_spec(130, 9, seed=12)]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    expected = []
    keep = []
    for k, spec in enumerate(specs):
        b = lbm.Batch([spec], "fp32_dev")
        b.init()
        b.step(5 + k)
        expected.append(b.mass(0))
        f_dev, rho_ref = _device_state(torch, b)
        mask = _device_mask(torch, spec)
        keep.append((f_dev, mask))
        lbm.lbm_total_mass_fp32_noalloc(f_dev.data_ptr(), spec.nx, spec.ny, rho_ref,
                                        0 if mask is None else mask.data_ptr(),
                                        out[k:k + 1].data_ptr(), 0)
        b.close()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k in range(2):
        assert got[k] == pytest.approx(expected[k], rel=1e-12, abs=0), k


def test_noalloc_mass_rejects_rows_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    f = torch.zeros(9 * 32, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_total_mass_fp32_noalloc(f.data_ptr(), 1, 32769, 0.0, 0, out.data_ptr(), 0)
    assert e.value.code == lbm.LBM_EINVAL
    assert "LBM_NOALLOC_MAX_NY" in str(e.value)
