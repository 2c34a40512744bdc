"""Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every computation runs in ``liblbm.so``'s CUDA kernels; this module converts
numpy arrays and PyTorch streams to the plain pointers the C functions take.
Function names are those of the header. If the library is missing the import
fails loudly; there is no CPU fallback.

``Batch`` wraps one context (a batch of independent lattices) for
convenience: ``Batch(specs, precision).init(); .step(n); .moments(i)``.
"""
import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_EINVAL = 1
LBM_ENOMEM = 2
LBM_ECUDA = 3
LBM_EPSI_DOMAIN = 4
LBM_ENONFINITE = 5
LBM_ETIMEOUT = 6

LBM_FP32_DEV = 0
LBM_FP32 = 1
LBM_FP64 = 2
LBM_INPLACE = 0x100   # OR'ed into a precision: one distribution array (lbm.h)

LBM_FLAG_PSI_CLAMPED = 1
LBM_FLAG_NONFINITE = 2
LBM_FLAG_TIMEOUT = 4

PRECISIONS = {"fp32_dev": LBM_FP32_DEV, "fp32": LBM_FP32, "fp64": LBM_FP64,
              "fp32_dev_inplace": LBM_FP32_DEV | LBM_INPLACE, "fp32_inplace": LBM_FP32 | LBM_INPLACE,
              "fp64_inplace": LBM_FP64 | LBM_INPLACE}

EXPORTED = [
    "lbm_create", "lbm_create_batch", "lbm_set_stream", "lbm_init_fields", "lbm_init_fields_all",
    "lbm_step", "lbm_read_moments", "lbm_read_moments_all", "lbm_total_mass", "lbm_status",
    "lbm_clear_status", "lbm_sync", "lbm_state_size", "lbm_save_state", "lbm_load_state",
    "lbm_tile_count", "lbm_tile_shape", "lbm_tile_kind", "lbm_set_tile", "lbm_autotune", "lbm_info",
    "lbm_last_error", "lbm_destroy", "lbm_total_mass_fp32_noalloc", "lbm_get_state_view",
    "lbm_set_open_x", "lbm_halo_pack", "lbm_halo_unpack", "lbm_total_momentum", "lbm_totals_all",
    "lbm_step_part",
]


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


LBM_EOS_CS, LBM_EOS_VDW, LBM_EOS_PR, LBM_PSI_EXP = 0, 1, 2, 3
EOS_KINDS = {"cs": LBM_EOS_CS, "vdw": LBM_EOS_VDW, "pr": LBM_EOS_PR, "psi_exp": LBM_PSI_EXP}


class lbm_eos_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
                ("T", ctypes.c_double), ("G", ctypes.c_double), ("kind", ctypes.c_int),
                ("omega", ctypes.c_double)]


class lbm_lattice_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("eos", lbm_eos_params),
                ("s", ctypes.c_double * 9), ("eps", ctypes.c_double), ("rho_ref", ctypes.c_double),
                ("wall_mask", ctypes.c_void_p)]


class lbm_info_t(ctypes.Structure):
    _fields_ = [("n_lattices", ctypes.c_int), ("precision", ctypes.c_int),
                ("nodes", ctypes.c_longlong), ("fluid_nodes", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("kernel_launches", ctypes.c_ulonglong),
                ("device_bytes", ctypes.c_size_t), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("n_tiles", ctypes.c_int), ("graph_chunk", ctypes.c_int), ("inplace", ctypes.c_int),
                ("l2_prefetch", ctypes.c_int), ("tile_grid", ctypes.c_int)]


class lbm_state_view(ctypes.Structure):
    _fields_ = [("base", ctypes.c_void_p), ("plane", ctypes.c_longlong), ("pitch", ctypes.c_int),
                ("rows", ctypes.c_int), ("x0", ctypes.c_int), ("y0", ctypes.c_int),
                ("elem_bytes", ctypes.c_int), ("deviation", ctypes.c_int), ("rho_ref", ctypes.c_double),
                ("layout", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_ctx = ctypes.c_void_p
_lib = None


def library_path() -> str:
    return os.environ.get("LBM_LIBRARY") or _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it first if allowed and needed). The
    environment variable LBM_LIBRARY names another build of it to load
    instead, e.g. the debug build (build.DEBUG_LIB), which must exist."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if os.environ.get("LBM_LIBRARY"):
        if not os.path.exists(path):
            raise RuntimeError(f"LBM_LIBRARY={path} does not exist")
    elif not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run paper_1605_01800_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    I = ctypes.c_int
    lib.lbm_create.argtypes = [I, I, ctypes.POINTER(lbm_eos_params), _dp, ctypes.c_double, _vp, I,
                               ctypes.POINTER(_ctx)]
    lib.lbm_create_batch.argtypes = [I, ctypes.POINTER(lbm_lattice_desc), I, ctypes.POINTER(_ctx)]
    lib.lbm_set_stream.argtypes = [_ctx, _vp]
    lib.lbm_init_fields.argtypes = [_ctx, I, _dp, _dp, _dp]
    lib.lbm_init_fields_all.argtypes = [_ctx, _dp, _dp, _dp]
    lib.lbm_step.argtypes = [_ctx, I]
    lib.lbm_read_moments.argtypes = [_ctx, I, _dp, _dp, _dp, _dp]
    lib.lbm_read_moments_all.argtypes = [_ctx, _dp, _dp, _dp, _dp]
    lib.lbm_total_mass.argtypes = [_ctx, I, _dp]
    lib.lbm_total_momentum.argtypes = [_ctx, I, _dp, _dp]
    lib.lbm_totals_all.argtypes = [_ctx, _dp]
    lib.lbm_status.argtypes = [_ctx, I, ctypes.POINTER(ctypes.c_uint32)]
    lib.lbm_clear_status.argtypes = [_ctx]
    lib.lbm_sync.argtypes = [_ctx]
    lib.lbm_state_size.argtypes = [_ctx, ctypes.POINTER(ctypes.c_size_t)]
    lib.lbm_save_state.argtypes = [_ctx, _vp, ctypes.c_size_t]
    lib.lbm_load_state.argtypes = [_ctx, _vp, ctypes.c_size_t]
    lib.lbm_tile_count.argtypes = []
    lib.lbm_tile_shape.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.lbm_tile_kind.argtypes = [I, ctypes.POINTER(I)]
    lib.lbm_set_tile.argtypes = [_ctx, I]
    lib.lbm_autotune.argtypes = [_ctx, I, ctypes.POINTER(I), _dp]
    lib.lbm_info.argtypes = [_ctx, ctypes.POINTER(lbm_info_t)]
    lib.lbm_get_state_view.argtypes = [_ctx, I, ctypes.POINTER(lbm_state_view)]
    lib.lbm_last_error.argtypes = []
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_total_mass_fp32_noalloc.argtypes = [_vp, I, I, ctypes.c_double, _vp, _vp, _vp]
    lib.lbm_set_open_x.argtypes = [_ctx, I, _vp]
    lib.lbm_halo_pack.argtypes = [_ctx, I, I, _vp, _vp]
    lib.lbm_halo_unpack.argtypes = [_ctx, I, I, _vp, _vp]
    lib.lbm_step_part.argtypes = [_ctx, I]
    lib.lbm_destroy.argtypes = [_ctx]
    lib.lbm_destroy.restype = None
    for name in EXPORTED:
        if name not in ("lbm_last_error", "lbm_destroy"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(rc, allow=()):
    if rc != LBM_OK and rc not in allow:
        raise LbmError(rc, load().lbm_last_error().decode())
    return rc


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


# ---------------------------------------------------------------- thin wrappers (same names as C)

def lbm_create(nx, ny, eos: lbm_eos_params, relax_rates, eps, wall_mask=None, precision=LBM_FP32_DEV):
    lib = load()
    rates = (ctypes.c_double * 9)(*relax_rates)
    mask = None if wall_mask is None else np.ascontiguousarray(wall_mask, dtype=np.uint8)
    ctx = _ctx()
    _check(lib.lbm_create(nx, ny, ctypes.byref(eos), rates, eps,
                          None if mask is None else mask.ctypes.data, precision, ctypes.byref(ctx)))
    return ctx


def lbm_create_batch(descs: Sequence[lbm_lattice_desc], precision=LBM_FP32_DEV):
    lib = load()
    arr = (lbm_lattice_desc * len(descs))(*descs)
    ctx = _ctx()
    _check(lib.lbm_create_batch(len(descs), arr, precision, ctypes.byref(ctx)))
    return ctx


def lbm_set_stream(ctx, stream_handle: int):
    _check(load().lbm_set_stream(ctx, stream_handle or None))


def lbm_init_fields(ctx, lat, rho, ux=None, uy=None):
    _check(load().lbm_init_fields(ctx, lat, _ptr(rho), _ptr(ux), _ptr(uy)))


def lbm_init_fields_all(ctx, rho, ux=None, uy=None):
    _check(load().lbm_init_fields_all(ctx, _ptr(rho), _ptr(ux), _ptr(uy)))


LBM_HALO_ROWS = 12   # values per lattice row in a packed halo (lbm.h)


def lbm_set_open_x(ctx, lat, halo_mask=None):
    """Mark lattice `lat` as an x-slab (lbm.h): halo_mask None or (4, ny) bytes."""
    hm = None
    if halo_mask is not None:
        hm = np.ascontiguousarray(halo_mask, dtype=np.uint8)
    _check(load().lbm_set_open_x(ctx, lat, None if hm is None else hm.ctypes.data))


def lbm_halo_pack(ctx, lat, side, dev_out_ptr, stream_handle=0):
    _check(load().lbm_halo_pack(ctx, lat, int(side), ctypes.c_void_p(dev_out_ptr), stream_handle or None))


def lbm_halo_unpack(ctx, lat, side, dev_in_ptr, stream_handle=0):
    _check(load().lbm_halo_unpack(ctx, lat, int(side), ctypes.c_void_p(dev_in_ptr), stream_handle or None))


def lbm_step(ctx, n):
    _check(load().lbm_step(ctx, int(n)))


LBM_STEP_EDGE = 1       # lbm_step_part: the tiles within two cells of an open x edge
LBM_STEP_INTERIOR = 2   # every other tile


def lbm_step_part(ctx, part):
    _check(load().lbm_step_part(ctx, int(part)))


def lbm_read_moments(ctx, lat, rho=None, ux=None, uy=None, p=None, allow_flags=False):
    allow = (LBM_EPSI_DOMAIN, LBM_ENONFINITE) if allow_flags else ()
    return _check(load().lbm_read_moments(ctx, lat, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(p)), allow)


def lbm_read_moments_all(ctx, rho=None, ux=None, uy=None, p=None, allow_flags=False):
    allow = (LBM_EPSI_DOMAIN, LBM_ENONFINITE) if allow_flags else ()
    return _check(load().lbm_read_moments_all(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(p)), allow)


def lbm_total_mass(ctx, lat, allow_flags=False):
    m = ctypes.c_double()
    allow = (LBM_EPSI_DOMAIN, LBM_ENONFINITE) if allow_flags else ()
    _check(load().lbm_total_mass(ctx, lat, ctypes.byref(m)), allow)
    return m.value


def lbm_total_momentum(ctx, lat, allow_flags=False):
    """(sum of rho v_x, sum of rho v_y) over the fluid nodes of lattice lat."""
    px, py = ctypes.c_double(), ctypes.c_double()
    allow = (LBM_EPSI_DOMAIN, LBM_ENONFINITE) if allow_flags else ()
    _check(load().lbm_total_momentum(ctx, lat, ctypes.byref(px), ctypes.byref(py)), allow)
    return px.value, py.value


def lbm_totals_all(ctx, n_lattices, allow_flags=False):
    """(n_lattices, 3) array: mass, momentum x, momentum y of every lattice."""
    out = np.zeros((n_lattices, 3))
    allow = (LBM_EPSI_DOMAIN, LBM_ENONFINITE) if allow_flags else ()
    _check(load().lbm_totals_all(ctx, _ptr(out)), allow)
    return out


def lbm_status(ctx, lat):
    v = ctypes.c_uint32()
    _check(load().lbm_status(ctx, lat, ctypes.byref(v)))
    return v.value


def lbm_clear_status(ctx):
    _check(load().lbm_clear_status(ctx))


def lbm_sync(ctx, allow_flags=False):
    allow = (LBM_EPSI_DOMAIN, LBM_ENONFINITE) if allow_flags else ()
    return _check(load().lbm_sync(ctx), allow)


def lbm_state_size(ctx):
    n = ctypes.c_size_t()
    _check(load().lbm_state_size(ctx, ctypes.byref(n)))
    return n.value


def lbm_save_state(ctx) -> bytes:
    n = lbm_state_size(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(load().lbm_save_state(ctx, buf, n))
    return buf.raw


def lbm_load_state(ctx, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().lbm_load_state(ctx, buf, len(blob)))


def lbm_tile_count():
    return load().lbm_tile_count()


def lbm_tile_shape(i):
    tx, ty = ctypes.c_int(), ctypes.c_int()
    _check(load().lbm_tile_shape(i, ctypes.byref(tx), ctypes.byref(ty)))
    return tx.value, ty.value


LBM_TILE_PLAIN, LBM_TILE_TMA, LBM_TILE_PIPELINED = 0, 1, 2


def lbm_tile_kind(i):
    k = ctypes.c_int()
    _check(load().lbm_tile_kind(i, ctypes.byref(k)))
    return k.value


def lbm_set_tile(ctx, i):
    _check(load().lbm_set_tile(ctx, i))


def lbm_autotune(ctx, steps):
    n = lbm_tile_count()
    ms = (ctypes.c_double * n)()
    best = ctypes.c_int()
    _check(load().lbm_autotune(ctx, steps, ctypes.byref(best), ms))
    return best.value, list(ms)


def lbm_info(ctx) -> dict:
    info = lbm_info_t()
    _check(load().lbm_info(ctx, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in lbm_info_t._fields_}


def lbm_get_state_view(ctx, lat) -> lbm_state_view:
    v = lbm_state_view()
    _check(load().lbm_get_state_view(ctx, lat, ctypes.byref(v)))
    return v


class StateArray:
    """The nine stored planes of one lattice's current state, (9, rows, pitch),
    exposed through ``__cuda_array_interface__`` (so that, e.g.,
    ``torch.as_tensor(StateArray(ctx, i), device="cuda")`` is a zero-copy view);
    node (x, y) is at ``[:, y + y0, x + x0]``. Only marshalling: the layout is the
    one lbm_get_state_view reports."""

    def __init__(self, ctx, lat):
        v = lbm_get_state_view(ctx, lat)
        self.view = v
        self.x0, self.y0 = v.x0, v.y0
        self.__cuda_array_interface__ = {
            "shape": (9, v.rows, v.pitch),
            "typestr": "<f4" if v.elem_bytes == 4 else "<f8",
            "data": (v.base, False),
            "strides": None,
            "version": 3,
            "stream": None,
        }


def lbm_last_error() -> str:
    return load().lbm_last_error().decode()


def lbm_total_mass_fp32_noalloc(f_dev_ptr, nx, ny, rho_ref, mask_dev_ptr, mass_dev_ptr, stream_handle=0):
    """Device-pointer entry point that allocates nothing (see include/lbm.h)."""
    return _check(load().lbm_total_mass_fp32_noalloc(f_dev_ptr, nx, ny, rho_ref, mask_dev_ptr or None,
                                                        mass_dev_ptr, stream_handle or None))


def lbm_destroy(ctx):
    if ctx:
        load().lbm_destroy(ctx)


# ---------------------------------------------------------------- convenience wrapper

def make_desc(spec) -> lbm_lattice_desc:
    """lbm_lattice_desc from an ``inputs.LatticeSpec`` (the mask array must be
    kept alive by the caller until lbm_create_batch returns)."""
    d = lbm_lattice_desc()
    d.nx, d.ny = spec.nx, spec.ny
    d.eos = lbm_eos_params(spec.a, spec.b, spec.R, spec.T, spec.G, EOS_KINDS[getattr(spec, "eos", "cs")],
                           getattr(spec, "omega", 0.0))
    d.s = (ctypes.c_double * 9)(*spec.s)
    d.eps = spec.eps
    d.rho_ref = spec.rho_ref
    d.wall_mask = None if spec.solid is None else spec.solid.ctypes.data
    return d


class Batch:
    """A context over a list of ``inputs.LatticeSpec`` (owns the context)."""

    def __init__(self, specs: List, precision="fp32_dev", stream=None):
        self.specs = list(specs)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        masks = [None if s.solid is None else np.ascontiguousarray(s.solid, dtype=np.uint8) for s in self.specs]
        descs = []
        for s, m in zip(self.specs, masks):
            d = make_desc(s)
            d.wall_mask = None if m is None else m.ctypes.data
            descs.append(d)
        self.ctx = lbm_create_batch(descs, self.precision)
        self.offsets = np.cumsum([0] + [s.nodes for s in self.specs])
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        handle = stream if isinstance(stream, int) else stream.cuda_stream
        lbm_set_stream(self.ctx, handle)

    def init(self, rho_list=None):
        rhos = rho_list if rho_list is not None else [s.rho for s in self.specs]
        for i, r in enumerate(rhos):
            lbm_init_fields(self.ctx, i, np.ascontiguousarray(r, dtype=np.float64))

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self, i, allow_flags=False):
        s = self.specs[i]
        out = [np.empty((s.ny, s.nx)) for _ in range(4)]
        lbm_read_moments(self.ctx, i, *out, allow_flags=allow_flags)
        return tuple(out)

    def mass(self, i, allow_flags=False):
        return lbm_total_mass(self.ctx, i, allow_flags=allow_flags)

    def momentum(self, i, allow_flags=False):
        return lbm_total_momentum(self.ctx, i, allow_flags=allow_flags)

    def totals(self, allow_flags=False):
        return lbm_totals_all(self.ctx, len(self.specs), allow_flags=allow_flags)

    def status(self, i):
        return lbm_status(self.ctx, i)

    def info(self):
        return lbm_info(self.ctx)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
