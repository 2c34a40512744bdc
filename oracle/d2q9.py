"""ctypes wrapper of the FP64 C oracle ``d2q9_oracle.c`` (test infrastructure only).

Every function follows the paper's scheme (arXiv:1605.01800, Sec. 2):
density and psi (Eq. 13, 15), force (Eq. 7), velocity (Eq. 6), MRT collision
with Li's source (Eq. 2-4, 14), streaming with periodic wrap and halfway
bounce-back (Eq. 5, Sec. 4.1). Arrays are numpy float64, f has shape
(9, ny, nx), fields (ny, nx).
"""
import ctypes
import numpy as np

from . import build as _build

Q = 9
FLAG_PSI_CLAMPED = 1
FLAG_NONFINITE = 2

_dp = ctypes.POINTER(ctypes.c_double)


class OracleParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("R", ctypes.c_double), ("T", ctypes.c_double),
                ("G", ctypes.c_double),
                ("s", ctypes.c_double * Q),
                ("eps", ctypes.c_double),
                ("solid", ctypes.c_void_p),
                ("eos", ctypes.c_int),
                ("omega", ctypes.c_double)]

EOS_KINDS = {"cs": 0, "vdw": 1, "pr": 2, "psi_exp": 3}


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        P = ctypes.POINTER(OracleParams)
        lib.oracle_moment_matrix.argtypes = [_dp, _dp]
        lib.oracle_p_eos.argtypes = [P, ctypes.c_double]
        lib.oracle_p_eos.restype = ctypes.c_double
        lib.oracle_psi.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_uint)]
        lib.oracle_psi.restype = ctypes.c_double
        lib.oracle_pressure.argtypes = [P, ctypes.c_double, ctypes.c_double]
        lib.oracle_pressure.restype = ctypes.c_double
        lib.oracle_force_from_psi.argtypes = [P, _dp, _dp, _dp]
        lib.oracle_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_collide_node.argtypes = [P, _dp, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_init.argtypes = [P, _dp, _dp, _dp, _dp]
        lib.oracle_step.argtypes = [P, _dp, _dp, ctypes.c_int]
        lib.oracle_step.restype = ctypes.c_uint
        lib.oracle_moments.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_moments.restype = ctypes.c_uint
        lib.oracle_mass.argtypes = [P, _dp]
        lib.oracle_mass.restype = ctypes.c_double
        lib.oracle_momentum.argtypes = [P, _dp, _dp, _dp, _dp]
        lib.oracle_momentum.restype = ctypes.c_uint
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_openmp.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Lattice:
    """One lattice of the oracle: parameters plus the FP64 distribution f.

    ``s`` is the diagonal of Lambda (Eq. 2) in the order
    (rho, e, zeta, j_x, q_x, j_y, q_y, p_xx, p_xy); ``eps`` is the epsilon of
    Eq. 14; ``solid`` an optional (ny, nx) uint8 mask (1 = solid node);
    ``eos`` the pseudopotential: "cs" (Eq. 13 with Eq. 15), "vdw" or "pr"
    (Eq. 13 with van der Waals or Peng-Robinson), "psi_exp" (Eq. 12 with
    the same eps); ``omega`` the Peng-Robinson acentric factor.
    """

    def __init__(self, nx, ny, a=1.0, b=4.0, R=1.0, T=0.0, G=-1.0, s=None, eps=0.0,
                 solid=None, eos="cs", omega=0.0):
        self.lib = _load()
        if s is None:
            s = [1.0] * Q
        self.nx, self.ny = int(nx), int(ny)
        self.solid = None
        if solid is not None:
            self.solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(ny, nx)
        self.p = OracleParams(self.nx, self.ny, a, b, R, T, G, (ctypes.c_double * Q)(*s),
                              eps, self.solid.ctypes.data if self.solid is not None else None,
                              EOS_KINDS[eos], omega)
        n = self.nx * self.ny
        self.f = np.zeros((Q, self.ny, self.nx))
        self._work = np.zeros((Q + 2) * n)
        self.flags = 0

    # --- thermodynamics of this lattice's parameters ---
    def p_eos(self, rho):
        return self.lib.oracle_p_eos(ctypes.byref(self.p), float(rho))

    def psi(self, rho):
        fl = ctypes.c_uint(0)
        v = self.lib.oracle_psi(ctypes.byref(self.p), float(rho), ctypes.byref(fl))
        return v, fl.value

    # --- state ---
    def init(self, rho, ux=None, uy=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ny, self.nx)
        ux = None if ux is None else np.ascontiguousarray(ux, dtype=np.float64).reshape(self.ny, self.nx)
        uy = None if uy is None else np.ascontiguousarray(uy, dtype=np.float64).reshape(self.ny, self.nx)
        self.lib.oracle_init(ctypes.byref(self.p), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(self.f))
        self.flags = 0

    def step(self, n=1):
        self.flags |= self.lib.oracle_step(ctypes.byref(self.p), _ptr(self.f), _ptr(self._work), int(n))
        return self.flags

    def moments(self):
        n = self.nx * self.ny
        shp = (self.ny, self.nx)
        rho, ux, uy, p = (np.zeros(shp) for _ in range(4))
        work = np.zeros(2 * n)
        self.lib.oracle_moments(ctypes.byref(self.p), _ptr(self.f), _ptr(work),
                                _ptr(rho), _ptr(ux), _ptr(uy), _ptr(p))
        return rho, ux, uy, p

    def mass(self):
        return self.lib.oracle_mass(ctypes.byref(self.p), _ptr(self.f))

    def momentum(self):
        """(sum of rho vx, sum of rho vy) over the fluid nodes, Eq. 6."""
        work = np.zeros(2 * self.nx * self.ny)
        px, py = ctypes.c_double(), ctypes.c_double()
        self.lib.oracle_momentum(ctypes.byref(self.p), _ptr(self.f), _ptr(work),
                                 ctypes.byref(px), ctypes.byref(py))
        return px.value, py.value

    def force_from_psi(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(self.ny, self.nx)
        Fx = np.zeros_like(psi)
        Fy = np.zeros_like(psi)
        self.lib.oracle_force_from_psi(ctypes.byref(self.p), _ptr(psi), _ptr(Fx), _ptr(Fy))
        return Fx, Fy

    def collide_node(self, f, Fx, Fy, psi, g2=0.0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(Q)
        self.lib.oracle_collide_node(ctypes.byref(self.p), _ptr(f), float(Fx), float(Fy),
                                     float(psi), float(g2), _ptr(out))
        return out


def set_threads(n: int) -> bool:
    """Run the sweeps of every lattice's step on n threads (1: serial, the
    default). Returns False if the oracle was built without OpenMP (then it
    stays serial). Results are bitwise the same for any n."""
    lib = _load()
    lib.oracle_set_threads(int(n))
    return bool(lib.oracle_openmp())


def moment_matrix():
    lib = _load()
    M = np.zeros((Q, Q))
    Minv = np.zeros((Q, Q))
    lib.oracle_moment_matrix(_ptr(M), _ptr(Minv))
    return M, Minv


def feq(rho, vx, vy):
    lib = _load()
    out = np.zeros(Q)
    lib.oracle_feq(float(rho), float(vx), float(vy), _ptr(out))
    return out


# Velocity set in the numbering of Eq. 7's weights (axis 1-4, diagonal 5-8).
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
