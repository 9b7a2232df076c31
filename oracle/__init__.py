"""FP64 CPU oracle for the D3Q27 central-Hermite MRT lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` (plus its ``--impl reference`` arm) are
the only users.  It shares no code with the CUDA path and imports nothing from
the product package.  The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64,
from the paper's definitions); this module only marshals numpy arrays.

Storage convention: dense box, cell b = x + nx*(y + ny*z); populations are
``f[b, i]`` (27 per cell) with i = 9(cz+1) + 3(cy+1) + (cx+1).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

Q = 27
THETA0 = 1.0 / 3.0
SOLID, FLUID, INLET, OUTLET = 0, 1, 2, 3
PLUG, PARABOLIC = 0, 1

_lib = None


class _Lattice(C.Structure):
    _fields_ = [
        ("flags", C.c_void_p),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("periodic", C.c_int32),
        ("omega", C.c_double),
        ("omega3", C.c_double), ("omega4", C.c_double), ("omega5", C.c_double), ("omega6", C.c_double),
        ("u_in", C.c_double), ("d_in", C.c_double), ("axis_x", C.c_double), ("axis_y", C.c_double),
        ("noise_amp", C.c_double), ("rho_out", C.c_double),
        ("seed", C.c_uint64),
        ("profile", C.c_int32), ("nthreads", C.c_int32),
        ("ramp", C.c_int32), ("reserved", C.c_int32),
        ("wall_q", C.c_void_p),
    ]


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        _lib = declare(C.CDLL(_build.build()))
    return _lib


def declare(L):
    """Declare the argument and result types of the oracle's C functions on a
    loaded library (also used by the tests that load deliberately broken
    copies of the oracle)."""
    dp = C.POINTER(C.c_double)
    L.orc_velocity.argtypes = [C.c_int, C.POINTER(C.c_int)]
    L.orc_weight.argtypes = [C.c_int]
    L.orc_weight.restype = C.c_double
    L.orc_hermite.argtypes = [C.POINTER(C.c_int), C.c_int, dp]
    L.orc_hermite.restype = C.c_double
    L.orc_hermite_m.argtypes = [C.c_int, dp]
    L.orc_hermite_m.restype = C.c_double
    L.orc_transform.argtypes = [dp, dp]
    L.orc_equilibrium.argtypes = [C.c_double, dp, dp]
    L.orc_equilibrium_tuples.argtypes = [C.c_double, dp, dp]
    L.orc_solve.argtypes = [dp, dp, C.c_int]
    L.orc_solve.restype = C.c_int
    L.orc_moments.argtypes = [dp, dp]
    L.orc_collide.argtypes = [dp, C.c_double, dp, C.c_double, dp, dp]
    L.orc_collide.restype = C.c_int
    L.orc_splitmix64.argtypes = [C.c_uint64]
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_noise.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int]
    L.orc_noise.restype = C.c_double
    L.orc_step.argtypes = [C.POINTER(_Lattice), dp, dp, dp, C.c_int64]
    L.orc_step.restype = C.c_int
    L.orc_field_moments.argtypes = [C.POINTER(_Lattice), dp, dp]
    L.orc_viscous_stress.argtypes = [dp, C.c_double, dp]
    L.orc_field_stress.argtypes = [C.POINTER(_Lattice), dp, dp]
    L.orc_totals.argtypes = [C.POINTER(_Lattice), dp, dp]
    L.orc_nee_neighbour.argtypes = [C.POINTER(_Lattice), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
    L.orc_nee_neighbour.restype = C.c_int64
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n
    return a


# ------------------------------------------------------------------ stencil

def velocities():
    """(27, 3) int array of lattice velocities."""
    out = np.zeros((Q, 3), dtype=np.int64)
    c = (C.c_int * 3)()
    for i in range(Q):
        lib().orc_velocity(i, c)
        out[i] = list(c)
    return out


def weights():
    return np.array([lib().orc_weight(i) for i in range(Q)])


def hermite(indices, xi):
    """Tensor Hermite polynomial H_{indices}(xi) (axis ids 0, 1, 2)."""
    idx = (C.c_int * max(1, len(indices)))(*indices)
    x = _vec(xi, 3)
    return lib().orc_hermite(idx, len(indices), _dp(x))


def hermite_m(m, xi):
    x = _vec(xi, 3)
    return lib().orc_hermite_m(int(m), _dp(x))


def transform(u):
    """Central Hermite transform T[m, i] = H_m(c_i - u), m = mx + 3 my + 9 mz."""
    T = np.zeros((Q, Q))
    lib().orc_transform(_dp(_vec(u, 3)), _dp(T))
    return T


def equilibrium(rho, u):
    out = np.zeros(Q)
    lib().orc_equilibrium(float(rho), _dp(_vec(u, 3)), _dp(out))
    return out


def equilibrium_tuples(rho, u):
    out = np.zeros(Q)
    lib().orc_equilibrium_tuples(float(rho), _dp(_vec(u, 3)), _dp(out))
    return out


def solve(A, b):
    A = np.array(A, dtype=np.float64, order="C")
    x = np.array(b, dtype=np.float64)
    rc = lib().orc_solve(_dp(A), _dp(x), len(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def moments(f):
    out = np.zeros(4)
    lib().orc_moments(_dp(_vec(f, Q)), _dp(out))
    return out


def collide(f, omega, ghost=(1.0, 1.0, 1.0, 1.0), omega_cons=1.0):
    """One CHM-MRT collision; returns (f_post, [rho, ux, uy, uz])."""
    fpost = np.zeros(Q)
    mom = np.zeros(4)
    g = _vec(ghost, 4)
    rc = lib().orc_collide(_dp(_vec(f, Q)), float(omega), _dp(g), float(omega_cons), _dp(fpost), _dp(mom))
    if rc != 0:
        raise np.linalg.LinAlgError("singular transform")
    return fpost, mom


def viscous_stress(f, omega):
    """sigma_ab (xx, yy, zz, xy, xz, yz) of pre-collision populations f."""
    out = np.zeros(6)
    lib().orc_viscous_stress(_dp(_vec(f, Q)), float(omega), _dp(out))
    return out


def splitmix64(x):
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def noise(seed, step, node, comp):
    return lib().orc_noise(C.c_uint64(seed), int(step), int(node), int(comp))


# ------------------------------------------------------------------ lattice

class Lattice:
    """A whole lattice advanced by the oracle.

    flags: uint8 array of shape (nz, ny, nx) (x fastest in memory).
    Parameters mirror the physical problem: omega (second-order rate),
    ghost rates, inlet profile / mean velocity / diameter / axis, inlet noise,
    outlet density.
    """

    def __init__(self, flags, omega, ghost=(1.0, 1.0, 1.0, 1.0), periodic=0,
                 profile=PLUG, u_in=0.0, d_in=None, axis=None, noise_amp=0.0, seed=0,
                 rho_out=1.0, nthreads=0, ramp=0, wall_q=None):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        assert flags.ndim == 3
        self.flags = flags
        nz, ny, nx = flags.shape
        self.shape = (nz, ny, nx)
        self.ncell = nx * ny * nz
        L = _Lattice()
        L.flags = flags.ctypes.data
        L.nx, L.ny, L.nz, L.periodic = nx, ny, nz, int(periodic)
        L.omega = float(omega)
        L.omega3, L.omega4, L.omega5, L.omega6 = (float(g) for g in ghost)
        L.u_in = float(u_in)
        L.d_in = float(d_in if d_in is not None else nx)
        ax = axis if axis is not None else (nx / 2.0, ny / 2.0)
        L.axis_x, L.axis_y = float(ax[0]), float(ax[1])
        L.noise_amp = float(noise_amp)
        L.rho_out = float(rho_out)
        L.seed = int(seed)
        L.profile = int(profile)
        L.nthreads = int(nthreads)
        L.ramp = int(ramp)
        if wall_q is not None:  # [ncell][27] uint8, q = k / 256 per wall link
            self._wall_q = np.ascontiguousarray(wall_q, dtype=np.uint8).reshape(self.ncell, Q)
            L.wall_q = self._wall_q.ctypes.data
        self._L = L
        self.f = np.zeros((self.ncell, Q))
        self.t = 0

    def init_equilibrium(self, rho, u):
        """f = f^eq(rho, u) on every active cell; rho, u scalars/3-vectors or
        per-box-cell arrays of shape (ncell,) and (ncell, 3)."""
        rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), (self.ncell,))
        u = np.broadcast_to(np.asarray(u, dtype=np.float64), (self.ncell, 3))
        active = self.flags.reshape(-1) != SOLID
        self.f[:] = 0.0
        for b in np.nonzero(active)[0]:
            self.f[b] = equilibrium(rho[b], u[b])
        self.t = 0

    def set_populations(self, f):
        self.f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ncell, Q).copy()

    def step(self, n=1):
        out = np.zeros_like(self.f)
        mom = np.zeros((self.ncell, 4))
        for _ in range(n):
            rc = lib().orc_step(C.byref(self._L), _dp(self.f), _dp(out), _dp(mom), self.t + 1)
            if rc != 0:
                raise RuntimeError("oracle step failed: %d" % rc)
            self.f, out = out, self.f
            self.t += 1
        self.last_moments = mom
        return self

    def moments(self):
        """(ncell, 4) array rho, ux, uy, uz of the current state (solid = 0)."""
        mom = np.zeros((self.ncell, 4))
        lib().orc_field_moments(C.byref(self._L), _dp(self.f), _dp(mom))
        return mom

    def field_stress(self):
        """(ncell, 6) viscous stress that the next step samples: every fluid
        cell's from its gathered populations, inlet/outlet nodes their
        partner's (solid = 0)."""
        sig = np.zeros((self.ncell, 6))
        if lib().orc_field_stress(C.byref(self._L), _dp(self.f), _dp(sig)) != 0:
            raise RuntimeError("boundary node without an interior partner")
        return sig

    def step_sampled(self, n):
        """n steps, each one sampled: time averages over those steps of u,
        u_a u_b (xx, yy, zz, xy, xz, yz), the viscous stress and rho of every
        box cell, as a dict of arrays (ncell, 3), (ncell, 6), (ncell, 6),
        (ncell,)."""
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        acc = dict(u=np.zeros((self.ncell, 3)), uu=np.zeros((self.ncell, 6)), sigma=np.zeros((self.ncell, 6)),
                   rho=np.zeros(self.ncell))
        for _ in range(n):
            acc["sigma"] += self.field_stress()
            self.step(1)
            m = self.last_moments
            acc["u"] += m[:, 1:4]
            acc["uu"] += np.stack([m[:, 1 + a] * m[:, 1 + b] for a, b in pairs], axis=1)
            acc["rho"] += m[:, 0]
        return {k: v / n for k, v in acc.items()}

    def totals(self):
        out = np.zeros(4)
        lib().orc_totals(C.byref(self._L), _dp(self.f), _dp(out))
        return out

    def nee_neighbour(self, x, y, z):
        n = (C.c_int * 3)()
        b = lib().orc_nee_neighbour(C.byref(self._L), x, y, z, n)
        return int(b), tuple(n)


def build():
    return _build.build()
